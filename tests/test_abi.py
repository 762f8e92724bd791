"""The C-ABI library builds for sm_103a, loads, and exports every entry point that
include/pkmom.h declares; host-side argument handling works without a GPU."""
import ctypes
import os
import re

import pytest

from paper_2005_06170_gb300 import pkmom

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "pkmom.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pkmom_[a-z0-9_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    L = pkmom.lib()
    names = declared_symbols()
    assert len(names) >= 15
    for name in names:
        assert hasattr(L, name), name
    assert set(names) == set(pkmom.EXPORTED)


def test_build_targets_sm_103a_only():
    from paper_2005_06170_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_params_default_and_sizes():
    p = pkmom.params(1000.0, 256, 128)
    assert p.order == 4 and p.nbins == 128 and p.kmax_kf == 128 and p.subtract_shot_noise == 1
    assert pkmom.Context.grid_bytes(256, pkmom.F32) == 4 * 256 * 256 * 258 * 4
    assert pkmom.Context.grid_bytes(64, pkmom.F64) == 4 * 64 * 64 * 66 * 8
    s = pkmom.Context.scratch_bytes(p, 256 ** 3)
    assert s >= 256 ** 3 * (32 + 4)
    assert pkmom.Context.footprint_bytes(p, 256 ** 3) > s + pkmom.Context.grid_bytes(256, 0)


@pytest.mark.parametrize("bad", [dict(ng=20), dict(ng=8), dict(nbins=0), dict(kmax_kf=200.0), dict(order=6),
                                 dict(box_L=-1.0), dict(bl_radius=1), dict(bl_radius=5),
                                 dict(order=3, bl_radius=2)])
def test_invalid_params_have_no_scratch_size(bad):
    kw = dict(box_L=100.0, ng=64, nbins=8)
    kw.update({k: v for k, v in bad.items() if k in kw})
    p = pkmom.params(**kw)
    for k, v in bad.items():
        setattr(p, k, v)
    assert pkmom.Context.scratch_bytes(p, 1000) == 0


def test_strerror_names_every_status():
    L = pkmom.lib()
    for code in pkmom.STATUS:
        assert L.pkmom_strerror(code).decode() != "unknown status"


def test_create_without_device_fails_cleanly():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    assert pkmom.lib().pkmom_create(ctypes.byref(h), 0) != 0
    assert not h.value


def test_checked_library_exports_the_same_symbols():
    Lc = pkmom.lib(checked=True)
    for name in declared_symbols():
        assert hasattr(Lc, name), name
    assert Lc.pkmom_checked() == 1
    assert pkmom.lib().pkmom_checked() == 0
