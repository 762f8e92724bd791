"""Host code under AddressSanitizer and UndefinedBehaviorSanitizer, on the CPU.

* The oracle's C deposit (oracle/deposit.c) on edge-case positions (0, L, beyond L,
  negative, far outside), orders 1-5 and four fields; field totals conserved.
* The binning's host-side shell tables and work-item list (csrc/shells.cu, plain C++)
  against brute force over every mode of small half spectra.
* The host-side entry points of the C-ABI (include/pkmom.h): defaults, scratch sizes and
  footprints over the parameter ranges, batch work sizes, argument errors, and context
  creation failing cleanly without a GPU. The library's CUDA sources are compiled with
  their host code instrumented (the device code as usual).
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HERE = os.path.join(ROOT, "tests", "sanitize")
SAN = ["-fsanitize=address,undefined", "-fno-sanitize-recover=all", "-fno-omit-frame-pointer", "-g"]


def _run(cmd, env=None, cwd=None):
    r = subprocess.run(cmd, capture_output=True, text=True, env=env, cwd=cwd, timeout=900)
    assert r.returncode == 0, f"{' '.join(cmd)}\n{r.stdout[-3000:]}\n{r.stderr[-3000:]}"
    return r


def test_oracle_deposit_under_sanitizers(tmp_path):
    if not shutil.which("gcc"):
        pytest.skip("gcc not found")
    exe = str(tmp_path / "deposit_san")
    _run(["gcc", "-O1", "-std=c99", *SAN, "-o", exe, os.path.join(HERE, "deposit_main.c"),
          os.path.join(ROOT, "oracle", "deposit.c"), "-lm"])
    r = _run([exe], env=dict(os.environ, ASAN_OPTIONS="detect_leaks=1", UBSAN_OPTIONS="print_stacktrace=1"))
    assert "deposit ok" in r.stdout


def test_shell_tables_and_item_list_under_sanitizers(tmp_path):
    gxx = shutil.which("g++")
    if not gxx:
        pytest.skip("g++ not found")
    exe = str(tmp_path / "shells_san")
    csrc = os.path.join(ROOT, "paper_2005_06170_gb300", "csrc")
    _run([gxx, "-O1", "-std=c++17", *SAN, "-I", csrc, "-o", exe, "-x", "c++", os.path.join(csrc, "shells.cu"),
          "-x", "c++", os.path.join(HERE, "shells_main.cpp")])
    r = _run([exe], env=dict(os.environ, ASAN_OPTIONS="detect_leaks=1", UBSAN_OPTIONS="print_stacktrace=1"))
    assert "shells ok" in r.stdout


@pytest.mark.slow
def test_capi_host_code_under_sanitizers(tmp_path):
    from paper_2005_06170_gb300 import build
    nv = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nv) or not shutil.which("gcc"):
        pytest.skip("nvcc or gcc not found")
    inc = ["-I", os.path.join(ROOT, "include")]
    # one -Xcompiler per flag (nvcc splits its argument at commas)
    host_san = []
    for f in ["-fsanitize=address", "-fsanitize=undefined", "-fno-sanitize-recover=all", "-fno-omit-frame-pointer"]:
        host_san += ["-Xcompiler", f]
    objs = []
    procs = []
    for src in build.sources():
        obj = str(tmp_path / (os.path.basename(src)[:-3] + ".o"))
        objs.append(obj)
        procs.append(subprocess.Popen([nv, *build.ARCH, "-O1", "-std=c++17", "-Xcompiler", "-fPIC",
                                       "--expt-relaxed-constexpr", *host_san, *inc, "-c", src, "-o", obj],
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    for p in procs:
        out, err = p.communicate(timeout=900)
        assert p.returncode == 0, err[-3000:]
    main_obj = str(tmp_path / "capi_main.o")
    _run(["gcc", "-O1", "-std=c99", *SAN, *inc, "-c", os.path.join(HERE, "capi_main.c"), "-o", main_obj])
    exe = str(tmp_path / "capi_san")
    _run([nv, *build.ARCH, *host_san, "-o", exe, main_obj, *objs, "-lcufft", "-lcudart"])
    env = dict(os.environ, ASAN_OPTIONS="detect_leaks=0:protect_shadow_gap=0", UBSAN_OPTIONS="print_stacktrace=1",
               CUDA_VISIBLE_DEVICES="")
    r = _run([exe], env=env)
    assert "capi ok" in r.stdout
