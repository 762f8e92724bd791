"""Python binding of libpkmom (include/pkmom.h): argument marshalling only.

Every step of the estimator runs in the library's CUDA kernels (and cuFFT);
PyTorch provides device memory and streams. There is no CPU fallback: if the
library cannot be loaded or built, importing this module raises.

Typical use::

    from paper_2005_06170_gb300 import pkmom
    ctx = pkmom.Context(0)
    p = pkmom.params(box_L=1000.0, ng=256, nbins=128)
    out = ctx.estimate(pos, vel, p)            # pos, vel: (n,3) CUDA tensors
    P_pp = out[pkmom.ROW["P_pp"]]
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

F32, F64 = 0, 1
NROWS = 14
ROW = {"k": 0, "n_modes": 1, "P_dd": 2, "P_pp": 3, "P_tt": 4, "P_dt": 5, "P_pp_b": 6, "P_tt_b": 7,
       "P_dt_b": 8, "SN_dd": 9, "SN_pp": 10, "SN_tt": 11, "SN_pp_b": 12, "SN_tt_b": 13}
STAGES = ("hist", "scan", "scatter", "deposit", "fft", "bin", "final")
STATUS = {0: "PKMOM_OK", -1: "PKMOM_EINVAL", -2: "PKMOM_ENOMEM", -3: "PKMOM_ECUDA", -4: "PKMOM_ECUFFT",
          -5: "PKMOM_ETIMEOUT", -6: "PKMOM_EUNSUPPORTED", -7: "PKMOM_ESCRATCH", -8: "PKMOM_EDATA"}
# rows of pkmom_spectra_mu (out[row * nbins * nmu + bin * nmu + mu_bin])
MU_NROWS = 16
MU_ROW = {"k": 0, "mu": 1, "n_modes": 2, "P_dd": 3, "P_pp": 4, "P_tt": 5, "Re_dt": 6, "Im_dt": 7, "P_pp_b": 8,
          "P_tt_b": 9, "Re_dt_b": 10, "Im_dt_b": 11, "Re_dpb_b": 12, "SN_dd": 13, "SN_tt": 14, "Im_SN_dt": 15}


class Params(ctypes.Structure):
    _fields_ = [("box_L", ctypes.c_double), ("ng", ctypes.c_int), ("order", ctypes.c_int),
                ("precision", ctypes.c_int), ("nbins", ctypes.c_int), ("kmin_kf", ctypes.c_double),
                ("kmax_kf", ctypes.c_double), ("theta_scale", ctypes.c_double),
                ("subtract_shot_noise", ctypes.c_int), ("bulk", ctypes.c_int), ("theta_sn_mode", ctypes.c_int),
                ("bl_radius", ctypes.c_int)]


class Catalog(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("x", ctypes.c_void_p), ("y", ctypes.c_void_p), ("z", ctypes.c_void_p),
                ("vx", ctypes.c_void_p), ("vy", ctypes.c_void_p), ("vz", ctypes.c_void_p),
                ("mass", ctypes.c_void_p), ("stride", ctypes.c_int64), ("dtype", ctypes.c_int)]


class BatchItem(ctypes.Structure):
    _fields_ = [("cat", Catalog), ("p", Params), ("grids", ctypes.c_void_p), ("moments_dev", ctypes.c_void_p),
                ("scratch", ctypes.c_void_p), ("scratch_bytes", ctypes.c_size_t), ("out_dev", ctypes.c_void_p),
                ("deposit_tile", ctypes.c_int), ("list_cap", ctypes.c_int)]


BATCH_MAX = 128


class PkmomError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


_libs = {}


def lib(checked: bool = False):
    """Load libpkmom.so, or with checked=True libpkmom_checked.so (index tests before every
    grid, buffer and bin access), building it in-tree with nvcc if missing or stale."""
    if checked in _libs:
        return _libs[checked]
    path = _build.build(checked=checked)
    L = ctypes.CDLL(path)
    vp, i64, i32, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
    sig = {
        "pkmom_params_default": (None, [ctypes.POINTER(Params), dbl, i32, i32]),
        "pkmom_create": (i32, [ctypes.POINTER(vp), i32]),
        "pkmom_destroy": (i32, [vp]),
        "pkmom_strerror": (ctypes.c_char_p, [i32]),
        "pkmom_last_error": (ctypes.c_char_p, [vp]),
        "pkmom_grid_bytes": (ctypes.c_size_t, [i32, i32]),
        "pkmom_assign_scratch_bytes": (ctypes.c_size_t, [ctypes.POINTER(Params), i64]),
        "pkmom_footprint_bytes": (ctypes.c_size_t, [ctypes.POINTER(Params), i64]),
        "pkmom_assign": (i32, [vp, ctypes.POINTER(Catalog), ctypes.POINTER(Params), vp, vp, vp, ctypes.c_size_t, vp]),
        "pkmom_fft": (i32, [vp, ctypes.POINTER(Params), vp, vp]),
        "pkmom_spectra": (i32, [vp, ctypes.POINTER(Params), vp, vp, vp, vp]),
        "pkmom_estimate": (i32, [vp, ctypes.POINTER(Catalog), ctypes.POINTER(Params), vp, vp]),
        "pkmom_estimate_host": (i32, [vp, ctypes.POINTER(Catalog), ctypes.POINTER(Params), vp, vp]),
        "pkmom_sync": (i32, [vp, vp]),
        "pkmom_timing_enable": (i32, [vp, i32]),
        "pkmom_timing_read": (i32, [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64)]),
        "pkmom_kernel_launches": (i64, [vp]),
        "pkmom_spectra_static": (i32, [ctypes.POINTER(Params), vp, vp, vp, vp]),
        "pkmom_spectra_mu": (i32, [vp, ctypes.POINTER(Params), vp, vp, ctypes.POINTER(ctypes.c_double), i32, vp, vp]),
        "pkmom_set_tuning": (i32, [vp, i32, i32]),
        "pkmom_assign_scratch_bytes_tuned": (ctypes.c_size_t, [vp, ctypes.POINTER(Params), i64]),
        "pkmom_context_bytes": (ctypes.c_size_t, [vp]),
        "pkmom_estimate_host_async": (i32, [vp, ctypes.POINTER(Catalog), ctypes.POINTER(Params), vp, vp,
                                            ctypes.POINTER(ctypes.c_int64)]),
        "pkmom_wait": (i32, [vp, i64]),
        "pkmom_batch_work_bytes": (ctypes.c_size_t, [i32, ctypes.POINTER(BatchItem)]),
        "pkmom_estimate_batch": (i32, [vp, i32, ctypes.POINTER(BatchItem), vp, ctypes.c_size_t, vp]),
        "pkmom_checked": (i32, []),
        "pkmom_checked_selftest": (i32, [vp, vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _libs[checked] = L
    return L


EXPORTED = ("pkmom_params_default", "pkmom_create", "pkmom_destroy", "pkmom_strerror", "pkmom_last_error",
            "pkmom_grid_bytes", "pkmom_assign_scratch_bytes", "pkmom_footprint_bytes", "pkmom_assign",
            "pkmom_fft", "pkmom_spectra", "pkmom_estimate", "pkmom_estimate_host", "pkmom_sync",
            "pkmom_timing_enable", "pkmom_timing_read", "pkmom_kernel_launches", "pkmom_spectra_static",
            "pkmom_set_tuning", "pkmom_assign_scratch_bytes_tuned", "pkmom_spectra_mu", "pkmom_context_bytes",
            "pkmom_estimate_host_async", "pkmom_wait", "pkmom_batch_work_bytes", "pkmom_estimate_batch",
            "pkmom_checked", "pkmom_checked_selftest")


def params(box_L: float, ng: int, nbins: int, *, order: int = 4, precision: int = F32, kmin_kf: float = 1.0,
           kmax_kf: float | None = None, theta_scale: float = 1.0, subtract_shot_noise: bool = True,
           bulk: bool = True, theta_sn: str = "tensor", bl_radius: int = 0) -> Params:
    """bl_radius > 0: the BL function truncated to that many cells, deposited directly."""
    p = Params()
    lib().pkmom_params_default(ctypes.byref(p), float(box_L), int(ng), int(nbins))
    p.order = order
    p.precision = precision
    p.kmin_kf = kmin_kf
    p.kmax_kf = ng / 2 if kmax_kf is None else kmax_kf
    p.theta_scale = theta_scale
    p.subtract_shot_noise = int(bool(subtract_shot_noise))
    p.bulk = int(bool(bulk))
    p.theta_sn_mode = {"tensor": 0, "isotropic": 1}[theta_sn]
    p.bl_radius = int(bl_radius)
    return p


def _stream_ptr(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _dtype_code(dtype) -> int:
    import torch
    if dtype in (torch.float32, np.float32):
        return F32
    if dtype in (torch.float64, np.float64):
        return F64
    raise TypeError(f"catalogue arrays must be float32 or float64, not {dtype}")


def catalog_from_tensors(pos, vel, mass=None) -> Catalog:
    """(n,3) contiguous CUDA tensors (and an optional (n,) mass) -> device Catalog."""
    import torch
    for t in (pos, vel) + ((mass,) if mass is not None else ()):
        if not isinstance(t, torch.Tensor) or not t.is_cuda or not t.is_contiguous():
            raise ValueError("catalogue arrays must be contiguous CUDA tensors")
    if pos.dim() != 2 or pos.shape[1] != 3 or vel.shape != pos.shape or pos.dtype != vel.dtype:
        raise ValueError("pos and vel must be (n,3) tensors of the same dtype")
    es = pos.element_size()
    c = Catalog()
    c.n = pos.shape[0]
    b, v = pos.data_ptr(), vel.data_ptr()
    c.x, c.y, c.z = b, b + es, b + 2 * es
    c.vx, c.vy, c.vz = v, v + es, v + 2 * es
    c.mass = mass.data_ptr() if mass is not None else None
    c.stride = 3
    c.dtype = _dtype_code(pos.dtype)
    return c


def catalog_from_numpy(pos: np.ndarray, vel: np.ndarray, mass: np.ndarray | None = None) -> Catalog:
    """(n,3) C-contiguous host arrays -> host Catalog (for pkmom_estimate_host)."""
    for a in (pos, vel) + ((mass,) if mass is not None else ()):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("host catalogue arrays must be C-contiguous")
    if pos.ndim != 2 or pos.shape[1] != 3 or vel.shape != pos.shape or pos.dtype != vel.dtype:
        raise ValueError("pos and vel must be (n,3) arrays of the same dtype")
    es = pos.itemsize
    c = Catalog()
    c.n = pos.shape[0]
    b, v = pos.ctypes.data, vel.ctypes.data
    c.x, c.y, c.z = b, b + es, b + 2 * es
    c.vx, c.vy, c.vz = v, v + es, v + 2 * es
    c.mass = mass.ctypes.data if mass is not None else None
    c.stride = 3
    c.dtype = _dtype_code(pos.dtype.type)
    return c


class Context:
    """A libpkmom context on one CUDA device (cuFFT plans and tables are cached in it)."""

    def __init__(self, device: int = 0, checked: bool = False):
        """checked: use libpkmom_checked.so (index tests before every access)."""
        self._L = lib(checked)
        self._h = ctypes.c_void_p()
        self._check(self._L.pkmom_create(ctypes.byref(self._h), int(device)))
        self.device = device
        self.checked = bool(checked)

    def close(self):
        if self._h:
            self._L.pkmom_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, status):
        if status != 0:
            L = self._L
            msg = L.pkmom_last_error(self._h).decode() if self._h else L.pkmom_strerror(status).decode()
            raise PkmomError(status, msg)

    # -- sizes
    @staticmethod
    def grid_bytes(ng: int, precision: int = F32) -> int:
        return lib().pkmom_grid_bytes(ng, precision)

    @staticmethod
    def scratch_bytes(p: Params, n: int) -> int:
        return lib().pkmom_assign_scratch_bytes(ctypes.byref(p), n)

    @staticmethod
    def footprint_bytes(p: Params, n: int) -> int:
        return lib().pkmom_footprint_bytes(ctypes.byref(p), n)

    # -- the four calls of the C-ABI
    def assign(self, cat: Catalog, p: Params, grids, moments, scratch, stream=None):
        self._check(self._L.pkmom_assign(self._h, ctypes.byref(cat), ctypes.byref(p), grids.data_ptr(),
                                       moments.data_ptr(), scratch.data_ptr(), scratch.numel() * scratch.element_size(),
                                       _stream_ptr(stream)))

    def fft(self, p: Params, grids, stream=None):
        self._check(self._L.pkmom_fft(self._h, ctypes.byref(p), grids.data_ptr(), _stream_ptr(stream)))

    def spectra(self, p: Params, grids, moments, out, stream=None):
        self._check(self._L.pkmom_spectra(self._h, ctypes.byref(p), grids.data_ptr(), moments.data_ptr(),
                                        out.data_ptr(), _stream_ptr(stream)))

    def spectra_mu(self, p: Params, grids, moments, nmu: int, direction=None, out=None, stream=None):
        """pkmom_spectra_mu: spectra in (|k|, mu) bins; returns a (MU_NROWS, nbins * nmu)
        float64 CUDA tensor. direction: 3 numbers, or None for the bulk flow."""
        import torch
        if out is None:
            out = torch.empty((MU_NROWS, p.nbins * nmu), dtype=torch.float64, device=grids.device)
        d = None if direction is None else (ctypes.c_double * 3)(*[float(x) for x in direction])
        self._check(self._L.pkmom_spectra_mu(self._h, ctypes.byref(p), grids.data_ptr(), moments.data_ptr(), d,
                                           int(nmu), out.data_ptr(), _stream_ptr(stream)))
        return out

    def estimate_mu(self, pos, vel, p: Params, nmu: int, direction=None, mass=None, stream=None):
        """Moments, deposit and FFT (pkmom_assign, pkmom_fft) into fresh device buffers,
        then pkmom_spectra_mu; returns the (MU_NROWS, nbins * nmu) tensor."""
        import torch
        cat = catalog_from_tensors(pos, vel, mass)
        dt = torch.float32 if p.precision == F32 else torch.float64
        item = 4 if p.precision == F32 else 8
        dev = pos.device
        grids = torch.empty(Context.grid_bytes(p.ng, p.precision) // item, dtype=dt, device=dev)
        mom = torch.zeros(16, dtype=torch.float64, device=dev)
        scratch = torch.empty(self.scratch_bytes_tuned(p, cat.n), dtype=torch.uint8, device=dev)
        self.assign(cat, p, grids, mom, scratch, stream=stream)
        self.fft(p, grids, stream=stream)
        return self.spectra_mu(p, grids, mom, nmu, direction=direction, stream=stream)

    def estimate(self, pos, vel, p: Params, mass=None, out=None, stream=None):
        """All steps on device tensors; returns a (NROWS, nbins) float64 CUDA tensor."""
        import torch
        cat = catalog_from_tensors(pos, vel, mass)
        if out is None:
            out = torch.empty((NROWS, p.nbins), dtype=torch.float64, device=pos.device)
        self._check(self._L.pkmom_estimate(self._h, ctypes.byref(cat), ctypes.byref(p), out.data_ptr(),
                                         _stream_ptr(stream)))
        return out

    def estimate_host(self, pos: np.ndarray, vel: np.ndarray, p: Params, mass=None, out=None, stream=None):
        """All steps on a host catalogue (copied in by the library); returns (NROWS, nbins) numpy."""
        cat = catalog_from_numpy(pos, vel, mass)
        if out is None:
            out = np.empty((NROWS, p.nbins), dtype=np.float64)
        self._check(self._L.pkmom_estimate_host(self._h, ctypes.byref(cat), ctypes.byref(p), out.ctypes.data,
                                              _stream_ptr(stream)))
        return out

    def estimate_host_async(self, pos: np.ndarray, vel: np.ndarray, p: Params, out: np.ndarray, mass=None,
                            stream=None) -> int:
        """pkmom_estimate_host_async: queues the estimate of a host catalogue (pinned (n,3)
        arrays) whose (NROWS, nbins) result lands in `out` (a C-contiguous float64 host
        array); returns the ticket for wait(). The arrays must stay alive and unchanged
        until then."""
        cat = catalog_from_numpy(pos, vel, mass)
        if out.dtype != np.float64 or not out.flags["C_CONTIGUOUS"] or out.size < NROWS * p.nbins:
            raise ValueError("out must be a C-contiguous float64 array of NROWS * nbins values")
        t = ctypes.c_int64()
        self._check(self._L.pkmom_estimate_host_async(self._h, ctypes.byref(cat), ctypes.byref(p), out.ctypes.data,
                                                    _stream_ptr(stream), ctypes.byref(t)))
        return int(t.value)

    def wait(self, ticket: int):
        """pkmom_wait: blocks until the result of that ticket is on the host."""
        self._check(self._L.pkmom_wait(self._h, int(ticket)))

    def estimate_batch(self, items, work, stream=None):
        """pkmom_estimate_batch over a ctypes array of BatchItem (see batch_items) with a
        device work buffer of at least batch_work_bytes(items) bytes."""
        self._check(self._L.pkmom_estimate_batch(self._h, len(items), items, work.data_ptr(),
                                               work.numel() * work.element_size(), _stream_ptr(stream)))

    def sync(self, stream=None):
        self._check(self._L.pkmom_sync(self._h, _stream_ptr(stream)))

    # -- instrumentation
    def timing(self, on: bool):
        self._check(self._L.pkmom_timing_enable(self._h, int(bool(on))))

    def timing_read(self) -> dict:
        ms = (ctypes.c_double * len(STAGES))()
        calls = (ctypes.c_int64 * len(STAGES))()
        self._check(self._L.pkmom_timing_read(self._h, ms, calls))
        return {s: (ms[i], calls[i]) for i, s in enumerate(STAGES)}

    def checked_selftest(self, stream=None):
        """pkmom_checked_selftest (checked build): the next sync raises PKMOM_EDATA."""
        self._check(self._L.pkmom_checked_selftest(self._h, _stream_ptr(stream)))

    def kernel_launches(self) -> int:
        return int(self._L.pkmom_kernel_launches(self._h))

    def set_tuning(self, deposit_tile: int = -1, list_cap: int = -1):
        """Deposit tile shape and particle-list capacity (-1: automatic); see include/pkmom.h."""
        self._check(self._L.pkmom_set_tuning(self._h, int(deposit_tile), int(list_cap)))

    def scratch_bytes_tuned(self, p: Params, n: int) -> int:
        return int(self._L.pkmom_assign_scratch_bytes_tuned(self._h, ctypes.byref(p), n))

    def context_bytes(self) -> int:
        """Device bytes the context holds (cuFFT plan workspaces, tables, owned buffers)."""
        return int(self._L.pkmom_context_bytes(self._h))


def batch_items(entries):
    """entries: (catalog, params, grids, moments, scratch, out, deposit_tile, list_cap) per
    catalogue (Catalog, Params and device tensors) -> a ctypes array of BatchItem."""
    arr = (BatchItem * len(entries))()
    for it, (cat, p, grids, mom, scratch, out, tile, cap) in zip(arr, entries):
        it.cat, it.p = cat, p
        it.grids, it.moments_dev, it.scratch = grids.data_ptr(), mom.data_ptr(), scratch.data_ptr()
        it.scratch_bytes = scratch.numel() * scratch.element_size()
        it.out_dev = out.data_ptr()
        it.deposit_tile, it.list_cap = int(tile), int(cap)
    return arr


def batch_work_bytes(items) -> int:
    n = int(lib().pkmom_batch_work_bytes(len(items), items))
    if n == 0:
        raise PkmomError(-1, "invalid batch items")
    return n


def spectra_static(p: Params, grids, moments, out, stream=None):
    """pkmom_spectra_static: the binning step without any device allocation (its scratch
    is a fixed device array inside the library); see include/pkmom.h."""
    st = lib().pkmom_spectra_static(ctypes.byref(p), grids.data_ptr(), moments.data_ptr(), out.data_ptr(),
                                    _stream_ptr(stream))
    if st != 0:
        raise PkmomError(st, lib().pkmom_strerror(st).decode())


def as_mu_dict(out, nbins: int, nmu: int) -> dict:
    """(MU_NROWS, nbins * nmu) array/tensor -> {row name: (nbins, nmu) numpy array}."""
    a = out.detach().cpu().numpy() if hasattr(out, "detach") else np.asarray(out)
    return {k: a[i].reshape(nbins, nmu) for k, i in MU_ROW.items()}


def as_dict(out) -> dict:
    """(NROWS, nbins) array/tensor -> {row name: numpy array}."""
    a = out.detach().cpu().numpy() if hasattr(out, "detach") else np.asarray(out)
    return {k: a[i] for k, i in ROW.items()}


def library_path(checked: bool = False) -> str:
    return os.path.abspath(_build.LIB_CHECKED if checked else _build.LIB)
