"""GB300-native RAS/ORAS-preconditioned FGMRES for the closest point method.

Python binding of the C ABI in include/cpm.h (method: May, Haynes & Ruuth,
arXiv:1909.08734).  The functions below only marshal arguments: device vectors are torch
CUDA tensors (FP64, contiguous), streams are torch.cuda.Stream objects (or None), and every
computation runs in the library's own CUDA kernels.  Importing this package does not touch
the GPU; the first call loads ``libcpm_gb300.so`` and raises if it has not been built.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import _capi
from ._capi import (CPM_BF16, CPM_FP32, CPM_FP64, CPM_ORAS, CPM_ORAS_R3, CPM_RAS,  # noqa: F401
                    CPM_SET_BC_A, CPM_SET_BC_G, CPM_SET_BC_GEN, CPM_SET_BC_NEARX, CPM_SET_GHOST,
                    CPM_SET_LAST, CPM_SET_OWN, CPM_SET_SIGMA, CPM_SPHERE, CPM_TORUS,
                    CPM_TRIMESH)

PRECISIONS = {"fp64": CPM_FP64, "fp32": CPM_FP32, "bf16": CPM_BF16}
TRANSMISSIONS = {"ras": CPM_RAS, "oras": CPM_ORAS, "oras_r3": CPM_ORAS_R3}
SURFACES = {"sphere": CPM_SPHERE, "torus": CPM_TORUS, "trimesh": CPM_TRIMESH}


class CpmError(RuntimeError):
    def __init__(self, status: int, where: str):
        lib = _capi.load()
        self.status = status
        name = lib.cpm_status_string(status).decode()
        msg = lib.cpm_last_error().decode()
        super().__init__(f"{where}: {name}: {msg}")


# outcomes reported per right-hand side (returned in the result list when not raising)
_PER_RHS_STATUS = (_capi.CPM_ERR_NOT_CONVERGED, _capi.CPM_ERR_BREAKDOWN, _capi.CPM_ERR_NAN,
                   _capi.CPM_ERR_TIMEOUT)


def _check(st: int, where: str):
    if st != 0:
        raise CpmError(st, where)


def _stream_ptr(stream):
    if stream is None:
        return None
    return C.c_void_p(stream.cuda_stream)


def _dev_ptr(t, n: int, name: str):
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise TypeError(f"{name} must be a contiguous float64 CUDA tensor")
    if t.numel() < n:
        raise ValueError(f"{name} has {t.numel()} entries, needs {n}")
    return C.c_void_p(t.data_ptr())


class Band:
    def __init__(self, handle):
        self._h = handle

    def __del__(self):
        if getattr(self, "_h", None):
            _capi.load().cpm_band_destroy(self._h)
            self._h = None

    @property
    def handle(self):
        return self._h

    def sizes(self) -> tuple[int, int, int]:
        """(N_A, N_G, p) without copying the band's arrays."""
        inf = _capi.cpm_band_info()
        _check(_capi.load().cpm_band_info_get(self._h, C.byref(inf)), "cpm_band_info_get")
        return int(inf.n_active), int(inf.n_ghost), int(inf.p)

    def info(self) -> dict:
        inf = _capi.cpm_band_info()
        _check(_capi.load().cpm_band_info_get(self._h, C.byref(inf)), "cpm_band_info_get")
        n = inf.n_active + inf.n_ghost
        arr = lambda p, cnt, dt: np.ctypeslib.as_array(p, shape=(cnt,)).astype(dt, copy=True)  # noqa: E731
        return {
            "n_active": inf.n_active, "n_ghost": inf.n_ghost, "p": inf.p, "h": inf.h,
            "lambda": inf.lambda_,
            "ijk": arr(inf.ijk, 3 * n, np.int64).reshape(n, 3),
            "cp": arr(inf.cp, 3 * n, np.float64).reshape(n, 3),
            "nbr": arr(inf.nbr, 6 * inf.n_active, np.int64).reshape(inf.n_active, 6),
            "base": arr(inf.base, 3 * n, np.int64).reshape(n, 3),
            "pencil": arr(inf.pencil, n * (inf.p + 1) ** 2, np.int32).reshape(n, (inf.p + 1) ** 2),
            "weights": arr(inf.weights, n * 3 * (inf.p + 1), np.float64).reshape(n, 3, inf.p + 1),
            "tri": arr(inf.tri, n, np.int64) if inf.tri else None,
        }


class Partition:
    def __init__(self, handle, band: Band, n_sub: int):
        self._h = handle
        self.band = band          # keeps the band alive
        self.n_sub = n_sub

    def __del__(self):
        if getattr(self, "_h", None):
            _capi.load().cpm_partition_destroy(self._h)
            self._h = None

    @property
    def handle(self):
        return self._h

    def labels(self) -> np.ndarray:
        p = C.POINTER(C.c_int32)()
        _check(_capi.load().cpm_partition_labels(self._h, C.byref(p)), "cpm_partition_labels")
        n = self.band.info()["n_active"]
        return np.ctypeslib.as_array(p, shape=(n,)).astype(np.int64)

    def set(self, j: int, which: int) -> np.ndarray:
        p = C.POINTER(C.c_int32)()
        n = C.c_int64()
        _check(_capi.load().cpm_partition_set(self._h, j, which, C.byref(p), C.byref(n)),
               "cpm_partition_set")
        if n.value == 0:
            return np.zeros(0, dtype=np.int64)
        return np.ctypeslib.as_array(p, shape=(n.value,)).astype(np.int64)

    def cross_points(self) -> np.ndarray:
        p = C.POINTER(C.c_int32)()
        n = C.c_int64()
        _check(_capi.load().cpm_partition_cross_points(self._h, C.byref(p), C.byref(n)),
               "cpm_partition_cross_points")
        if n.value == 0:
            return np.zeros(0, dtype=np.int64)
        return np.ctypeslib.as_array(p, shape=(n.value,)).astype(np.int64)


class Preconditioner:
    def __init__(self, handle, band: Band, part: Partition):
        self._h = handle
        self.band = band
        self.part = part

    def __del__(self):
        if getattr(self, "_h", None):
            _capi.load().oras_destroy(self._h)
            self._h = None

    @property
    def handle(self):
        return self._h

    def info(self) -> dict:
        inf = _capi.oras_info()
        _check(_capi.load().oras_info_get(self._h, C.byref(inf)), "oras_info_get")
        return {f: getattr(inf, f) for f, _ in _capi.oras_info._fields_}

    def local_sizes(self) -> np.ndarray:
        out = np.zeros(self.part.n_sub, dtype=np.int64)
        _check(_capi.load().oras_local_sizes(self._h, out.ctypes.data_as(C.c_void_p)), "oras_local_sizes")
        return out

    @property
    def n_active(self) -> int:
        return self.info()["n_active"]


# ---------------------------------------------------------------- entry points
def cpm_build_band(surface: str, R: float, r: float, h: float, p: int,
                   lambda_over_h: float = 0.0, verts=None, tris=None,
                   construction: str = "tube", on_device: bool = False, stream=None) -> Band:
    """Band of a sphere / torus (R, r) or of a triangulated surface (verts (n,3), tris (m,3));
    construction "tube" (radius lambda_over_h * h) or "algorithmic" (interpolation closure).
    on_device: build the tube band on the current CUDA device (cpm_build_band_device; the same
    band bit for bit, its device copies left resident)."""
    s = _capi.cpm_surface(SURFACES[surface], float(R), float(r))
    if surface == "trimesh":
        V = np.ascontiguousarray(verts, dtype=np.float64)
        T = np.ascontiguousarray(tris, dtype=np.int32)
        if V.ndim != 2 or V.shape[1] != 3 or T.ndim != 2 or T.shape[1] != 3:
            raise ValueError("cpm_build_band: verts (n,3) and tris (m,3) expected")
        s.verts = V.ctypes.data_as(C.POINTER(C.c_double))
        s.n_verts = V.shape[0]
        s.tris = T.ctypes.data_as(C.POINTER(C.c_int32))
        s.n_tris = T.shape[0]
    h_out = C.c_void_p()
    if on_device and construction != "tube":
        raise ValueError("on_device builds the tube band only")
    if construction == "algorithmic":
        _check(_capi.load().cpm_build_band_algorithmic(C.byref(s), float(h), int(p), C.byref(h_out)),
               "cpm_build_band_algorithmic")
    elif construction == "tube" and on_device:
        _check(_capi.load().cpm_build_band_device(C.byref(s), float(h), int(p), float(lambda_over_h),
                                                  _stream_ptr(stream), C.byref(h_out)), "cpm_build_band_device")
    elif construction == "tube":
        _check(_capi.load().cpm_build_band(C.byref(s), float(h), int(p), float(lambda_over_h),
                                           C.byref(h_out)), "cpm_build_band")
    else:
        raise ValueError(construction)
    return Band(h_out)


def cpm_partition(band: Band, n_sub: int, leaf_weights=None, n_overlap: int = 2,
                  align_passes: int = 0, split: str = "coordinate") -> Partition:
    """split: "coordinate" (recursive coordinate bisection, cpm_partition) or "graph"
    (recursive graph bisection of the active 6-neighbour graph, cpm_partition_graph)."""
    if split not in ("coordinate", "graph"):
        raise ValueError('split must be "coordinate" or "graph"')
    lib = _capi.load()
    wptr = None
    if leaf_weights is not None:
        w = np.ascontiguousarray(leaf_weights, dtype=np.int64)
        if len(w) != n_sub:
            raise ValueError("leaf_weights must have n_sub entries")
        wptr = w.ctypes.data_as(C.POINTER(C.c_int64))
    h_out = C.c_void_p()
    fn, name = (lib.cpm_partition, "cpm_partition") if split == "coordinate" else \
        (lib.cpm_partition_graph, "cpm_partition_graph")
    _check(fn(band.handle, int(n_sub), wptr, int(n_overlap), int(align_passes), C.byref(h_out)), name)
    return Partition(h_out, band, n_sub)


def cpm_partition_from_labels(band: Band, labels, n_overlap: int = 2, n_sub: int | None = None) -> Partition:
    """Partition from caller-supplied labels (one per active node, in [0, n_sub))."""
    lab = np.ascontiguousarray(labels, dtype=np.int32)
    n_active = band.sizes()[0]
    if lab.ndim != 1 or lab.size != n_active:
        raise ValueError(f"labels must be a 1-D array of {n_active} entries (one per active node), "
                         f"got shape {lab.shape}")
    if n_sub is None:
        n_sub = int(lab.max()) + 1 if lab.size else 0
    h_out = C.c_void_p()
    _check(_capi.load().cpm_partition_from_labels(band.handle, int(n_sub), lab.ctypes.data_as(C.c_void_p),
                                                  int(n_overlap), C.byref(h_out)), "cpm_partition_from_labels")
    return Partition(h_out, band, int(n_sub))


def cpm_partition_save(part: Partition, path: str) -> None:
    _check(_capi.load().cpm_partition_save(part.handle, os.fsencode(path)), "cpm_partition_save")


def cpm_partition_load(band: Band, path: str) -> Partition:
    h_out = C.c_void_p()
    _check(_capi.load().cpm_partition_load(band.handle, os.fsencode(path), C.byref(h_out)), "cpm_partition_load")
    p = Partition(h_out, band, 0)
    p.n_sub = int(p.labels().max()) + 1       # every subdomain is non-empty
    return p


def cpm_local_coo(band: Band, part: Partition, c: float, transmission: str, alpha: float,
                  alpha_x: float, j: int):
    lib = _capi.load()
    n = C.c_int64()
    nnz = C.c_int64()
    tr = TRANSMISSIONS[transmission]
    _check(lib.cpm_local_coo(band.handle, part.handle, float(c), tr, float(alpha), float(alpha_x),
                             int(j), C.byref(n), C.byref(nnz), None, None, None), "cpm_local_coo")
    rows = np.zeros(nnz.value, np.int32)
    cols = np.zeros(nnz.value, np.int32)
    vals = np.zeros(nnz.value, np.float64)
    _check(lib.cpm_local_coo(band.handle, part.handle, float(c), tr, float(alpha), float(alpha_x),
                             int(j), C.byref(n), C.byref(nnz), rows.ctypes.data_as(C.c_void_p),
                             cols.ctypes.data_as(C.c_void_p), vals.ctypes.data_as(C.c_void_p)),
           "cpm_local_coo")
    return n.value, rows, cols, vals


def cpm_local_order(band: Band, part: Partition, c: float, transmission: str, alpha: float,
                    alpha_x: float, j: int):
    """(perm, first, last, pend) of local operator j: see include/cpm.h."""
    lib = _capi.load()
    n = C.c_int64()
    T = C.c_int()
    tr = TRANSMISSIONS[transmission]
    args = (band.handle, part.handle, float(c), tr, float(alpha), float(alpha_x), int(j), C.byref(n), C.byref(T))
    _check(lib.cpm_local_order(*args, None, None, None, None), "cpm_local_order")
    perm = np.zeros(n.value, np.int32)
    first = np.zeros(64 * T.value, np.int32)
    last = np.zeros(64 * T.value, np.int32)
    pend = np.zeros(T.value, np.int32)
    _check(lib.cpm_local_order(*args, *(x.ctypes.data_as(C.c_void_p) for x in (perm, first, last, pend))),
           "cpm_local_order")
    return perm, first, last, pend


def oras_setup(band: Band, part: Partition, c: float, transmission: str = "oras",
               alpha: float = 4.0, alpha_x: float = 40.0, precision: str = "fp64",
               stream=None, simt_lu: bool = False) -> Preconditioner:
    """simt_lu=True runs the LU trailing updates on the CUDA cores (validation reference)."""
    h_out = C.c_void_p()
    prec = PRECISIONS[precision] | (_capi.CPM_SETUP_SIMT_LU if simt_lu else 0)
    _check(_capi.load().oras_setup(band.handle, part.handle, float(c), TRANSMISSIONS[transmission],
                                   float(alpha), float(alpha_x), prec,
                                   _stream_ptr(stream), C.byref(h_out)), "oras_setup")
    return Preconditioner(h_out, band, part)


def oras_setup_selftest_singular(band: Band, part: Partition, c: float, transmission: str, alpha: float,
                                 alpha_x: float, precision: str, subdomain: int, stream=None):
    """Set-up with local column 0 of one subdomain's matrix zeroed; returns (status, message)."""
    st = _capi.load().oras_setup_selftest_singular(band.handle, part.handle, float(c), TRANSMISSIONS[transmission],
                                                    float(alpha), float(alpha_x), PRECISIONS[precision],
                                                    int(subdomain), _stream_ptr(stream))
    return int(st), _capi.load().cpm_last_error().decode()


def oras_plan(band: Band, part: Partition, transmission: str = "oras", precision: str = "fp64",
              restart: int = 50, nrhs: int = 1) -> dict:
    """Host-side device-memory plan of oras_setup + solves (bytes); touches no GPU."""
    out = _capi.oras_plan_info()
    _check(_capi.load().oras_plan(band.handle, part.handle, TRANSMISSIONS[transmission],
                                  PRECISIONS[precision], int(restart), int(nrhs), C.byref(out)),
           "oras_plan")
    return {f: getattr(out, f) for f, _ in _capi.oras_plan_info._fields_}


def cpm_op_apply(pc: Preconditioner, x, y, nrhs: int = 1, stream=None):
    n = pc.n_active * nrhs
    _check(_capi.load().cpm_op_apply(pc.handle, _dev_ptr(x, n, "x"), _dev_ptr(y, n, "y"), int(nrhs),
                                     _stream_ptr(stream)), "cpm_op_apply")


CPM_NOALLOC_MAX_NODES = 1 << 20


def cpm_op_apply_noalloc(pencil, weights, nbr, n_active: int, n_nodes: int, p: int, c: float,
                         h: float, x, y, stream=None):
    """y = A x for callers that cannot allocate device memory: every argument is caller-owned
    device memory (torch CUDA tensors: pencil int32, weights float64, nbr int32, x / y
    float64); the library's scratch is a static device array, looked up on the first call
    per device.  Calls that overlap on the GPU race on that shared array.  Sizes, dtypes and
    devices are checked here, before any launch; the index values (pencil starts, neighbours)
    must be the band's own (cpm_band_info), as they are read without bounds checks."""
    import torch
    P = int(p) + 1
    dev = torch.cuda.current_device()
    need = {"pencil": int(n_nodes) * P * P, "weights": 3 * P * int(n_nodes), "nbr": 6 * int(n_active),
            "x": int(n_active), "y": int(n_active)}
    for t, dt, name in ((pencil, torch.int32, "pencil"), (weights, torch.float64, "weights"),
                        (nbr, torch.int32, "nbr"), (x, torch.float64, "x"), (y, torch.float64, "y")):
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == dt and t.is_contiguous()):
            raise TypeError(f"{name} must be a contiguous {dt} CUDA tensor")
        if t.device.index != dev:
            raise ValueError(f"{name} is on cuda:{t.device.index}, the current device is cuda:{dev}")
        if t.numel() < need[name]:
            raise ValueError(f"{name} has {t.numel()} entries, needs {need[name]} for n_active = {n_active}, "
                             f"n_nodes = {n_nodes}, p = {p}")
    _check(_capi.load().cpm_op_apply_noalloc(
        C.c_void_p(pencil.data_ptr()), C.c_void_p(weights.data_ptr()), C.c_void_p(nbr.data_ptr()),
        int(n_active), int(n_nodes), int(p), float(c), float(h), _dev_ptr(x, n_active, "x"),
        _dev_ptr(y, n_active, "y"), _stream_ptr(stream)), "cpm_op_apply_noalloc")


def oras_apply(pc: Preconditioner, r, z, nrhs: int = 1, stream=None):
    n = pc.n_active * nrhs
    _check(_capi.load().oras_apply(pc.handle, _dev_ptr(r, n, "r"), _dev_ptr(z, n, "z"), int(nrhs),
                                   _stream_ptr(stream)), "oras_apply")


TUNE_KNOBS = {"ctas_per_sm": _capi.CPM_TUNE_SOLVE_CTAS_PER_SM, "kseg": _capi.CPM_TUNE_SOLVE_KSEG,
              "prefetch": _capi.CPM_TUNE_SOLVE_PREFETCH, "stagger": _capi.CPM_TUNE_SOLVE_STAGGER}


def oras_tune(pc: Preconditioner, **knobs):
    """Set schedule knobs of the batched solve: ctas_per_sm=, kseg=, prefetch=, stagger=."""
    for k, v in knobs.items():
        _check(_capi.load().oras_tune(pc.handle, TUNE_KNOBS[k], int(v)), "oras_tune")


def oras_autotune(pc: Preconditioner, stream=None) -> dict:
    """Time the candidate schedules of the batched solve and keep the fastest."""
    _check(_capi.load().oras_autotune(pc.handle, _stream_ptr(stream)), "oras_autotune")
    inf = pc.info()
    return {k: inf["solve_" + k] for k in ("ctas_per_sm", "kseg", "prefetch", "stagger")}


def oras_check_status(pc: Preconditioner, stream=None):
    _check(_capi.load().oras_check_status(pc.handle, _stream_ptr(stream)), "oras_check_status")


def cpm_gmres_solve(pc: Preconditioner, f, u, nrhs: int = 1, restart: int = 50, tol: float = 1e-8,
                    max_it: int = 1000, use_graph: bool = True, zero_guess: bool = True,
                    stream=None, raise_on_failure: bool = True):
    """Returns a list of dicts (iterations, relres, status) per right-hand side."""
    n = pc.n_active * nrhs
    opts = _capi.cpm_gmres_opts(int(restart), float(tol), int(max_it), int(bool(use_graph)),
                                int(bool(zero_guess)))
    res = (_capi.cpm_gmres_result * nrhs)()
    st = _capi.load().cpm_gmres_solve(pc.handle, _dev_ptr(f, n, "f"), _dev_ptr(u, n, "u"), int(nrhs),
                                      C.byref(opts), res, _stream_ptr(stream))
    out = [{"iterations": r.iterations, "relres": r.relres, "status": r.status} for r in res]
    if st != 0 and (raise_on_failure or st not in _PER_RHS_STATUS):
        raise CpmError(st, "cpm_gmres_solve")
    return out


def oras_stationary_solve(pc: Preconditioner, f, u, nrhs: int = 1, tol: float = 1e-8,
                          max_it: int = 1000, stream=None, raise_on_failure: bool = True):
    """(O)RAS as a solver, u <- u + M^{-1}(f - A u) (Eq. algRAS).  List of dicts per rhs."""
    n = pc.n_active * nrhs
    res = (_capi.cpm_gmres_result * nrhs)()
    st = _capi.load().oras_stationary_solve(pc.handle, _dev_ptr(f, n, "f"), _dev_ptr(u, n, "u"),
                                            int(nrhs), float(tol), int(max_it), res,
                                            _stream_ptr(stream))
    out = [{"iterations": r.iterations, "relres": r.relres, "status": r.status} for r in res]
    if st != 0 and (raise_on_failure or st not in _PER_RHS_STATUS):
        raise CpmError(st, "oras_stationary_solve")
    return out


def cpm_vec_axpby(a: float, x, b: float, y, n: int | None = None, stream=None):
    """y = a x + b y on the device (b == 0: y = a x)."""
    n = y.numel() if n is None else int(n)
    _check(_capi.load().cpm_vec_axpby(n, float(a), _dev_ptr(x, n, "x"), float(b), _dev_ptr(y, n, "y"),
                                      _stream_ptr(stream)), "cpm_vec_axpby")


def cpm_probe_fp64(blocks: int, threads: int, chains: int, iters: int = 4096, latency: bool = True):
    """FP64 FMA probe: (TFLOP/s of the throughput kernel, cycles per dependent FMA or None)."""
    t = C.c_double(0.0)
    c = C.c_double(0.0)
    _check(_capi.load().cpm_probe_fp64(int(blocks), int(threads), int(chains), int(iters), C.byref(t),
                                       C.byref(c) if latency else None), "cpm_probe_fp64")
    return t.value, (c.value if latency else None)


def cpm_selftest_bounded_wait(pc: Preconditioner, limit_s: float = 0.2, stream=None) -> int:
    """Let a bounded device wait expire on purpose; returns the status (CPM_ERR_TIMEOUT)."""
    return int(_capi.load().cpm_selftest_bounded_wait(pc.handle, float(limit_s), _stream_ptr(stream)))


def cpm_selftest_zero_operator(pc: Preconditioner) -> None:
    """Make pc's operator the zero matrix (breakdown self-test; the handle is not usable for
    real solves afterwards)."""
    _check(_capi.load().cpm_selftest_zero_operator(pc.handle), "cpm_selftest_zero_operator")


def status_string(code: int) -> str:
    return _capi.load().cpm_status_string(int(code)).decode()
