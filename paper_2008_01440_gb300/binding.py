"""ctypes binding of libncpcg (include/nc_pcg.h): argument marshalling only.

Every function here has the name of the C entry point it calls and does no
arithmetic of its own: torch tensors are turned into device pointers and
streams into ``cudaStream_t`` handles; every step of the solve runs in the
library's CUDA kernels.  Importing this module fails loudly when the library
has not been built (``__graft_entry__.build()`` or
``python -m paper_2008_01440_gb300.build``).
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libncpcg.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"libncpcg.so not built at {LIB_PATH}; run paper_2008_01440_gb300.build.build()")

lib = ctypes.CDLL(LIB_PATH)

NC_OK, NC_ERR_ARG, NC_ERR_CUDA, NC_ERR_OOM, NC_ERR_INDEFINITE, NC_ERR_MAXIT, NC_ERR_BREAKDOWN, \
    NC_ERR_UNSUPPORTED, NC_ERR_SCRATCH_LIMIT, NC_ERR_ADMISSION, NC_ERR_TIMEOUT = range(11)
NC_F64, NC_F32, NC_BF16 = 0, 1, 2
_DTYPES = {"f64": NC_F64, "f32": NC_F32, "bf16": NC_BF16}
# statuses a solve may end with while still returning a meaningful iterate
SOLVE_STATUSES = (NC_OK, NC_ERR_MAXIT, NC_ERR_INDEFINITE, NC_ERR_BREAKDOWN)


NC_FORMAT_AUTO, NC_FORMAT_CSR, NC_FORMAT_SELL, NC_FORMAT_TUNE, NC_FORMAT_PSELL = 0, 1, 2, 3, 4
_FORMATS = {"auto": NC_FORMAT_AUTO, "csr": NC_FORMAT_CSR, "sell": NC_FORMAT_SELL, "tune": NC_FORMAT_TUNE,
            "psell": NC_FORMAT_PSELL}


NC_STEP_AUTO, NC_STEP_DIRECT, NC_STEP_STAGED, NC_STEP_TUNE, NC_STEP_SPLIT = 0, 1, 2, 3, 4
_STEPS = {"auto": NC_STEP_AUTO, "direct": NC_STEP_DIRECT, "staged": NC_STEP_STAGED, "tune": NC_STEP_TUNE,
          "split": NC_STEP_SPLIT}
_STEP_NAMES = {NC_STEP_DIRECT: "direct", NC_STEP_STAGED: "staged", NC_STEP_SPLIT: "split"}


class nc_options(ctypes.Structure):
    _fields_ = [("apply_dtype", ctypes.c_int), ("rr_period", ctypes.c_int),
                ("x0_is_zero", ctypes.c_int), ("use_graph", ctypes.c_int), ("spmv_format", ctypes.c_int),
                ("poly_form", ctypes.c_int), ("step_kernel", ctypes.c_int), ("step_stages", ctypes.c_int),
                ("step_ctas_per_sm", ctypes.c_int), ("step_rows_per_thread", ctypes.c_int),
                ("step_tile_order", ctypes.c_int), ("prefetch_tiles", ctypes.c_int),
                ("red_ctas_per_sm", ctypes.c_int), ("keep_diagonal", ctypes.c_int)]


class nc_solver_info(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("degree_k", ctypes.c_int32), ("spmv_format", ctypes.c_int32),
                ("apply_dtype", ctypes.c_int32), ("persistent", ctypes.c_int32), ("padding", ctypes.c_double),
                ("theta", ctypes.c_double), ("delta", ctypes.c_double), ("sigma", ctypes.c_double),
                ("shift", ctypes.c_double), ("tune_us_plain", ctypes.c_double), ("tune_us_sliced", ctypes.c_double),
                ("patterns", ctypes.c_int64), ("step_kernel", ctypes.c_int32), ("dot_step_kernel", ctypes.c_int32),
                ("step_stages", ctypes.c_int32), ("step_ctas_per_sm", ctypes.c_int32),
                ("step_rows_per_thread", ctypes.c_int32), ("step_tile_order", ctypes.c_int32),
                ("dot_step_stages", ctypes.c_int32), ("dot_step_ctas_per_sm", ctypes.c_int32),
                ("dot_step_rows_per_thread", ctypes.c_int32), ("dot_step_tile_order", ctypes.c_int32),
                ("prefetch_tiles", ctypes.c_int32), ("red_ctas_per_sm", ctypes.c_int32),
                ("tune_candidates", ctypes.c_int32), ("num_sms", ctypes.c_int32), ("faults", ctypes.c_int32),
                ("tune_from_cache", ctypes.c_int32), ("stencil_zchunk", ctypes.c_int32),
                ("stencil_planes_per_batch", ctypes.c_int32), ("diag_folded", ctypes.c_int32),
                ("reserved1", ctypes.c_int32), ("diag_value", ctypes.c_double)]


class nc_tune_candidate(ctypes.Structure):
    _fields_ = [("op", ctypes.c_int32), ("step_kernel", ctypes.c_int32), ("stages", ctypes.c_int32),
                ("ctas_per_sm", ctypes.c_int32), ("rows_per_thread", ctypes.c_int32), ("tile_order", ctypes.c_int32),
                ("prefetch_tiles", ctypes.c_int32),
                ("red_ctas_per_sm", ctypes.c_int32), ("zchunk", ctypes.c_int32),
                ("planes_per_batch", ctypes.c_int32), ("us", ctypes.c_double), ("chosen", ctypes.c_int32),
                ("reserved0", ctypes.c_int32)]


class nc_result(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("status", ctypes.c_int32), ("relres", ctypes.c_double),
                ("true_relres", ctypes.c_double), ("n_spmv", ctypes.c_int64), ("n_dot", ctypes.c_int64),
                ("n_replace", ctypes.c_int64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_vp = ctypes.c_void_p
_i64 = ctypes.c_int64
_dbl = ctypes.c_double
_pd = ctypes.POINTER(ctypes.c_double)

_SIGS = {
    "nc_options_default": (None, [ctypes.POINTER(nc_options)]),
    "nc_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "nc_version": (ctypes.c_char_p, []),
    "nc_last_cuda_error": (ctypes.c_char_p, []),
    "nc_matrix_csr": (ctypes.c_int, [_i64, _i64, _vp, _vp, _vp, ctypes.POINTER(_vp)]),
    "nc_matrix_jacobi": (ctypes.c_int, [_vp, _vp, ctypes.POINTER(_vp)]),
    "nc_matrix_block_jacobi": (ctypes.c_int, [_vp, _vp, ctypes.POINTER(_vp)]),
    "nc_matrix_bsr3": (ctypes.c_int, [_i64, _i64, _vp, _vp, _vp, ctypes.POINTER(_vp)]),
    "nc_matrix_stencil7": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, _dbl, _dbl, _dbl, _dbl,
                                          ctypes.POINTER(_vp)]),
    "nc_matvec": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "nc_bounds_lanczos": (ctypes.c_int, [_vp, ctypes.c_int, _vp, _vp, _pd, _pd, _pd, _pd]),
    "nc_bounds_power": (ctypes.c_int, [_vp, ctypes.c_int, _vp, _vp, _pd]),
    "nc_gershgorin": (ctypes.c_int, [_vp, _vp, _pd]),
    "nc_matrix_destroy": (ctypes.c_int, [_vp]),
    "pcg_setup": (ctypes.c_int, [_vp, _dbl, _dbl, ctypes.c_int, _dbl, ctypes.POINTER(nc_options), _vp,
                                 ctypes.POINTER(_vp)]),
    "pcg_apply_poly": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "pcg_solve": (ctypes.c_int, [_vp, _vp, _vp, _dbl, ctypes.c_int, _vp, ctypes.POINTER(nc_result)]),
    "pcg_solve_host": (ctypes.c_int, [_vp, _vp, _vp, _dbl, ctypes.c_int, _vp, ctypes.POINTER(nc_result)]),
    "pcg_solve_multi": (ctypes.c_int, [_vp, ctypes.c_int, _vp, _vp, _dbl, ctypes.c_int, _vp,
                                       ctypes.POINTER(nc_result)]),
    "pcg_destroy": (ctypes.c_int, [_vp]),
    "pcg_get_info": (ctypes.c_int, [_vp, ctypes.POINTER(nc_solver_info)]),
    "pcg_tune_candidate": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.POINTER(nc_tune_candidate)]),
    "nc_apply_poly_csr_noalloc": (ctypes.c_int, [_i64, _vp, _vp, _vp, _dbl, _dbl, ctypes.c_int, _dbl, _vp, _vp,
                                                 _vp]),
    "nc_apply_poly_noalloc_max_n": (_i64, []),
    "pcg_batch_create": (ctypes.c_int, [ctypes.c_int, _i64, ctypes.c_int, ctypes.c_int, _vp, ctypes.POINTER(_vp)]),
    "pcg_batch_add": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, _dbl, _dbl, _dbl, _dbl, _dbl,
                                     _dbl, ctypes.c_int, _dbl, _vp, _vp, ctypes.POINTER(ctypes.c_int)]),
    "pcg_batch_add_solver": (ctypes.c_int, [_vp, _vp, _vp, _vp, ctypes.POINTER(ctypes.c_int)]),
    "pcg_batch_add_solver_multi": (ctypes.c_int, [_vp, _vp, ctypes.c_int, _vp, ctypes.c_int64, _vp,
                                                  ctypes.POINTER(ctypes.c_int)]),
    "pcg_solve_batched": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(_vp), ctypes.POINTER(ctypes.c_int),
                                         ctypes.POINTER(_vp), ctypes.POINTER(_vp), _dbl, ctypes.c_int, _vp,
                                         ctypes.POINTER(nc_result)]),
    "pcg_batch_run": (ctypes.c_int, [_vp, _dbl, ctypes.c_int, ctypes.c_int, _vp, ctypes.POINTER(ctypes.c_int)]),
    "pcg_batch_status": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(nc_result)]),
    "pcg_batch_collect": (ctypes.c_int, [_vp, ctypes.c_int, _vp, _vp]),
    "pcg_batch_release": (ctypes.c_int, [_vp, ctypes.c_int, _vp]),
    "pcg_batch_free_units": (ctypes.c_int, [_vp, ctypes.POINTER(_i64), ctypes.POINTER(_i64)]),
    "pcg_batch_stats": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]),
    "pcg_batch_destroy": (ctypes.c_int, [_vp]),
    "nc_batch_last_cuda_error": (ctypes.c_char_p, []),
}
for _name, (_res, _args) in _SIGS.items():
    _f = getattr(lib, _name)
    _f.restype = _res
    _f.argtypes = _args


class NcError(RuntimeError):
    def __init__(self, status: int, where: str):
        msg = lib.nc_strerror(status).decode()
        if status == NC_ERR_CUDA:
            src = lib.nc_batch_last_cuda_error if where.startswith("pcg_batch") else lib.nc_last_cuda_error
            msg += ": " + src().decode()
        super().__init__(f"{where}: {msg} (status {status})")
        self.status = status


def _check(status: int, where: str):
    if status != NC_OK:
        raise NcError(status, where)


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _check_device(index, current, what="tensor"):
    """The library launches on the CURRENT device and looks up its per-device
    state (the no-allocation array, solver workspaces) there, so a tensor on
    another device would hand its kernels foreign pointers: refuse it."""
    if index != current:
        raise ValueError(f"{what}: on cuda:{index} but the current device is cuda:{current}; "
                         f"call inside torch.cuda.device({index})")


def _ptr(t, dtype=None, n=None, what="tensor"):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{what}: expected a CUDA tensor")
    _check_device(t.device.index, torch.cuda.current_device(), what)
    if not t.is_contiguous():
        raise ValueError(f"{what}: must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{what}: expected {dtype}, got {t.dtype}")
    if n is not None and t.numel() != n:
        raise ValueError(f"{what}: expected {n} elements, got {t.numel()}")
    return t.data_ptr()


@dataclass
class Matrix:
    """Owning wrapper of an nc_matrix handle; keeps the borrowed tensors alive."""
    handle: int
    n: int
    keep: tuple
    parent: "Matrix | None" = None

    def close(self):
        if self.handle:
            lib.nc_matrix_destroy(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


@dataclass
class Solver:
    handle: int
    n: int
    matrix: Matrix
    degree: int

    def close(self):
        if self.handle:
            lib.pcg_destroy(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def nc_version() -> str:
    return lib.nc_version().decode()


def nc_matrix_csr(rowptr, col, val) -> Matrix:
    import torch
    n = rowptr.numel() - 1
    nnz = col.numel()
    h = _vp()
    _check(lib.nc_matrix_csr(n, nnz, _ptr(rowptr, torch.int32, what="rowptr"),
                             _ptr(col, torch.int32, what="col"), _ptr(val, torch.float64, nnz, "val"),
                             ctypes.byref(h)), "nc_matrix_csr")
    return Matrix(h.value, n, (rowptr, col, val))


def nc_matrix_bsr3(browptr, bcol, val) -> Matrix:
    """val: float64, 9 entries per block (row-major 3x3), shape (nnzb, 3, 3) or flat."""
    import torch
    nb = browptr.numel() - 1
    nnzb = bcol.numel()
    h = _vp()
    _check(lib.nc_matrix_bsr3(nb, nnzb, _ptr(browptr, torch.int32, what="browptr"), _ptr(bcol, torch.int32, what="bcol"),
                              _ptr(val, torch.float64, 9 * nnzb, "val"), ctypes.byref(h)), "nc_matrix_bsr3")
    return Matrix(h.value, 3 * nb, (browptr, bcol, val))


def nc_matrix_stencil7(nx: int, ny: int, nz: int, c0: float, cx: float, cy: float, cz: float) -> Matrix:
    h = _vp()
    _check(lib.nc_matrix_stencil7(int(nx), int(ny), int(nz), float(c0), float(cx), float(cy), float(cz),
                                  ctypes.byref(h)), "nc_matrix_stencil7")
    return Matrix(h.value, int(nx) * int(ny) * int(nz), ())


def nc_matrix_jacobi(A: Matrix, stream=None) -> Matrix:
    h = _vp()
    _check(lib.nc_matrix_jacobi(A.handle, _stream(stream), ctypes.byref(h)), "nc_matrix_jacobi")
    return Matrix(h.value, A.n, A.keep, parent=A)


def nc_matrix_block_jacobi(A: Matrix, stream=None) -> Matrix:
    """W^T A W with W = blockdiag(L_i^{-T}) (block-Jacobi first level) for a
    3x3-block matrix; solvers on it take the original b and return the original x."""
    h = _vp()
    _check(lib.nc_matrix_block_jacobi(A.handle, _stream(stream), ctypes.byref(h)), "nc_matrix_block_jacobi")
    return Matrix(h.value, A.n, A.keep, parent=A)


def nc_matvec(A: Matrix, x, y, stream=None):
    import torch
    _check(lib.nc_matvec(A.handle, _ptr(x, torch.float64, A.n, "x"), _ptr(y, torch.float64, A.n, "y"),
                         _stream(stream)), "nc_matvec")


def nc_gershgorin(A: Matrix, stream=None) -> float:
    out = ctypes.c_double()
    _check(lib.nc_gershgorin(A.handle, _stream(stream), ctypes.byref(out)), "nc_gershgorin")
    return out.value


def nc_bounds_lanczos(A: Matrix, steps: int, v0, stream=None):
    """Return (lmin, lmax, ritz_min, ritz_max)."""
    import torch
    lo, hi, rmin, rmax = (ctypes.c_double() for _ in range(4))
    _check(lib.nc_bounds_lanczos(A.handle, steps, _ptr(v0, torch.float64, A.n, "v0"), _stream(stream),
                                 ctypes.byref(lo), ctypes.byref(hi), ctypes.byref(rmin), ctypes.byref(rmax)),
           "nc_bounds_lanczos")
    return lo.value, hi.value, rmin.value, rmax.value


def nc_bounds_power(A: Matrix, iters: int, v0, stream=None) -> float:
    """lambda_max estimate: the Rayleigh quotient after `iters` power iterations."""
    import torch
    lam = ctypes.c_double()
    _check(lib.nc_bounds_power(A.handle, int(iters), _ptr(v0, torch.float64, A.n, "v0"), _stream(stream),
                               ctypes.byref(lam)), "nc_bounds_power")
    return lam.value


_POLY = {"chebyshev": 0, "newton": 1}


def make_options(apply_dtype="f64", rr_period=0, x0_is_zero=False, use_graph=True, spmv_format="auto",
                 persistent=False, poly="chebyshev", step_kernel="auto", step_stages=0, step_ctas_per_sm=0,
                 step_rows_per_thread=0, step_tile_order=0, prefetch_tiles=0, red_ctas_per_sm=0,
                 keep_diagonal=False) -> nc_options:
    o = nc_options()
    lib.nc_options_default(ctypes.byref(o))
    o.spmv_format = _FORMATS[spmv_format] if isinstance(spmv_format, str) else int(spmv_format)
    o.apply_dtype = _DTYPES[apply_dtype] if isinstance(apply_dtype, str) else int(apply_dtype)
    o.rr_period = int(rr_period)
    o.x0_is_zero = int(bool(x0_is_zero))
    o.use_graph = 2 if persistent else int(bool(use_graph))
    o.poly_form = _POLY[poly] if isinstance(poly, str) else int(poly)
    o.step_kernel = _STEPS[step_kernel] if isinstance(step_kernel, str) else int(step_kernel)
    o.step_stages = int(step_stages)
    o.step_ctas_per_sm = int(step_ctas_per_sm)
    o.step_rows_per_thread = int(step_rows_per_thread)
    o.step_tile_order = int(step_tile_order)
    o.prefetch_tiles = int(prefetch_tiles)
    o.red_ctas_per_sm = int(red_ctas_per_sm)
    o.keep_diagonal = int(bool(keep_diagonal))
    return o


def pcg_setup(A: Matrix, lambda_min: float, lambda_max: float, degree_k: int, theta_scale: float = 1.0,
              stream=None, **options) -> Solver:
    opt = make_options(**options)
    h = _vp()
    _check(lib.pcg_setup(A.handle, float(lambda_min), float(lambda_max), int(degree_k), float(theta_scale),
                         ctypes.byref(opt), _stream(stream), ctypes.byref(h)), "pcg_setup")
    return Solver(h.value, A.n, A, int(degree_k))


def pcg_get_info(S: Solver) -> dict:
    info = nc_solver_info()
    _check(lib.pcg_get_info(S.handle, ctypes.byref(info)), "pcg_get_info")
    d = {f: getattr(info, f) for f, _ in info._fields_}
    d["persistent"] = bool(d["persistent"])
    d["spmv_format"] = {NC_FORMAT_CSR: "csr", NC_FORMAT_SELL: "sell", NC_FORMAT_PSELL: "psell"}.get(
        d["spmv_format"], d["spmv_format"])
    d["step_kernel"] = _STEP_NAMES.get(d["step_kernel"], d["step_kernel"])
    d["dot_step_kernel"] = _STEP_NAMES.get(d["dot_step_kernel"], d["dot_step_kernel"])
    return d


_TUNE_OPS = {0: "step", 1: "last_step_dot", 2: "q_dot"}


def pcg_tune_candidates(S: Solver) -> list:
    """Every launch configuration the tuner timed during pcg_setup, in order
    (empty when the solver was not tuned)."""
    out = []
    for i in range(pcg_get_info(S)["tune_candidates"]):
        c = nc_tune_candidate()
        _check(lib.pcg_tune_candidate(S.handle, i, ctypes.byref(c)), "pcg_tune_candidate")
        d = {f: getattr(c, f) for f, _ in c._fields_ if f != "reserved0"}
        d["op"] = _TUNE_OPS.get(d["op"], d["op"])
        d["step_kernel"] = _STEP_NAMES.get(d["step_kernel"], d["step_kernel"])
        d["chosen"] = bool(d["chosen"])
        out.append(d)
    return out


def pcg_apply_poly(S: Solver, v, z, stream=None):
    import torch
    _check(lib.pcg_apply_poly(S.handle, _ptr(v, torch.float64, S.n, "v"), _ptr(z, torch.float64, S.n, "z"),
                              _stream(stream)), "pcg_apply_poly")


def pcg_solve(S: Solver, b, x, tol: float, maxit: int, stream=None) -> dict:
    import torch
    res = nc_result()
    st = lib.pcg_solve(S.handle, _ptr(b, torch.float64, S.n, "b"), _ptr(x, torch.float64, S.n, "x"),
                       float(tol), int(maxit), _stream(stream), ctypes.byref(res))
    if st not in SOLVE_STATUSES:
        _check(st, "pcg_solve")
    return res.as_dict()


def pcg_solve_multi(S: Solver, B, X, tol: float, maxit: int, stream=None) -> list:
    """B, X: CUDA float64 tensors of shape (m, n) (row c = right-hand side /
    solution c, i.e. the n x m block column-major), 1 <= m <= 8."""
    import torch
    if B.dim() != 2 or B.shape != X.shape or B.shape[1] != S.n:
        raise ValueError(f"B, X: expected equal shapes (m, {S.n})")
    m = int(B.shape[0])
    res = (nc_result * m)()
    st = lib.pcg_solve_multi(S.handle, m, _ptr(B, torch.float64, m * S.n, "B"), _ptr(X, torch.float64, m * S.n, "X"),
                             float(tol), int(maxit), _stream(stream), res)
    if st not in SOLVE_STATUSES:
        _check(st, "pcg_solve_multi")
    return [r.as_dict() for r in res]


def pcg_solve_host(S: Solver, b, x, tol: float, maxit: int, stream=None) -> dict:
    """b, x: host (CPU) float64 tensors or numpy arrays of length n (pinned for async copies)."""
    res = nc_result()

    def hptr(a, what):
        import numpy as np
        try:
            import torch
            if isinstance(a, torch.Tensor):
                if a.is_cuda or a.dtype != torch.float64 or not a.is_contiguous() or a.numel() != S.n:
                    raise TypeError(f"{what}: expected a contiguous CPU float64 tensor of length {S.n}")
                return a.data_ptr()
        except ImportError:
            pass
        if not (isinstance(a, np.ndarray) and a.dtype == np.float64 and a.flags.c_contiguous and a.size == S.n):
            raise TypeError(f"{what}: expected a contiguous float64 array of length {S.n}")
        return a.ctypes.data

    st = lib.pcg_solve_host(S.handle, hptr(b, "b"), hptr(x, "x"), float(tol), int(maxit), _stream(stream),
                            ctypes.byref(res))
    if st not in SOLVE_STATUSES:
        _check(st, "pcg_solve_host")
    return res.as_dict()


def nc_apply_poly_noalloc_max_n() -> int:
    return int(lib.nc_apply_poly_noalloc_max_n())


def nc_apply_poly_csr_noalloc(rowptr, col, val, lambda_min: float, lambda_max: float, degree_k: int,
                              theta_scale: float, v, z, stream=None):
    """z = P_k(A) v without any device allocation by the library (for callers
    that cannot allocate; see include/nc_pcg.h).  Same arguments as
    nc_matrix_csr + pcg_setup + pcg_apply_poly in one call."""
    import torch
    n = rowptr.numel() - 1
    _check(lib.nc_apply_poly_csr_noalloc(n, _ptr(rowptr, torch.int32, what="rowptr"),
                                         _ptr(col, torch.int32, what="col"), _ptr(val, torch.float64, what="val"),
                                         float(lambda_min), float(lambda_max), int(degree_k), float(theta_scale),
                                         _ptr(v, torch.float64, n, "v"), _ptr(z, torch.float64, n, "z"),
                                         _stream(stream)), "nc_apply_poly_csr_noalloc")


def pcg_destroy(S: Solver):
    S.close()


def nc_matrix_destroy(A: Matrix):
    A.close()


class Batch:
    """Owning wrapper of an nc_batch engine (see include/nc_pcg.h)."""

    def __init__(self, handle: int):
        self.handle = handle

    def close(self):
        if self.handle:
            lib.pcg_batch_destroy(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


NC_BATCH_HOST_LOOP = 1
NC_BATCH_F64_APPLY = 2


def pcg_batch_create(max_slots: int, max_unknowns: int, kmax: int, stream=None, host_loop: bool = False,
                     f64_apply: bool = False) -> Batch:
    h = _vp()
    flags = (NC_BATCH_HOST_LOOP if host_loop else 0) | (NC_BATCH_F64_APPLY if f64_apply else 0)
    _check(lib.pcg_batch_create(int(max_slots), int(max_unknowns), int(kmax), flags, _stream(stream),
                                ctypes.byref(h)), "pcg_batch_create")
    return Batch(h.value)


def pcg_batch_add(B: Batch, nx: int, ny: int, nz: int, c0: float, cx: float, cy: float, cz: float,
                  lambda_min: float, lambda_max: float, degree_k: int, theta_scale: float, b, stream=None):
    """Admit one system; returns the slot id, or None when the engine is full
    (NC_ERR_ADMISSION)."""
    import torch
    slot = ctypes.c_int(-1)
    n = int(nx) * int(ny) * int(nz)
    st = lib.pcg_batch_add(B.handle, int(nx), int(ny), int(nz), float(c0), float(cx), float(cy), float(cz),
                           float(lambda_min), float(lambda_max), int(degree_k), float(theta_scale),
                           _ptr(b, torch.float64, n, "b"), _stream(stream), ctypes.byref(slot))
    if st == NC_ERR_ADMISSION:
        return None
    _check(st, "pcg_batch_add")
    return slot.value


def pcg_batch_add_solver(B: Batch, S: Solver, b, stream=None):
    """Admit one right-hand side of an explicit-matrix solver (pcg_setup of a
    CSR handle in a sliced layout) as a slot; returns the slot id, or None when
    the engine is full (NC_ERR_ADMISSION)."""
    import torch
    slot = ctypes.c_int(-1)
    st = lib.pcg_batch_add_solver(B.handle, S.handle, _ptr(b, torch.float64, S.n, "b"), _stream(stream),
                                  ctypes.byref(slot))
    if st == NC_ERR_ADMISSION:
        return None
    _check(st, "pcg_batch_add_solver")
    return slot.value


def pcg_batch_add_solver_multi(B: Batch, S: Solver, Bm, stream=None):
    """Admit the m <= 8 right-hand sides Bm (contiguous CUDA float64, shape
    (m, n)) of one explicit-matrix solver as a group whose step kernels read
    the matrix once for all m; returns the m slot ids, or None when the
    engine has no room (NC_ERR_ADMISSION)."""
    import torch
    if Bm.dim() != 2 or Bm.shape[1] != S.n:
        raise ValueError(f"Bm: expected shape (m, {S.n})")
    m = int(Bm.shape[0])
    slots = (ctypes.c_int * max(m, 1))()
    st = lib.pcg_batch_add_solver_multi(B.handle, S.handle, m, _ptr(Bm, torch.float64, m * S.n, "Bm"), S.n,
                                        _stream(stream), slots)
    if st == NC_ERR_ADMISSION:
        return None
    _check(st, "pcg_batch_add_solver_multi")
    return [slots[c] for c in range(m)]


def pcg_solve_batched(solvers, Bs, Xs, tol: float, maxit: int, stream=None) -> list:
    """Solve every system i (solvers[i]) for the right-hand sides Bs[i] (CUDA
    float64, shape (m_i, n_i) or (n_i,)) into Xs[i] (same shape) in one engine
    launch; returns one result dict per (system, right-hand side)."""
    import torch
    ns = len(solvers)
    if not (len(Bs) == len(Xs) == ns) or ns < 1:
        raise ValueError("solvers, Bs, Xs: equal, non-zero lengths")
    hs = (_vp * ns)(*[S.handle for S in solvers])
    nrhs = (ctypes.c_int * ns)()
    bp = (_vp * ns)()
    xp = (_vp * ns)()
    for i, (S, b, x) in enumerate(zip(solvers, Bs, Xs)):
        if b.shape != x.shape or b.shape[-1] != S.n or b.dim() not in (1, 2):
            raise ValueError(f"Bs[{i}], Xs[{i}]: expected equal shapes (m, {S.n}) or ({S.n},)")
        m = 1 if b.dim() == 1 else int(b.shape[0])
        nrhs[i] = m
        bp[i] = _ptr(b, torch.float64, m * S.n, f"Bs[{i}]")
        xp[i] = _ptr(x, torch.float64, m * S.n, f"Xs[{i}]")
    total = sum(nrhs)
    res = (nc_result * total)()
    st = lib.pcg_solve_batched(ns, hs, nrhs, bp, xp, float(tol), int(maxit), _stream(stream), res)
    if st not in SOLVE_STATUSES:
        _check(st, "pcg_solve_batched")
    return [r.as_dict() for r in res]


def pcg_batch_run(B: Batch, tol: float, maxit: int, iter_limit: int = 0, stream=None) -> int:
    left = ctypes.c_int(0)
    _check(lib.pcg_batch_run(B.handle, float(tol), int(maxit), int(iter_limit), _stream(stream), ctypes.byref(left)),
           "pcg_batch_run")
    return left.value


def pcg_batch_status(B: Batch, slot: int):
    done = ctypes.c_int(0)
    res = nc_result()
    _check(lib.pcg_batch_status(B.handle, int(slot), ctypes.byref(done), ctypes.byref(res)), "pcg_batch_status")
    return bool(done.value), res.as_dict()


def pcg_batch_collect(B: Batch, slot: int, x, stream=None):
    import torch
    _check(lib.pcg_batch_collect(B.handle, int(slot), _ptr(x, torch.float64, what="x"), _stream(stream)),
           "pcg_batch_collect")


def pcg_batch_release(B: Batch, slot: int, stream=None):
    _check(lib.pcg_batch_release(B.handle, int(slot), _stream(stream)), "pcg_batch_release")


def pcg_batch_stats(B: Batch):
    """(engine iterations run, kernels launched) since creation."""
    it, ln = ctypes.c_int64(), ctypes.c_int64()
    _check(lib.pcg_batch_stats(B.handle, ctypes.byref(it), ctypes.byref(ln)), "pcg_batch_stats")
    return it.value, ln.value


def pcg_batch_free_units(B: Batch):
    lg, tt = _i64(0), _i64(0)
    _check(lib.pcg_batch_free_units(B.handle, ctypes.byref(lg), ctypes.byref(tt)), "pcg_batch_free_units")
    return lg.value, tt.value


def pcg_batch_destroy(B: Batch):
    B.close()
