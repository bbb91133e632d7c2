"""GB300-native Newton-Chebyshev polynomial-preconditioned CG (sm_103a).

The compute path is the C-ABI library ``libncpcg.so`` (hand-written CUDA,
``csrc/``); ``binding`` marshals torch tensors into its calls.  There is no
CPU fallback: importing the package builds the library if it is missing
(nvcc required) and raises if that is impossible.
"""
import os as _os

from .build import LIB as _LIB
from .build import build as _build

if not _os.path.exists(_LIB):
    _build()

from .binding import (  # noqa: F401
    NC_BF16,
    NC_ERR_ARG,
    NC_ERR_BREAKDOWN,
    NC_ERR_CUDA,
    NC_ERR_INDEFINITE,
    NC_ERR_MAXIT,
    NC_ERR_OOM,
    NC_ERR_SCRATCH_LIMIT,
    NC_ERR_TIMEOUT,
    NC_ERR_UNSUPPORTED,
    NC_F32,
    NC_F64,
    NC_FORMAT_AUTO,
    NC_FORMAT_CSR,
    NC_FORMAT_PSELL,
    NC_FORMAT_SELL,
    NC_FORMAT_TUNE,
    NC_OK,
    NC_STEP_AUTO,
    NC_STEP_DIRECT,
    NC_STEP_STAGED,
    NC_STEP_TUNE,
    LIB_PATH,
    Matrix,
    NcError,
    Solver,
    lib,
    make_options,
    nc_apply_poly_csr_noalloc,
    nc_apply_poly_noalloc_max_n,
    nc_bounds_lanczos,
    nc_bounds_power,
    nc_gershgorin,
    nc_matrix_bsr3,
    nc_matrix_csr,
    nc_matrix_destroy,
    nc_matrix_block_jacobi,
    nc_matrix_jacobi,
    nc_matrix_stencil7,
    nc_matvec,
    nc_version,
    Batch,
    NC_ERR_ADMISSION,
    pcg_apply_poly,
    pcg_batch_add,
    pcg_batch_add_solver,
    pcg_batch_collect,
    pcg_batch_create,
    pcg_batch_destroy,
    pcg_batch_free_units,
    pcg_batch_release,
    pcg_batch_run,
    pcg_batch_stats,
    pcg_batch_status,
    pcg_destroy,
    pcg_get_info,
    pcg_setup,
    pcg_solve,
    pcg_solve_host,
    pcg_solve_batched,
    pcg_solve_multi,
    pcg_tune_candidates,
)
