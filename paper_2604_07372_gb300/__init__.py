"""GB300 (sm_103a) NS-RGS: Newton-Schulz Riemannian gradient synchronisation.

Thin binding over the C ABI of ``libnsrgs.so`` (declared in include/nsrgs.h).
Every step of the method runs in the library's CUDA kernels; this module only
marshals torch device tensors and the current CUDA stream into the C calls.
There is no CPU fallback: when the library has not been built, importing the
binding works but the first call raises.
"""
from ._lib import (  # noqa: F401
    F32,
    BF16,
    FP8E4M3,
    DENSE_F32,
    DENSE_BF16,
    BCSR_F32,
    BCSR_BF16,
    STORAGE,
    NsrgsError,
    PackedA,
    Info,
    lib,
    lib_path,
    nsrgs_packed_bytes,
    nsrgs_workspace_bytes,
    nsrgs_bcsr_packed_bytes,
    nsrgs_pack_upper,
    nsrgs_pack_dense,
    nsrgs_spectral_init,
    nsrgs_step,
    nsrgs_solve,
    nsrgs_solve_host,
    nsrgs_solve_objective,
    nsrgs_solve_ex,
    SolveOpts,
    STOP_UPDATE_NORM,
    STOP_REL_DECREASE,
    nsrgs_objective,
    nsrgs_stiefel_solve,
    nsrgs_se_pack,
    nsrgs_se_solve,
    nsrgs_dF,
    nsrgs_version,
    nsrgs_set_kernel_timing,
    nsrgs_kernel_timing,
    workspace,
    nsrgs_batch_workspace_bytes,
    nsrgs_batch_solve,
    nsrgs_step_static,
    Server,
    nsrgs_product,
    nsrgs_gpm_solve,
    ServerResult,
)
