"""GB300 (sm_103a) synchronous and asynchronous Parareal for the heat equation.

The compute path is libparareal.so (hand-written CUDA, C ABI in
include/parareal.h); this package is its thin Python binding with the same
function names, plus a torch.autograd.Function over the discrete adjoint.
"""
from ._abi import (PR_EXPLICIT_EULER, PR_IMPLICIT_EULER, PR_CRANK_NICOLSON, PR_SOLVER_CG,  # noqa: F401
                   PR_SOLVER_THOMAS, PR_OK, PR_ENOTCONV, PR_EINVAL, PR_ETIMEOUT, PR_ESTATE,
                   PR_ELOGFULL, PR_ECUDA, PR_ENOMEM, PR_OPT_PIPELINE, PR_OPT_PIPELINE_CHUNKS,
                   PR_OPT_CG_BLOCKS_PER_SM, PR_OPT_G_CHEBYSHEV, PR_OPT_G_CG, PR_OPT_F_STEPS_PER_PASS,
                   pr_problem, pr_stats, pr_async_opts, pr_event)
from .api import (PararealError, make_async_opts, make_problem, parareal_adjoint,  # noqa: F401
                  parareal_adjoint_async,
                  parareal_coarse, parareal_coarse_noalloc, parareal_correct, parareal_create, parareal_destroy,
                  parareal_fine, parareal_last_error, parareal_run_async, parareal_run_sync,
                  parareal_run_sync_host, parareal_serial_fine, parareal_set_problem, parareal_probe_fp64, parareal_probe_convert,
                  parareal_set_option, parareal_slice_stats, parareal_version)
