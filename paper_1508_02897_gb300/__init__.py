"""GB300-native one-step overlapping DDM preconditioner for the 2D Helmholtz
equation with PML (Leng & Ju, arXiv 1508.02897): CUDA kernels for sm_103a
behind a C ABI (include/hd.h), with this thin Python binding on top."""
from . import _binding  # noqa: F401
from ._binding import (HD_ARNOLDI_DS, HD_ARNOLDI_FP64, HD_C64, HD_C64_B, HD_C64_H, HD_C128, HDError, declared_symbols, hd_apply_precond, hd_check_status,  # noqa: F401
                       hd_destroy, hd_factor_subdomains, hd_get_timers, hd_gmres_solve, hd_last_error, hd_matvec,
                       hd_query_workspace, hd_rhs_from_source, hd_set_profiling, hd_setup_medium, hd_version, lib)

__all__ = ["HelmholtzDDM", "solve_host", "lib", "declared_symbols"]


def __getattr__(name):
    if name in ("HelmholtzDDM", "solve_host"):
        from . import solver
        return getattr(solver, name)
    raise AttributeError(name)
