"""B300-native LS-AMG-DD: least-squares AMG domain-decomposition preconditioning for
conforming finite elements (element Gram factors, local spectral coarse spaces,
multiplicative Schwarz V-cycle), CUDA kernels for sm_103a behind a C ABI.

    from paper_2607_07485_b300 import Lsamg
    amg = Lsamg(n, elem_dofs, elem_mats, coef)      # set-up on the GPU
    x, its, relres, status = amg.solve(b)           # FP64 flexible CG, FP32 V-cycle

The compiled library is loaded on first use of any of the names below (so that
``python -m paper_2607_07485_b300.build`` can rebuild it); a missing library raises.
"""
_LIB_NAMES = ("Lsamg", "LsamgError", "options", "LIB_PATH", "EXPORTS", "Q", "kernel_stats",
              "launch_count", "gram_spmv_static", "dgemm_nt")
_AD_NAMES = ("LsamgSolve", "solve_with_grad")
__all__ = list(_LIB_NAMES + _AD_NAMES)


def __getattr__(name):
    if name in _LIB_NAMES:
        from . import lsamg
        return getattr(lsamg, name)
    if name in _AD_NAMES:
        from . import autograd
        return getattr(autograd, name)
    raise AttributeError(name)
