"""B300-native LS-AMG-DD: least-squares AMG domain-decomposition preconditioning for
conforming finite elements (element Gram factors, local spectral coarse spaces,
multiplicative Schwarz V-cycle), CUDA kernels for sm_103a behind a C ABI.

    from paper_2607_07485_b300 import Lsamg
    amg = Lsamg(n, elem_dofs, elem_mats, coef)      # set-up on the GPU
    x, its, relres, status = amg.solve(b)           # FP64 flexible CG, FP32 V-cycle
"""
from .lsamg import Lsamg, LsamgError, options, LIB_PATH, EXPORTS, Q  # noqa: F401
from .autograd import LsamgSolve, solve_with_grad  # noqa: F401
