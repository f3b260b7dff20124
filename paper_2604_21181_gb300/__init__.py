"""GB300 (sm_103a) implementation of the hot path of the nodal P2 Mueller
boundary-integral solver (arXiv 2604.21181): dense Galerkin assembly of the
coupled (J, M) system over curved P2 triangles (regular pairs by product
Gauss rules, touching pairs by Sauter-Schwab), the dense complex matvec,
the Morton-ordered block-Jacobi preconditioner and restarted GMRES (FP64, or
complex64 with FP64 iterative refinement), and the far-field cross sections.

The compute lives in ``lib/libmueller.so`` (C ABI: ``include/mueller.h``);
``api`` is the Python binding.
"""

from .api import (  # noqa: F401
    FRAME_PAPER,
    FRAME_POLAR,
    MUELLER_C128,
    MUELLER_C64_NEAR64,
    MUELLER_OP_K1_MIRRORED,
    MUELLER_OP_ADJOINT,
    SOLVE_DENSE_LU,
    SOLVE_GMRES,
    SOLVE_GMRES_IR,
    EXPORTS,
    Mesh,
    MuellerError,
    Operator,
    Params,
    SolverOpts,
    assemble,
    assemble_batch,
    dz_matvec,
    zshape_vjp,
    zshape_vjp_multi,
    rhs_shape_vjp,
    cross_section_partials,
    far_field,
    launch_count,
    load_library,
    profile_enable,
    profile_report,
    profile_reset,
    matvec,
    matvec_mrhs,
    precond_build,
    precond_build_batch,
    solve,
    solve_workspace_bytes,
    sync,
)
from .buildlib import build  # noqa: F401
from . import grad, sweep  # noqa: F401
