"""FP64 CPU oracle for ML-CG ptychography (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import this package.  The product path (``paper_2106_07575_gb300``) never imports it.
"""
from .orc import (  # noqa: F401
    build,
    fft2,
    shift_probe,
    subpixel_probes,
    Q,
    QH,
    forward,
    adjoint,
    objective,
    gradient,
    cg_solve,
    OrcOpts,
    EST_ML,
    EST_LS,
    SOLVER_CG,
    SOLVER_GD,
    ORC_OK,
    ORC_ERR_ARG,
    ORC_ERR_BOUNDS,
    ORC_STALLED,
)
