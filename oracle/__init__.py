"""Plain FP64 CPU oracle of SNMPBB, Graph-SNMPBB and LAI-SNMPBB.

TEST INFRASTRUCTURE ONLY.  Only the tests, the package's smoke check and the CPU
baseline leg of the benchmark may import this package.  The product path (the
C-ABI library and its Python binding) never calls it, and it shares no code with
the CUDA path.

Every function cites the passage of the paper it follows (section, equation,
algorithm).  Where the paper is silent the reading taken is stated in the
docstring.  Parity status: all functions are pinned by the CPU tests
(closed forms, finite differences, theorem invariants, special cases and brute
force); the paper's printed numbers (Table 1) are not a pin because the seeds,
stopping rule and hardware are not given.
"""
from .snmpbb import (  # noqa: F401
    Options,
    LaiOperator,
    apply_A,
    dense_of,
    proj,
    inner,
    spectral_norm,
    projected_gradient,
    direct_objective,
    direct_gradient,
    penalty_objective,
    penalty_grad_W,
    penalty_grad_Ht,
    paper_laplacian,
    nmpbb,
    snmpbb_direct,
    snmpbb_penalty,
    snmpbb_naive,
    resolve_lambda,
    svd_init,
)
from .philox import philox4x32, philox_uniform, philox_gaussian  # noqa: F401
from .lai import lai_sketch  # noqa: F401
from . import mlp  # noqa: F401
from . import knn  # noqa: F401
