"""GB300-native Pauli decomposition (arXiv 2403.11644, PTDR) over a C ABI.

``decompose(A)`` returns all 4^n coefficients c_P = 2^-n tr(P A) of a complex
2^n x 2^n CUDA matrix; ``compose`` rebuilds A; ``decompose_structured`` handles
diagonal/band matrices on their reachable masks; ``decompose_batched`` runs
many matrices in one persistent launch; ``decompose_host`` takes host matrices
and overlaps their transfers; ``PtdrDecompose`` is the autograd Function.  All compute runs in libptdr's sm_103a kernels (include/ptdr.h).
"""
from .ptdr import (  # noqa: F401
    PRECISIONS,
    BatchedPlan,
    PtdrDecompose,
    autotune,
    block_diag,
    compose,
    decompose,
    decompose_autograd,
    decompose_batched,
    decompose_host,
    decompose_matrix_free,
    decompose_structured,
    hermitian_augment,
    host_scratch_size,
    last_device_status,
    lincomb,
    select,
    structured_masks,
    workspace_size,
)
from ._lib import PtdrError, load  # noqa: F401
