"""GB300-native (sm_103a) Tensor-Train sweep library: the data-parallel hot path of T3F
(Novikov et al., JMLR 2020) -- Gram matrices and norms, element gather with the completion
loss, TT-matrix x TT-vector, FP64 orthogonalisation and the Riemannian project_sum, each with
a hand-written adjoint -- behind the C ABI of include/t3f.h.

The Python layer is argument marshalling over libt3f.so; import fails loudly at call time if
the library has not been built (``python -m paper_1801_01928_gb300.build``).
"""
from . import autograd  # noqa: F401,E402
from ._binding import (  # noqa: F401
    BF16, DEFAULT_TILES, EXPORTS, F32, F64, LIB_PATH, RaggedTT, T3FError, TT, autotune_gram_groups,
    device_status, gather, gather_backward, gram_groups, gram_groups_backward, gram_groups_prepare,
    gram, gram_backward, launch_count, load, matvec, matvec_backward, norm, orth_ranks, orthogonalize,
    project_sum, project_sum_backward, project, tangent_gram, project_matvec, completion_hvp, fma_probe, round_tt, round_ranks,
    workspace,
)
