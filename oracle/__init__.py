"""FP64 CPU oracle for the TT hot path -- TEST INFRASTRUCTURE ONLY.

A plain, slow, obviously correct NumPy (float64) statement of what the library computes:
the TT definition, transfer-matrix sweeps for inner products and Gram matrices, element
gather and the completion loss with its gradient, TT-matrix x TT-vector, Householder
orthogonalisation and the Riemannian tangent-space projection (project / project_sum) with
its adjoint, the tailored tangent-space operations (Gram matrix of tangent vectors,
projected matrix-by-vector product, linearised Riemannian Hessian of the completion loss)
and TT rounding. Only the tests, the smoke check and the benchmark's CPU-baseline leg may
import it; the library itself never does, and it shares no code with the CUDA path.

Parity pins (see tests/test_oracle_pins.py) tie every function here to something other than
itself: brute force against the full tensor, closed forms, invariants of the projector,
central finite differences. No function is "parity unpinned".
"""
from .tt_oracle import *  # noqa: F401,F403
