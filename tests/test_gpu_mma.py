"""Tensor-core (tcgen05) Gram sweep: TF32 and BF16 operands with FP32 accumulation against the
FP64 oracle, at the stated tolerances (5e-3 TF32, 2e-2 BF16, normwise relative). TF32 runs on
FP32 cores (the oracle sees the same FP32 values); BF16 runs on BF16 cores (the oracle sees the
same BF16-rounded values), so the measured error is the arithmetic's alone. Shapes cover the
three padded ranks (16, 32, 64), ragged tile edges and unequal padded ranks on the two sides
(either order)."""
import math

import numpy as np
import pytest

import oracle as O
import synth as S
from tests._util import TOL, assert_gram_blocks, objects, rel_err, round32, round_bf16

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

CASES = [  # (n, ranks of A, ranks of B, batch A, batch B)
    ([4, 3, 5, 2, 4], [1, 10, 7, 10, 9, 1], [1, 6, 10, 8, 10, 1], 37, 29),
    ([3, 4, 2, 3], [1, 3, 20, 17, 1], [1, 3, 12, 31, 1], 21, 14),
    ([2, 3, 4, 2], [1, 2, 6, 40, 1], [1, 2, 6, 64, 1], 5, 7),
    ([3, 2, 4], [1, 12, 9, 1], [1, 50, 33, 1], 19, 6),     # padded ranks 16 x 64
    ([4, 3, 3], [1, 30, 28, 1], [1, 7, 11, 1], 11, 23),    # 32 x 16: sides swapped inside
]


def _tt(lib, cores, dtype):
    return lib.TT.from_cores([np.asarray(c, np.float32) for c in cores], dtype=dtype, device="cuda")


@pytest.mark.parametrize("case", range(len(CASES)))
@pytest.mark.parametrize("math_", ["tf32", "bf16"])
def test_gram_mma_vs_oracle(lib, case, math_):
    n, ra, rb, ba, bb = CASES[case]
    rng = np.random.default_rng(600 + case)
    A = S.random_tt(rng, ba, n, ra, 1.0 / math.sqrt(max(ra)))
    B = S.random_tt(rng, bb, n, rb, 1.0 / math.sqrt(max(rb)))
    if math_ == "tf32":
        A, B, dt = round32(A), round32(B), torch.float32
    else:
        A, B, dt = round_bf16(A), round_bf16(B), torch.bfloat16
    G = lib.gram(_tt(lib, A, dt), _tt(lib, B, dt), math=math_).double().cpu().numpy()
    Gref = O.gram(objects(A), objects(B))
    assert G.shape == (ba, bb)
    assert np.isfinite(G).all()
    assert rel_err(G, Gref) < TOL[math_]


@pytest.mark.parametrize("math_", ["tf32", "bf16"])
def test_gram_mma_config3a(lib, math_):
    cfg = S.config3a()
    A, B = round32(cfg.A), round32(cfg.B)
    G = lib.gram(_tt(lib, A, torch.float32), _tt(lib, B, torch.float32), math=math_).double().cpu().numpy()
    Gref = O.gram(objects(A), objects(B))
    assert rel_err(G, Gref) < TOL[math_]


def test_gram_mma_self_gram_diagonal(lib):
    # Gram of a batch with itself: the diagonal holds the squared norms (positive)
    rng = np.random.default_rng(610)
    A = round32(S.random_tt(rng, 19, [5, 4, 6], [1, 30, 30, 1], 1.0 / math.sqrt(30)))
    At = _tt(lib, A, torch.float32)
    G = lib.gram(At, At, math="tf32").double().cpu().numpy()
    nrm = np.array([O.norm(o) for o in objects(A)])
    assert rel_err(np.diag(G), nrm ** 2) < TOL["tf32"]
    assert rel_err(G, G.T) < TOL["tf32"]
    # diagonal and off-diagonal entries scored separately against the oracle
    assert_gram_blocks(G, O.gram(objects(A), objects(A)), [19], TOL["tf32"])
