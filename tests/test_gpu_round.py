"""TT rounding (paper Section 3, t3f.round) on the GPU against the FP64 oracle: cores element
by element (same sign convention of the singular vectors), the rank bookkeeping exactly, the
exact recompression of X + X, and the rank-100 matvec products of config 3b rounded to rank
10 (cores, and the squared error against the sum of the discarded singular values)."""
import math

import numpy as np
import pytest

import oracle as O
import synth as S
from tests._util import TOL, objects, rel_err, rel_err_cores, round32

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def dev_tt(t3f, cores):
    return t3f.TT.from_cores([np.asarray(c, np.float32) for c in cores], device="cuda")


def host_objects(tt):
    return objects([c.detach().double().cpu().numpy() for c in tt.cores()])


@pytest.mark.parametrize("case", [
    (900, [3, 4, 2, 3], [1, 3, 5, 4, 1], 2, 4),
    (901, [2, 3, 3, 2, 4], [1, 2, 6, 6, 5, 1], 3, 3),
    (902, [5, 4, 6], [1, 5, 7, 1], 9, 2),          # max_rank above the ranks: orthogonalisation only
    (903, [7], [1, 1], 3, 2),                       # d = 1: a copy
])
def test_round_small(lib, case):
    seed, n, r, maxr, batch = case
    rng = np.random.default_rng(seed)
    X = round32(S.random_tt(rng, batch, n, r))
    Y = lib.round_tt(dev_tt(lib, X), maxr)
    assert Y.ranks == O.round_ranks(n, r, maxr) == lib.round_ranks(n, r, maxr)
    for j, Xo in enumerate(objects(X)):
        ref, _ = O.round_tt(Xo, maxr)
        assert rel_err_cores(host_objects(Y)[j], ref) < TOL["fp32"], j


def test_round_exact_recompression(lib):
    rng = np.random.default_rng(904)
    n = [3, 2, 4, 3]
    X = round32(S.random_tt(rng, 1, n, [1, 2, 3, 2, 1]))
    XX = O.tt_add(objects(X)[0], objects(X)[0])    # rank 2r, true rank r
    Y = lib.round_tt(dev_tt(lib, [c[None] for c in XX]), 3)
    Yf = O.full(host_objects(Y)[0])
    assert rel_err(Yf, 2 * O.full(objects(X)[0])) < TOL["fp32"]


def test_round_matvec_products_config3b_shapes(lib):
    # rank-100 products A_p x_p (d = 10, 4 x 4 modes) rounded to rank 10
    cfg = S.config3b(batch=6)
    A, x = round32(cfg.A), round32(cfg.x)
    C = lib.matvec(dev_tt(lib, A), dev_tt(lib, x))
    Cd = host_objects(C)
    Y = lib.round_tt(C, 10)
    assert Y.ranks == O.round_ranks([4] * 10, C.ranks, 10)
    Yh = host_objects(Y)
    for p in range(6):
        Cp = [np.asarray(c, np.float32).astype(np.float64) for c in Cd[p]]
        ref, disc = O.round_tt(Cp, 10)
        assert rel_err_cores(Yh[p], ref) < TOL["fp32"], p
        # ||C - Y||^2 = ||C||^2 - 2 <C, Y> + ||Y||^2 equals the discarded sigma^2
        e2 = O.dot(Cp, Cp) - 2 * O.dot(Cp, Yh[p]) + O.dot(Yh[p], Yh[p])
        assert abs(e2 - sum(disc)) <= 1e-4 * O.dot(Cp, Cp), p
