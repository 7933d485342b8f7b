"""Tangent-space operations on the GPU against the FP64 oracle: the batched projection, the
Gram matrix of tangent vectors, the projected matrix-by-vector product and the linearised
Riemannian Hessian of the completion loss (paper Section 3.2). Inputs are rounded once to
FP32 and the same values go to the oracle; errors are normwise relative per output array
(Gram matrices per diagonal / off-diagonal entries), FP32 tolerance 1e-5."""
import math

import numpy as np
import pytest

import oracle as O
import synth as S
from tests._util import TOL, assert_gram_blocks, batched, objects, rel_err, rel_err_cores, round32

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def dev_tt(t3f, cores):
    return t3f.TT.from_cores([np.asarray(c, np.float32) for c in cores], device="cuda")


def host_objects(tt):
    return objects([c.detach().double().cpu().numpy() for c in tt.cores()])


def _uv(lib, X):
    U, V = lib.orthogonalize(dev_tt(lib, X), dtype=torch.float32)
    return U, V, host_objects(U)[0], host_objects(V)[0]


@pytest.mark.parametrize("shape", ["config1", "config5_small"])
@pytest.mark.parametrize("weights", [True, False])
def test_project_batch(lib, shape, weights):
    if shape == "config1":
        cfg = S.config1()
        X, Z, c = round32(cfg.X), round32(cfg.B), cfg.c.astype(np.float32)
    else:
        cfg = S.config5(batch=40)
        X, Z, c = round32(cfg.X), round32(cfg.Z), cfg.c.astype(np.float32)
    U, V, Uh, Vh = _uv(lib, X)
    ct = torch.tensor(c, device="cuda") if weights else None
    dU = lib.project(U, V, dev_tt(lib, Z), ct)
    got = host_objects(dU)
    ref = O.project_batch(Uh, Vh, objects(Z), c.astype(np.float64) if weights else None)
    assert len(got) == len(ref)
    for j in range(len(ref)):
        assert rel_err_cores(got[j], ref[j]) < TOL["fp32"], j
    if weights:
        # the batched coordinates sum to project_sum's
        tot = [sum(g[k] for g in got) for k in range(len(got[0]))]
        ps = host_objects(lib.project_sum(U, V, dev_tt(lib, Z), ct))[0]
        assert rel_err_cores(tot, ps) < TOL["fp32"]


def test_tangent_gram_coordinates(lib):
    # the definition on given coordinate arrays: sum_k <dA_k, dB_k>, several tiles and splits
    rng = np.random.default_rng(700)
    n, r = [5, 4, 6, 3], [1, 3, 7, 5, 1]
    dA = round32(S.random_tt(rng, 70, n, r))
    dB = round32(S.random_tt(rng, 67, n, r))
    G = lib.tangent_gram(dev_tt(lib, dA), dev_tt(lib, dB)).double().cpu().numpy()
    assert G.shape == (70, 67)
    assert rel_err(G, O.tangent_gram(objects(dA), objects(dB))) < TOL["fp32"]


def test_tangent_gram_of_projected_batch_config5_shape(lib):
    # end to end: project 48 rank-8 TTs onto T_X (d = 20, n = 16, r_X = 32) on the GPU, Gram
    # matrix of the tangent vectors, against the oracle's projection and Gram matrix
    cfg = S.config5(batch=48)
    X, Z, c = round32(cfg.X), round32(cfg.Z), cfg.c.astype(np.float32)
    U, V, Uh, Vh = _uv(lib, X)
    dU = lib.project(U, V, dev_tt(lib, Z), torch.tensor(c, device="cuda"))
    G = lib.tangent_gram(dU, dU).double().cpu().numpy()
    ref_coords = O.project_batch(Uh, Vh, objects(Z), c.astype(np.float64))
    Gref = O.tangent_gram(ref_coords, ref_coords)
    assert_gram_blocks(G, Gref, [48], TOL["fp32"])
    # the same matrix from the GPU's own coordinates through the oracle's definition
    assert_gram_blocks(G, O.tangent_gram(host_objects(dU), host_objects(dU)), [48], TOL["fp32"])


def _pmv_case(seed, d, m, n, rA, rx, rX, batch, A_batch):
    rng = np.random.default_rng(seed)
    A = round32(S.random_ttm(rng, A_batch, m, n, S.tt_ranks(d, rA), 1 / math.sqrt(rA)))
    x = round32(S.random_tt(rng, batch, n, S.tt_ranks(d, rx), 1 / math.sqrt(rx)))
    X = round32(S.random_tt(rng, 1, m, S.tt_ranks(d, rX), 1 / math.sqrt(rX)))
    return A, x, X


@pytest.mark.parametrize("case", [
    (800, 4, [2, 3, 2, 3], [3, 2, 2, 3], 3, 2, 3, 5, 1),     # tiny, A broadcast
    (801, 5, [3, 2, 3, 2, 2], [2, 2, 3, 2, 3], 2, 3, 4, 4, 4),  # A zip
    (802, 10, [4] * 10, [4] * 10, 10, 10, 10, 12, 1),      # config-3b shapes (product rank 100)
])
def test_project_matvec(lib, case):
    seed, d, m, n, rA, rx, rX, batch, A_batch = case
    A, x, X = _pmv_case(seed, d, m, n, rA, rx, rX, batch, A_batch)
    U, V, Uh, Vh = _uv(lib, X)
    dU = lib.project_matvec(U, V, dev_tt(lib, A), dev_tt(lib, x))
    got = host_objects(dU)
    Ao, xo = objects(A), objects(x)
    for j in range(batch):
        ref = O.project_matvec(Uh, Vh, Ao[0 if A_batch == 1 else j], [xo[j]])[0]
        assert rel_err_cores(got[j], ref) < TOL["fp32"], j


def test_completion_hvp_config1(lib):
    cfg = S.config1()
    X = round32(cfg.X)
    U, V, Uh, Vh = _uv(lib, X)
    xi = O.project(Uh, Vh, objects(round32(cfg.B))[3])
    xi32 = [np.asarray(c, np.float32).astype(np.float64) for c in xi]
    idx = torch.tensor(cfg.idx, device="cuda")
    H = lib.completion_hvp(U, V, idx, dev_tt(lib, [c[None] for c in xi32]))
    ref = O.completion_hvp(Uh, Vh, cfg.idx, xi32)
    assert rel_err_cores(host_objects(H)[0], ref) < TOL["fp32"]


def test_completion_hvp_config2_shape(lib):
    # completion shapes (d = 10, n = 10, model rank 8), 200k tuples; the direction is the
    # projection of a random rank-4 TT
    cfg = S.config2(N=200_000)
    X = round32(cfg.X)
    U, V, Uh, Vh = _uv(lib, X)
    xi = O.project(Uh, Vh, objects(round32(cfg.T))[0])
    xi32 = [np.asarray(c, np.float32).astype(np.float64) for c in xi]
    idx = torch.tensor(cfg.idx, device="cuda")
    H, ws = lib.completion_hvp(U, V, idx, dev_tt(lib, [c[None] for c in xi32]), return_ws=True)
    assert lib.device_status(ws) == 0
    ref = O.completion_hvp(Uh, Vh, cfg.idx, xi32)
    assert rel_err_cores(host_objects(H)[0], ref) < TOL["fp32"]
    # symmetric positive semi-definite: <xi, H xi> = sum_t xi(i_t)^2 >= 0
    q = O.tangent_gram([xi32], [host_objects(H)[0]])[0, 0]
    assert np.isclose(q, np.sum(O.tangent_gather(Uh, Vh, xi32, cfg.idx) ** 2), rtol=1e-4)


def test_completion_hvp_out_of_range_index(lib):
    cfg = S.config1()
    X = round32(cfg.X)
    U, V, Uh, Vh = _uv(lib, X)
    bad = cfg.idx.copy()
    bad[2, 5] = 3  # n = 3: one past the end, clamped on the device and recorded
    xi = [np.zeros((1,) + c.shape) for c in Uh]
    _, ws = lib.completion_hvp(U, V, torch.tensor(bad, device="cuda"), dev_tt(lib, xi), return_ws=True)
    assert lib.device_status(ws) == -1


def test_tangent_gram_tf32_projected_config5_shape(lib):
    # TMA + tcgen05 TF32 path on the self Gram matrix of 48 projected rank-8 TTs (one operand
    # per diagonal tile), diagonal and off-diagonal entries within the TF32 tolerance
    cfg = S.config5(batch=48)
    X, Z, c = round32(cfg.X), round32(cfg.Z), cfg.c.astype(np.float32)
    U, V, Uh, Vh = _uv(lib, X)
    dU = lib.project(U, V, dev_tt(lib, Z), torch.tensor(c, device="cuda"))
    G = lib.tangent_gram(dU, dU, math="tf32").double().cpu().numpy()
    coords = host_objects(dU)
    assert_gram_blocks(G, O.tangent_gram(coords, coords), [48], TOL["tf32"])


def test_tangent_gram_tf32_two_operands_several_tiles(lib):
    # 200 x 130 pairs: 2 x 2 tiles of 128, both operands loaded, ragged tile edges
    rng = np.random.default_rng(701)
    n, r = [4, 4, 4, 4, 4], [1, 4, 8, 8, 4, 1]
    dA = round32(S.random_tt(rng, 200, n, r))
    dB = round32(S.random_tt(rng, 130, n, r))
    G = lib.tangent_gram(dev_tt(lib, dA), dev_tt(lib, dB), math="tf32").double().cpu().numpy()
    Gref = O.tangent_gram(objects(dA), objects(dB))
    assert G.shape == (200, 130)
    assert rel_err(G, Gref) < TOL["tf32"]
    # the FP32 path on the same inputs
    G32 = lib.tangent_gram(dev_tt(lib, dA), dev_tt(lib, dB)).double().cpu().numpy()
    assert rel_err(G32, Gref) < TOL["fp32"]


def test_tangent_gram_tf32_rejects_unaligned_rows(lib):
    rng = np.random.default_rng(702)
    dA = round32(S.random_tt(rng, 5, [3, 3], [1, 3, 1]))  # 9 floats per core row
    with pytest.raises(lib.T3FError) as e:
        lib.tangent_gram(dev_tt(lib, dA), dev_tt(lib, dA), math="tf32")
    assert e.value.status == -7
