"""GPU parity: every C-ABI entry point against the FP64 oracle on the same seeded inputs.

Inputs are drawn by `synth`, rounded once to FP32, and the same rounded values are given to
the oracle (widened to FP64) and to the CUDA path. The error measure is the normwise
relative error of each output array; the FP32 tolerance is 1e-5. Index bookkeeping
(orthogonal ranks, device error words) must match exactly.
"""
import math

import numpy as np
import pytest

import oracle as O
import synth as S
from tests._util import TOL, batched, objects, rel_err, rel_err_cores, round32

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def dev_tt(t3f, cores, dtype=None):
    return t3f.TT.from_cores([np.asarray(c, np.float32) for c in cores],
                             dtype=dtype or torch.float32, device="cuda")


def host_cores(tt):
    return [c.detach().double().cpu().numpy() for c in tt.cores()]


def host_objects(tt):
    return objects(host_cores(tt))


# ---------------------------------------------------------------------------------------
# Gram / norm
# ---------------------------------------------------------------------------------------

def _gram_case(t3f, A, B):
    A, B = round32(A), round32(B)
    G = t3f.gram(dev_tt(t3f, A), dev_tt(t3f, B)).double().cpu().numpy()
    Gref = O.gram(objects(A), objects(B))
    return G, Gref


def test_gram_config1(lib):
    cfg = S.config1()
    G, Gref = _gram_case(lib, cfg.A, cfg.B)
    assert rel_err(G, Gref) < TOL["fp32"]


def test_gram_ragged_tiles_mixed_ranks(lib):
    rng = np.random.default_rng(100)
    n = [5, 3, 4, 6, 2, 5]
    A = S.random_tt(rng, 37, n, [1, 3, 4, 5, 4, 3, 1], 0.5)
    B = S.random_tt(rng, 29, n, [1, 2, 6, 3, 7, 2, 1], 0.5)
    G, Gref = _gram_case(lib, A, B)
    assert G.shape == (37, 29)
    assert rel_err(G, Gref) < TOL["fp32"]


def test_gram_config3_full(lib):
    cfg = S.config3a()
    G, Gref = _gram_case(lib, cfg.A, cfg.B)
    assert G.shape == (100, 100)
    assert rel_err(G, Gref) < TOL["fp32"]


def test_gram_large_rank_and_d1(lib):
    rng = np.random.default_rng(101)
    A = S.random_tt(rng, 3, [4, 3, 5], [1, 40, 64, 1], 0.2)
    B = S.random_tt(rng, 2, [4, 3, 5], [1, 17, 33, 1], 0.2)
    G, Gref = _gram_case(lib, A, B)
    assert rel_err(G, Gref) < TOL["fp32"]
    # d = 1: a plain vector inner product
    A1 = S.random_tt(rng, 4, [7], [1, 1])
    B1 = S.random_tt(rng, 3, [7], [1, 1])
    G, Gref = _gram_case(lib, A1, B1)
    assert rel_err(G, Gref) < TOL["fp32"]


def test_norm(lib):
    cfg = S.config3a(bA=13, bB=1)
    A = round32(cfg.A)
    nrm = lib.norm(dev_tt(lib, A)).cpu().numpy()
    ref = np.array([O.norm(a) for a in objects(A)])
    assert rel_err(nrm, ref) < TOL["fp32"]


def test_norm_dtypes_ranks_and_large_cores(lib):
    # BF16-stored cores (exact in FP32 arithmetic), ranks that change from core to core, d = 1,
    # and a core too large for whole-core staging (16 x 16 x 64: two copies and the slice
    # products exceed the budget, so the slice-by-slice sweep takes the batch)
    from tests._util import round_bf16
    rng = np.random.default_rng(150)
    cases = [(S.random_tt(rng, 9, [3, 5, 2, 4], [1, 6, 11, 3, 1], 0.4), torch.bfloat16, True),
             (S.random_tt(rng, 5, [6], [1, 1], 1.0), torch.float32, False),
             (S.random_tt(rng, 3, [16, 16, 16], [1, 16, 64, 1], 0.125), torch.float32, False)]
    for A, dt, bf in cases:
        A = round_bf16(A) if bf else round32(A)
        nrm = lib.norm(dev_tt(lib, A, dt)).cpu().numpy()
        ref = np.array([O.norm(a) for a in objects(A)])
        assert rel_err(nrm, ref) < TOL["fp32"], (dt, len(A))


def test_gram_backward(lib):
    rng = np.random.default_rng(102)
    n = [3, 4, 2, 3, 5]
    A = round32(S.random_tt(rng, 11, n, [1, 3, 4, 2, 3, 1]))
    B = round32(S.random_tt(rng, 9, n, [1, 2, 3, 5, 2, 1]))
    dG = rng.normal(size=(11, 9)).astype(np.float32)
    dA, dB = lib.gram_backward(dev_tt(lib, A), dev_tt(lib, B), torch.tensor(dG, device="cuda"))
    rA, rB = O.gram_vjp(objects(A), objects(B), dG.astype(np.float64))
    assert rel_err_cores(host_cores(dA), batched(rA)) < TOL["fp32"]
    assert rel_err_cores(host_cores(dB), batched(rB)) < TOL["fp32"]


def test_gram_backward_config3_sampled(lib):
    cfg = S.config3a()
    A, B = round32(cfg.A), round32(cfg.B)
    dG = np.random.default_rng(103).normal(size=(100, 100)).astype(np.float32)
    dA, dB = lib.gram_backward(dev_tt(lib, A), dev_tt(lib, B), torch.tensor(dG, device="cuda"))
    hA, hB = host_objects(dA), host_objects(dB)
    oa, ob = objects(A), objects(B)
    for a in (0, 57, 99):
        rA, _ = O.gram_vjp([oa[a]], ob, dG[a:a + 1].astype(np.float64))
        assert rel_err_cores(hA[a], rA[0]) < TOL["fp32"]
    for b in (3, 64):
        _, rB = O.gram_vjp(oa, [ob[b]], dG[:, b:b + 1].astype(np.float64))
        assert rel_err_cores(hB[b], rB[0]) < TOL["fp32"]


# ---------------------------------------------------------------------------------------
# Gather / completion loss / adjoints
# ---------------------------------------------------------------------------------------

def _completion_inputs(cfg_T, cfg_X, idx, noise):
    T = round32(cfg_T)
    X = round32(cfg_X)
    y = (O.gather(objects(T)[0], idx) + noise).astype(np.float32).astype(np.float64)
    return X, y


def test_gather_and_loss_config1(lib):
    cfg = S.config1()
    X, y = _completion_inputs(cfg.A, cfg.X, cfg.idx, cfg.noise)
    idx = torch.tensor(cfg.idx, device="cuda")
    yt = torch.tensor(y, dtype=torch.float32, device="cuda")
    vals, loss = lib.gather(dev_tt(lib, X), idx, yt, want_vals=True, want_loss=True)
    Xo = objects(X)[0]
    assert rel_err(vals.cpu().numpy(), O.gather(Xo, cfg.idx)) < TOL["fp32"]
    assert abs(loss.item() - O.completion_loss(Xo, cfg.idx, y)) <= TOL["fp32"] * O.completion_loss(Xo, cfg.idx, y)


@pytest.mark.parametrize("N", [0, 1, 129, 20011])
def test_gather_backward_sizes(lib, N):
    rng = np.random.default_rng(104 + N)
    n = [10] * 10
    X = round32(S.random_tt(rng, 1, n, S.tt_ranks(10, 8), 1 / math.sqrt(8)))
    idx = S.random_indices(rng, N, n)
    y = rng.normal(size=N).astype(np.float32).astype(np.float64)
    dX, loss = lib.gather_backward(dev_tt(lib, X), torch.tensor(idx, device="cuda"),
                                   y=torch.tensor(y, dtype=torch.float32, device="cuda"), want_loss=True)
    Xo = objects(X)[0]
    if N == 0:
        assert loss.item() == 0.0
        assert float(dX.data.abs().max()) == 0.0
        return
    L, g = O.completion_loss_grad(Xo, idx, y)
    assert abs(loss.item() - L) <= TOL["fp32"] * L
    assert rel_err_cores(host_objects(dX)[0], g) < TOL["fp32"]


def test_gather_backward_weights_and_ranks(lib):
    rng = np.random.default_rng(105)
    n = [3, 7, 2, 5]
    X = round32(S.random_tt(rng, 1, n, [1, 3, 5, 2, 1]))
    idx = S.random_indices(rng, 3001, n)
    w = rng.normal(size=3001).astype(np.float32)
    dX, _ = lib.gather_backward(dev_tt(lib, X), torch.tensor(idx, device="cuda"),
                                w=torch.tensor(w, device="cuda"))
    ref = O.gather_vjp(objects(X)[0], idx, w.astype(np.float64))
    assert rel_err_cores(host_objects(dX)[0], ref) < TOL["fp32"]


def test_completion_config2_full(lib):
    cfg = S.config2()
    X, y = _completion_inputs(cfg.T, cfg.X, cfg.idx, cfg.noise)
    Xd = dev_tt(lib, X)
    idx = torch.tensor(cfg.idx, device="cuda")
    yt = torch.tensor(y, dtype=torch.float32, device="cuda")
    vals, loss = lib.gather(Xd, idx, yt, want_vals=True, want_loss=True)
    dX, loss2 = lib.gather_backward(Xd, idx, y=yt, want_loss=True)
    Xo = objects(X)[0]
    ref_vals = O.gather(Xo, cfg.idx)
    assert rel_err(vals.cpu().numpy(), ref_vals) < TOL["fp32"]
    L, g = O.completion_loss_grad(Xo, cfg.idx, y)
    assert abs(loss.item() - L) <= TOL["fp32"] * L
    assert abs(loss2.item() - L) <= TOL["fp32"] * L
    assert rel_err_cores(host_objects(dX)[0], g) < TOL["fp32"]


def test_gather_out_of_range_index_sets_device_error(lib):
    rng = np.random.default_rng(106)
    n = [4, 4, 4]
    X = round32(S.random_tt(rng, 1, n, [1, 2, 2, 1]))
    idx = S.random_indices(rng, 100, n)
    idx[1, 17] = 4  # one past the end of mode 1
    _, _, ws = lib.gather_backward(dev_tt(lib, X), torch.tensor(idx, device="cuda"),
                                   w=torch.ones(100, device="cuda"), return_ws=True)
    assert lib.device_status(ws) == -1  # T3F_ERR_ARG recorded on the device


# ---------------------------------------------------------------------------------------
# Orthogonalisation / Riemannian operations
# ---------------------------------------------------------------------------------------

def _orth(lib, X, dtype=torch.float64):
    U, V = lib.orthogonalize(dev_tt(lib, X), dtype=dtype)
    return U, V


@pytest.mark.parametrize("case", ["config1", "redundant", "config5"])
def test_orthogonalize(lib, case):
    rng = np.random.default_rng(107)
    if case == "config1":
        X = round32(S.config1().X)
    elif case == "redundant":
        X = round32(S.random_tt(rng, 2, [2, 3, 4, 2], [1, 4, 5, 6, 1]))
    else:
        X = round32(S.config5(batch=1).X)
    U, V = _orth(lib, X)
    for b, Xo in enumerate(objects(X)):
        Ur, Vr, r = O.orthogonalize(Xo)
        assert U.ranks == r and V.ranks == r  # integer bookkeeping, exact
        Ug, Vg = host_objects(U)[b], host_objects(V)[b]
        assert rel_err_cores(Ug, Ur) < 1e-9
        assert rel_err_cores(Vg, Vr) < 1e-9


def test_project_sum_config1(lib):
    cfg = S.config1()
    X = round32(cfg.X)
    Z = round32(cfg.B)
    c = cfg.c.astype(np.float32)
    U, V = _orth(lib, X, torch.float32)
    dU = lib.project_sum(U, V, dev_tt(lib, Z), torch.tensor(c, device="cuda"))
    Uo, Vo, _ = O.orthogonalize(objects(X)[0])
    ref = O.project_sum(Uo, Vo, objects(Z), c.astype(np.float64))
    assert rel_err_cores(host_objects(dU)[0], ref) < TOL["fp32"]


def test_project_sum_config5_full(lib):
    cfg = S.config5()
    X, Z = round32(cfg.X), round32(cfg.Z)
    c = cfg.c.astype(np.float32)
    U, V = _orth(lib, X, torch.float32)
    dU = lib.project_sum(U, V, dev_tt(lib, Z), torch.tensor(c, device="cuda"))
    Uo, Vo, _ = O.orthogonalize(objects(X)[0])
    ref = O.project_sum(Uo, Vo, objects(Z), c.astype(np.float64))
    assert rel_err_cores(host_objects(dU)[0], ref) < TOL["fp32"]


def test_project_sum_config5_invariants_on_gpu(lib):
    # P o P = P and P_X X = X, checked on the library's own outputs: the tangent vector S of
    # project_sum (its rank-2r TT built from the GPU's U, V and dU) projected again on the GPU
    # gives back the same coordinates; X itself projects to dU_k = 0 (k < d), dU_d = U_d.
    cfg = S.config5()
    X, Z = round32(cfg.X), round32(cfg.Z)
    c = cfg.c.astype(np.float32)
    U, V = _orth(lib, X, torch.float32)
    dU = lib.project_sum(U, V, dev_tt(lib, Z), torch.tensor(c, device="cuda"))
    Uh, Vh, dUh = host_objects(U)[0], host_objects(V)[0], host_objects(dU)[0]
    S_tt = O.tangent_to_tt(Uh, Vh, dUh)
    assert max(O.tt_ranks_of(S_tt)) <= 2 * max(U.ranks)  # tangent rank <= 2r
    one = torch.ones(1, device="cuda")
    dU2 = lib.project_sum(U, V, dev_tt(lib, [s_[None] for s_ in S_tt]), one)
    assert rel_err_cores(host_objects(dU2)[0], dUh) < TOL["fp32"]
    dUx = host_objects(lib.project_sum(U, V, dev_tt(lib, X), one))[0]
    d = len(dUx)
    scale = np.linalg.norm(Uh[-1])
    assert max(np.linalg.norm(dUx[k]) for k in range(d - 1)) < TOL["fp32"] * scale
    assert rel_err(dUx[-1], Uh[-1]) < TOL["fp32"]


def test_project_sum_backward(lib):
    cfg = S.config5(batch=37, d=6, n=5, rX=6, rZ=3)
    X, Z = round32(cfg.X), round32(cfg.Z)
    c = cfg.c.astype(np.float32)
    U, V = _orth(lib, X, torch.float32)
    Uo, Vo, r = O.orthogonalize(objects(X)[0])
    rng = np.random.default_rng(108)
    dUbar = [rng.normal(size=(1, r[k], 5, r[k + 1])).astype(np.float32) for k in range(6)]
    dZ, dc = lib.project_sum_backward(U, V, dev_tt(lib, Z), torch.tensor(c, device="cuda"),
                                      dev_tt(lib, dUbar))
    rZ, rc = O.project_sum_vjp(Uo, Vo, objects(Z), c.astype(np.float64), [u[0].astype(np.float64) for u in dUbar])
    assert rel_err_cores(host_cores(dZ), batched(rZ)) < TOL["fp32"]
    assert rel_err(dc.cpu().numpy(), rc) < TOL["fp32"]


def test_riemannian_grad_completion(lib):
    rng = np.random.default_rng(109)
    n = [6] * 6
    T = S.random_tt(rng, 1, n, S.tt_ranks(6, 3), 0.6)
    X = round32(S.random_tt(rng, 1, n, S.tt_ranks(6, 5), 0.45))
    idx = S.random_indices(rng, 5003, n)
    y = (O.gather(objects(round32(T))[0], idx) + 0.01 * rng.normal(size=5003)).astype(np.float32).astype(np.float64)
    U, V = _orth(lib, X, torch.float32)
    dU, loss = lib.gather_backward(None, torch.tensor(idx, device="cuda"),
                                   y=torch.tensor(y, dtype=torch.float32, device="cuda"),
                                   want_loss=True, riemannian=True, U=U, V=V)
    Uo, Vo, _ = O.orthogonalize(objects(X)[0])
    L, ref = O.riemannian_grad_completion(Uo, Vo, idx, y)
    assert abs(loss.item() - L) <= TOL["fp32"] * L
    assert rel_err_cores(host_objects(dU)[0], ref) < TOL["fp32"]


# ---------------------------------------------------------------------------------------
# Matvec
# ---------------------------------------------------------------------------------------

@pytest.mark.parametrize("bA,bx", [(7, 7), (1, 5), (4, 1)])
def test_matvec_and_backward(lib, bA, bx):
    rng = np.random.default_rng(110 + bA)
    d = 4
    m, n = [2, 3, 4, 2], [3, 2, 4, 3]
    A = round32(S.random_ttm(rng, bA, m, n, [1, 3, 4, 2, 1]))
    x = round32(S.random_tt(rng, bx, n, [1, 2, 5, 3, 1]))
    Ad, xd = dev_tt(lib, A), dev_tt(lib, x)
    C = lib.matvec(Ad, xd)
    P = max(bA, bx)
    Ao, xo = objects(A), objects(x)
    refC = [O.matvec(Ao[0 if bA == 1 else p], xo[0 if bx == 1 else p]) for p in range(P)]
    assert C.ranks == [1, 6, 20, 6, 1]
    assert rel_err_cores(host_cores(C), batched(refC)) < TOL["fp32"]
    dC = [rng.normal(size=c.shape).astype(np.float32) for c in host_cores(C)]
    dA, dx = lib.matvec_backward(Ad, xd, dev_tt(lib, dC))
    rdA = [np.zeros_like(c) for c in A]
    rdx = [np.zeros_like(c) for c in x]
    dCo = objects(dC)
    for p in range(P):
        ga, gx = O.matvec_vjp(Ao[0 if bA == 1 else p], xo[0 if bx == 1 else p], dCo[p])
        for k in range(d):
            rdA[k][0 if bA == 1 else p] += ga[k]
            rdx[k][0 if bx == 1 else p] += gx[k]
    assert rel_err_cores(host_cores(dA), rdA) < TOL["fp32"]
    assert rel_err_cores(host_cores(dx), rdx) < TOL["fp32"]


def test_matvec_config3b_sampled(lib):
    cfg = S.config3b()
    A, x = round32(cfg.A), round32(cfg.x)
    C = lib.matvec(dev_tt(lib, A), dev_tt(lib, x))
    assert C.ranks == [1] + [100] * 9 + [1]
    hc = host_objects(C)
    Ao, xo = objects(A), objects(x)
    for p in (0, 41, 99):
        assert rel_err_cores(hc[p], O.matvec(Ao[p], xo[p])) < TOL["fp32"]


def test_matvec_backward_config3b_sampled(lib):
    # the rank-100 adjoint the benchmark times, full batch, with a random cotangent of the
    # product's shape; sampled pairs against the oracle's vjp
    cfg = S.config3b()
    A, x = round32(cfg.A), round32(cfg.x)
    rc = [a * b for a, b in zip(S.tt_ranks(10, 10), S.tt_ranks(10, 10))]
    rng = np.random.default_rng(112)
    dC = [rng.normal(size=(100, rc[k], 4, rc[k + 1])).astype(np.float32) for k in range(10)]
    dA, dx = lib.matvec_backward(dev_tt(lib, A), dev_tt(lib, x), dev_tt(lib, dC))
    hA, hx = host_objects(dA), host_objects(dx)
    Ao, xo, Co = objects(A), objects(x), objects(round32(dC))
    for p in (0, 41, 99):
        rA, rx = O.matvec_vjp(Ao[p], xo[p], Co[p])
        assert rel_err_cores(hA[p], rA) < TOL["fp32"], p
        assert rel_err_cores(hx[p], rx) < TOL["fp32"], p


def test_riemannian_grad_config2_full(lib):
    cfg = S.config2()
    X, y = _completion_inputs(cfg.T, cfg.X, cfg.idx, cfg.noise)
    U, V = _orth(lib, X, torch.float32)
    dU, loss = lib.gather_backward(None, torch.tensor(cfg.idx, device="cuda"),
                                   y=torch.tensor(y, dtype=torch.float32, device="cuda"),
                                   want_loss=True, riemannian=True, U=U, V=V)
    Uo, Vo, _ = O.orthogonalize(objects(X)[0])
    L, ref = O.riemannian_grad_completion(Uo, Vo, cfg.idx, y)
    assert abs(loss.item() - L) <= TOL["fp32"] * L
    assert rel_err_cores(host_objects(dU)[0], ref) < TOL["fp32"]


@pytest.mark.parametrize("shape", [dict(batch=160, d=20, n=16, rX=32, rZ=8),   # config-5 shape
                                   dict(batch=23, d=5, n=4, rX=12, rZ=5),     # rank-16 tiles
                                   dict(batch=9, d=3, n=7, rX=20, rZ=8)])
def test_project_sum_fwd_bwd_shapes(lib, shape):
    cfg = S.config5(**shape)
    X, Z = round32(cfg.X), round32(cfg.Z)
    c = cfg.c.astype(np.float32)
    U, V = _orth(lib, X, torch.float32)
    Zd = dev_tt(lib, Z)
    ct = torch.tensor(c, device="cuda")
    dU = lib.project_sum(U, V, Zd, ct)
    Uo, Vo, r = O.orthogonalize(objects(X)[0])
    ref = O.project_sum(Uo, Vo, objects(Z), c.astype(np.float64))
    assert rel_err_cores(host_objects(dU)[0], ref) < TOL["fp32"]
    # adjoint of 1/2 ||S||^2: the cotangent of the coordinates is the forward output
    dZ, dc = lib.project_sum_backward(U, V, Zd, ct, dU)
    rZ, rc = O.project_sum_vjp(Uo, Vo, objects(Z), c.astype(np.float64), host_objects(dU)[0])
    assert rel_err_cores(host_cores(dZ), batched(rZ)) < TOL["fp32"]
    assert rel_err(dc.cpu().numpy(), rc) < TOL["fp32"]


def test_project_sum_tf32_config5_full(lib):
    # the U- and V-side contractions of both sweeps on the tensor cores (TF32), at config 5
    cfg = S.config5()
    X, Z = round32(cfg.X), round32(cfg.Z)
    c = cfg.c.astype(np.float32)
    U, V = _orth(lib, X, torch.float32)
    Zt, ct = dev_tt(lib, Z), torch.tensor(c, device="cuda")
    dU = lib.project_sum(U, V, Zt, ct, math="tf32")
    Uo, Vo, _ = O.orthogonalize(objects(X)[0])
    ref = O.project_sum(Uo, Vo, objects(Z), c.astype(np.float64))
    err = rel_err_cores(host_objects(dU)[0], ref)
    assert err < TOL["tf32"]
    assert err > 1e-7  # the reduced-precision path really ran


def test_project_sum_tf32_ragged_batch(lib):
    # 37 objects (the last CTA holds 5), X ranks 1..12, Z ranks 5, modes 8
    cfg = S.config5(batch=37, d=6, n=8, rX=12, rZ=5)
    X, Z = round32(cfg.X), round32(cfg.Z)
    c = cfg.c.astype(np.float32)
    U, V = _orth(lib, X, torch.float32)
    dU = lib.project_sum(U, V, dev_tt(lib, Z), torch.tensor(c, device="cuda"), math="tf32")
    Uo, Vo, _ = O.orthogonalize(objects(X)[0])
    ref = O.project_sum(Uo, Vo, objects(Z), c.astype(np.float64))
    assert rel_err_cores(host_objects(dU)[0], ref) < TOL["tf32"]


def test_project_sum_reduced_precision_limits(lib):
    # modes that are not multiples of 8 have no tensor-core form, nor has BF16: both refused
    cfg = S.config1()
    X, Z = round32(cfg.X), round32(cfg.B)
    U, V = _orth(lib, X, torch.float32)
    Zt, c = dev_tt(lib, Z), torch.tensor(cfg.c.astype(np.float32), device="cuda")
    for m in ("tf32", "bf16"):
        with pytest.raises(lib.T3FError) as e:
            lib.project_sum(U, V, Zt, c, math=m)
        assert e.value.status == -7
