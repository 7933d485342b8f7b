"""Pins for the FP64 oracle: each routine is checked against something other than itself
(hand-evaluated fixtures, brute force over the full tensor, textbook special cases, closed
forms, invariants of the tangent-space projector, central finite differences)."""
import json
import os

import numpy as np
import pytest

import oracle as O
import synth as S

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def single(cores_batched, b=0):
    return [c[b] for c in cores_batched]


def rand_tt(rng, n, ranks, std=1.0):
    return single(S.random_tt(rng, 1, n, ranks, std))


# ---------------------------------------------------------------------------------------
# TT definition
# ---------------------------------------------------------------------------------------

def test_full_matches_hand_worked_example():
    g = json.load(open(os.path.join(GOLDEN, "tt_d3_n2_r2_hand.json")))
    cores = [np.array(c, dtype=float) for c in g["cores"]]
    np.testing.assert_array_equal(O.full(cores), np.array(g["full"], dtype=float))
    np.testing.assert_array_equal(O.full_brute(cores), np.array(g["full"], dtype=float))
    assert O.dot(cores, cores) == g["squared_norm"]


@pytest.mark.parametrize("n,ranks", [([3, 3, 3, 3], [1, 2, 2, 2, 1]),
                                     ([2, 3, 2], [1, 2, 3, 1]),
                                     ([4], [1, 1])])
def test_full_matches_nested_sum(n, ranks):
    rng = np.random.default_rng(10)
    X = rand_tt(rng, n, ranks)
    np.testing.assert_allclose(O.full(X), O.full_brute(X), rtol=1e-13, atol=1e-13)


def test_full_special_cases():
    rng = np.random.default_rng(11)
    # d = 2: the TT is the matrix product G1 G2
    A = rand_tt(rng, [4, 5], [1, 3, 1])
    np.testing.assert_allclose(O.full(A), A[0][0] @ A[1][:, :, 0], rtol=1e-14)
    # rank 1: outer product of the core vectors
    v = [rng.normal(size=k) for k in (2, 3, 4)]
    cores = [x.reshape(1, -1, 1) for x in v]
    np.testing.assert_allclose(O.full(cores), np.multiply.outer(np.multiply.outer(v[0], v[1]), v[2]))


def test_storage_count_formula():
    # Section 1: r n (r (d - 2) + 2) numbers for d cores of mode n and rank r
    for d, n, r in [(4, 3, 2), (10, 10, 10), (20, 16, 32)]:
        cores = S.random_tt(np.random.default_rng(0), 1, n, S.tt_ranks(d, r))
        assert sum(c.size for c in cores) == r * n * (r * (d - 2) + 2)


def test_tt_add_scale():
    rng = np.random.default_rng(12)
    A = rand_tt(rng, [3, 2, 3], [1, 2, 2, 1])
    B = rand_tt(rng, [3, 2, 3], [1, 3, 1, 1])
    np.testing.assert_allclose(O.full(O.tt_add(A, B)), O.full(A) + O.full(B), rtol=1e-13)
    np.testing.assert_allclose(O.full(O.tt_scale(A, -2.5)), -2.5 * O.full(A), rtol=1e-14)


# ---------------------------------------------------------------------------------------
# Inner products / Gram / norm
# ---------------------------------------------------------------------------------------

def test_dot_brute_force_config1():
    cfg = S.config1()
    for a in range(8):
        for b in range(8):
            A, B = single(cfg.A, a), single(cfg.B, b)
            ref = float(np.sum(O.full(A) * O.full(B)))
            assert abs(O.dot(A, B) - ref) <= 1e-12 * (1 + abs(ref))


def test_dot_closed_forms_and_bilinearity():
    rng = np.random.default_rng(13)
    n, ranks = [3, 4, 2, 3], [1, 2, 3, 2, 1]
    A, A2 = rand_tt(rng, n, ranks), rand_tt(rng, n, [1, 3, 2, 2, 1])
    B = rand_tt(rng, n, [1, 2, 2, 3, 1])
    assert np.isclose(O.dot(A, A), np.sum(O.full(A) ** 2), rtol=1e-13)
    assert np.isclose(O.norm(A), np.linalg.norm(O.full(A).ravel()), rtol=1e-13)
    al, be = 0.7, -1.3
    lhs = O.dot(O.tt_add(O.tt_scale(A, al), O.tt_scale(A2, be)), B)
    assert np.isclose(lhs, al * O.dot(A, B) + be * O.dot(A2, B), rtol=1e-12)
    assert np.isclose(O.dot(A, B), O.dot(B, A), rtol=1e-13)
    # d = 2: <A, B> = trace(A1 A2 (B1 B2)^T), a plain matrix inner product
    P = rand_tt(rng, [5, 6], [1, 3, 1])
    Q = rand_tt(rng, [5, 6], [1, 2, 1])
    Pm, Qm = P[0][0] @ P[1][:, :, 0], Q[0][0] @ Q[1][:, :, 0]
    assert np.isclose(O.dot(P, Q), np.trace(Pm @ Qm.T), rtol=1e-13)


def test_gram_symmetric_and_norms():
    cfg = S.config1()
    As = [single(cfg.A, a) for a in range(8)]
    G = O.gram(As, As)
    np.testing.assert_allclose(G, G.T, rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(np.sqrt(np.diag(G)), [O.norm(A) for A in As], rtol=1e-13)
    assert np.all(np.linalg.eigvalsh(G) > -1e-9)  # a Gram matrix is PSD


def test_gram_vjp_matches_finite_differences():
    rng = np.random.default_rng(14)
    n, ranks = [3, 2, 3], [1, 2, 3, 1]
    As = [rand_tt(rng, n, ranks) for _ in range(2)]
    Bs = [rand_tt(rng, n, [1, 3, 2, 1]) for _ in range(3)]
    Gbar = rng.normal(size=(2, 3))
    dAs, dBs = O.gram_vjp(As, Bs, Gbar)
    f = lambda As_, Bs_: float(np.sum(Gbar * O.gram(As_, Bs_)))
    h = 1e-6
    for a in range(2):
        for k in range(3):
            D = rng.normal(size=As[a][k].shape)
            Ap = [list(x) for x in As]; Am = [list(x) for x in As]
            Ap[a][k] = As[a][k] + h * D; Am[a][k] = As[a][k] - h * D
            fd = (f(Ap, Bs) - f(Am, Bs)) / (2 * h)
            assert np.isclose(fd, np.sum(dAs[a][k] * D), rtol=1e-7, atol=1e-8)
    for b in range(3):
        for k in range(3):
            D = rng.normal(size=Bs[b][k].shape)
            Bp = [list(x) for x in Bs]; Bm = [list(x) for x in Bs]
            Bp[b][k] = Bs[b][k] + h * D; Bm[b][k] = Bs[b][k] - h * D
            fd = (f(As, Bp) - f(As, Bm)) / (2 * h)
            assert np.isclose(fd, np.sum(dBs[b][k] * D), rtol=1e-7, atol=1e-8)


def test_partials_contract_to_the_dot_at_every_interface():
    rng = np.random.default_rng(15)
    A = rand_tt(rng, [3, 3, 3, 3], [1, 2, 3, 2, 1])
    B = rand_tt(rng, [3, 3, 3, 3], [1, 3, 2, 2, 1])
    M, R = O.left_partials(A, B), O.right_partials(A, B)
    for k in range(1, 5):
        assert np.isclose(np.sum(M[k - 1] * R[k]), O.dot(A, B), rtol=1e-12)


# ---------------------------------------------------------------------------------------
# Gather / completion loss
# ---------------------------------------------------------------------------------------

def test_gather_is_full_entry():
    cfg = S.config1()
    X = single(cfg.X)
    F = O.full(X)
    np.testing.assert_allclose(O.gather(X, cfg.idx), F[tuple(cfg.idx)], rtol=1e-13, atol=1e-13)
    # d = 2: a row of G1 times a column of G2
    rng = np.random.default_rng(16)
    P = rand_tt(rng, [5, 6], [1, 3, 1])
    idx = S.random_indices(rng, 50, [5, 6])
    ref = np.array([P[0][0, i, :] @ P[1][:, j, 0] for i, j in idx.T])
    np.testing.assert_allclose(O.gather(P, idx), ref, rtol=1e-14)


def test_gather_vjp_is_jacobian_transpose():
    # dG^k = J^T vec(W) with W the dense tensor of scattered weights
    cfg = S.config1()
    X = single(cfg.X)
    w = np.random.default_rng(17).normal(size=cfg.idx.shape[1])
    g = O.gather_vjp(X, cfg.idx, w)
    W = np.zeros(O.full(X).shape)
    np.add.at(W, tuple(cfg.idx), w)
    J = O.tangent_basis_jacobian(X)
    np.testing.assert_allclose(np.concatenate([x.ravel() for x in g]), J.T @ W.ravel(),
                               rtol=1e-11, atol=1e-11)


def test_completion_loss_grad_finite_differences():
    cfg = S.config1()
    X = single(cfg.X)
    y = O.gather(single(cfg.A, 0), cfg.idx) + cfg.noise
    L, g = O.completion_loss_grad(X, cfg.idx, y)
    res = O.full(X)[tuple(cfg.idx)] - y
    assert np.isclose(L, 0.5 * np.sum(res ** 2), rtol=1e-13)
    rng = np.random.default_rng(18)
    h = 1e-6
    for k in range(4):
        D = rng.normal(size=X[k].shape)
        Xp = list(X); Xm = list(X)
        Xp[k] = X[k] + h * D; Xm[k] = X[k] - h * D
        fd = (O.completion_loss(Xp, cfg.idx, y) - O.completion_loss(Xm, cfg.idx, y)) / (2 * h)
        assert np.isclose(fd, np.sum(g[k] * D), rtol=1e-7)


# ---------------------------------------------------------------------------------------
# Matvec
# ---------------------------------------------------------------------------------------

def test_full_matrix_kron_and_matvec_dense():
    rng = np.random.default_rng(19)
    # rank-1 TT-matrix == Kronecker product of its factor matrices
    F = [rng.normal(size=(2, 3)), rng.normal(size=(3, 2)), rng.normal(size=(2, 2))]
    cores = [f.reshape(1, *f.shape, 1) for f in F]
    np.testing.assert_allclose(O.full_matrix(cores), np.kron(np.kron(F[0], F[1]), F[2]), rtol=1e-13)
    # matvec == dense M v at d=3, m=n=2
    A = [rng.normal(size=s) for s in [(1, 2, 2, 3), (3, 2, 2, 2), (2, 2, 2, 1)]]
    x = rand_tt(rng, [2, 2, 2], [1, 2, 3, 1])
    C = O.matvec(A, x)
    assert O.tt_ranks_of(C) == [1, 6, 6, 1]
    np.testing.assert_allclose(O.full(C).ravel(), O.full_matrix(A) @ O.full(x).ravel(), rtol=1e-12)
    # identity TT-matrix (rank-1 delta cores) leaves x unchanged
    I = [np.eye(2).reshape(1, 2, 2, 1)] * 3
    np.testing.assert_allclose(O.full(O.matvec(I, x)), O.full(x), rtol=1e-14)


def test_matvec_vjp_finite_differences():
    rng = np.random.default_rng(20)
    A = [rng.normal(size=s) for s in [(1, 2, 3, 2), (2, 3, 2, 2), (2, 2, 2, 1)]]
    x = rand_tt(rng, [3, 2, 2], [1, 3, 2, 1])
    C = O.matvec(A, x)
    dC = [rng.normal(size=c.shape) for c in C]
    dA, dx = O.matvec_vjp(A, x, dC)
    f = lambda A_, x_: sum(float(np.sum(g * c)) for g, c in zip(dC, O.matvec(A_, x_)))
    h = 1e-6
    for k in range(3):
        D = rng.normal(size=A[k].shape)
        Ap = list(A); Am = list(A); Ap[k] = A[k] + h * D; Am[k] = A[k] - h * D
        assert np.isclose((f(Ap, x) - f(Am, x)) / (2 * h), np.sum(dA[k] * D), rtol=1e-7)
        D = rng.normal(size=x[k].shape)
        xp = list(x); xm = list(x); xp[k] = x[k] + h * D; xm[k] = x[k] - h * D
        assert np.isclose((f(A, xp) - f(A, xm)) / (2 * h), np.sum(dx[k] * D), rtol=1e-7)


# ---------------------------------------------------------------------------------------
# Orthogonalisation
# ---------------------------------------------------------------------------------------

@pytest.mark.parametrize("n,ranks", [([3, 3, 3, 3], [1, 2, 2, 2, 1]),
                                     ([2, 3, 4, 2], [1, 4, 5, 6, 1]),   # redundant ranks
                                     ([4, 4, 4], [1, 3, 3, 1])])
def test_orthogonalize_invariants(n, ranks):
    rng = np.random.default_rng(21)
    X = rand_tt(rng, n, ranks)
    U, V, r = O.orthogonalize(X)
    d = len(n)
    F = O.full(X)
    np.testing.assert_allclose(O.full(U), F, rtol=1e-11, atol=1e-12)
    np.testing.assert_allclose(O.full(V), F, rtol=1e-11, atol=1e-12)
    for k in range(d - 1):
        Ul = U[k].reshape(-1, U[k].shape[2])
        np.testing.assert_allclose(Ul.T @ Ul, np.eye(Ul.shape[1]), atol=1e-12)
    for k in range(1, d):
        Vr = V[k].reshape(V[k].shape[0], -1)
        np.testing.assert_allclose(Vr @ Vr.T, np.eye(Vr.shape[0]), atol=1e-12)
    # ranks equal the exact ranks of the unfoldings of the full tensor (generic input)
    true = [1] + [int(np.linalg.matrix_rank(F.reshape(int(np.prod(n[:k])), -1))) for k in range(1, d)] + [1]
    assert r == true == O.orth_ranks(n, ranks)


def test_qr_pos_is_a_sign_normalised_qr():
    rng = np.random.default_rng(22)
    M = rng.normal(size=(12, 5))
    Q, R = O.qr_pos(M)
    np.testing.assert_allclose(Q @ R, M, rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(Q.T @ Q, np.eye(5), atol=1e-13)
    assert np.all(np.diag(R) >= 0) and np.allclose(np.tril(R, -1), 0)
    # uniqueness of the positive-diagonal QR: R is the Cholesky factor of M^T M
    np.testing.assert_allclose(R, np.linalg.cholesky(M.T @ M).T, rtol=1e-10, atol=1e-12)


def test_orth_ranks_config5():
    assert O.orth_ranks([16] * 20, S.tt_ranks(20, 32)) == [1, 16] + [32] * 17 + [16, 1]


# ---------------------------------------------------------------------------------------
# Projection / project_sum
# ---------------------------------------------------------------------------------------

def _proj_full(U, V, Z):
    return O.full(O.tangent_to_tt(U, V, O.project(U, V, Z)))


def test_projection_matches_explicit_projector_config1():
    cfg = S.config1()
    X = single(cfg.X)
    U, V, r = O.orthogonalize(X)
    P = O.explicit_projector(X)
    assert np.isclose(np.trace(P), O.manifold_dim([3] * 4, r), atol=1e-8)
    np.testing.assert_allclose(P, P.T, atol=1e-12)
    np.testing.assert_allclose(P @ P, P, atol=1e-10)
    for b in range(8):
        Z = single(cfg.B, b)
        np.testing.assert_allclose(_proj_full(U, V, Z).ravel(), P @ O.full(Z).ravel(),
                                   rtol=1e-10, atol=1e-10)


def test_projection_invariants():
    cfg = S.config1()
    X = single(cfg.X)
    U, V, r = O.orthogonalize(X)
    Z, W = single(cfg.B, 0), single(cfg.B, 1)
    # P_X X = X
    np.testing.assert_allclose(_proj_full(U, V, X), O.full(X), rtol=1e-10, atol=1e-12)
    # P(P(Z)) = P(Z), via the rank-2r TT of the tangent vector
    T = O.tangent_to_tt(U, V, O.project(U, V, Z))
    assert all(a <= 2 * b for a, b in zip(O.tt_ranks_of(T), r))
    np.testing.assert_allclose(_proj_full(U, V, T), O.full(T), rtol=1e-10, atol=1e-12)
    # symmetry <P Z, W> = <Z, P W>
    assert np.isclose(np.sum(_proj_full(U, V, Z) * O.full(W)),
                      np.sum(O.full(Z) * _proj_full(U, V, W)), rtol=1e-10)
    # gauge conditions
    dU = O.project(U, V, Z)
    for k in range(3):
        Ul = U[k].reshape(-1, U[k].shape[2])
        assert np.abs(Ul.T @ dU[k].reshape(Ul.shape[0], -1)).max() < 1e-12
    # the orthogonal terms make ||P Z||^2 the sum of the coordinate norms
    assert np.isclose(np.sum(_proj_full(U, V, Z) ** 2), sum(np.sum(x * x) for x in dU), rtol=1e-10)


def test_project_sum_linearity():
    cfg = S.config1()
    X = single(cfg.X)
    U, V, _ = O.orthogonalize(X)
    Zs = [single(cfg.B, b) for b in range(8)]
    S_ = O.project_sum(U, V, Zs, cfg.c)
    acc = O.tt_scale(Zs[0], cfg.c[0])
    for Z, c in zip(Zs[1:], cfg.c[1:]):
        acc = O.tt_add(acc, O.tt_scale(Z, c))
    np.testing.assert_allclose(O.full(O.tangent_to_tt(U, V, S_)), _proj_full(U, V, acc),
                               rtol=1e-10, atol=1e-10)


def test_project_sum_vjp_finite_differences():
    cfg = S.config1()
    X = single(cfg.X)
    U, V, _ = O.orthogonalize(X)
    Zs = [single(cfg.B, b) for b in range(3)]
    c = cfg.c[:3]
    rng = np.random.default_rng(23)
    S0 = O.project_sum(U, V, Zs, c)
    dUbar = [rng.normal(size=s.shape) for s in S0]
    dZ, dc = O.project_sum_vjp(U, V, Zs, c, dUbar)
    phi = lambda Zs_, c_: sum(float(np.sum(a * b)) for a, b in zip(dUbar, O.project_sum(U, V, Zs_, c_)))
    h = 1e-6
    for i in range(3):
        e = np.zeros(3); e[i] = h
        assert np.isclose((phi(Zs, c + e) - phi(Zs, c - e)) / (2 * h), dc[i], rtol=1e-7, atol=1e-9)
        for k in range(4):
            D = rng.normal(size=Zs[i][k].shape)
            Zp = [list(z) for z in Zs]; Zm = [list(z) for z in Zs]
            Zp[i][k] = Zs[i][k] + h * D; Zm[i][k] = Zs[i][k] - h * D
            assert np.isclose((phi(Zp, c) - phi(Zm, c)) / (2 * h), np.sum(dZ[i][k] * D),
                              rtol=1e-7, atol=1e-9)
    # ||S||^2 special case: dUbar = 2 dU gives dc_i = 2 <S, Z_i>
    _, dc2 = O.project_sum_vjp(U, V, Zs, c, [2 * s for s in S0])
    Sf = O.full(O.tangent_to_tt(U, V, S0))
    np.testing.assert_allclose(dc2, [2 * np.sum(Sf * O.full(Z)) for Z in Zs], rtol=1e-9)


def test_riemannian_grad_completion():
    cfg = S.config1()
    X = single(cfg.X)
    U, V, _ = O.orthogonalize(X)
    y = O.gather(single(cfg.A, 0), cfg.idx) + cfg.noise
    L, dU = O.riemannian_grad_completion(U, V, cfg.idx, y)
    assert np.isclose(L, O.completion_loss(X, cfg.idx, y), rtol=1e-11)
    # equals the explicit projector applied to the dense Euclidean gradient
    res = O.full(X)[tuple(cfg.idx)] - y
    Gd = np.zeros(O.full(X).shape)
    np.add.at(Gd, tuple(cfg.idx), res)
    P = O.explicit_projector(X)
    np.testing.assert_allclose(O.full(O.tangent_to_tt(U, V, dU)).ravel(), P @ Gd.ravel(),
                               rtol=1e-9, atol=1e-9)
    # directional derivative along a tangent vector xi = P_X(B_1)
    xi = O.tangent_to_tt(U, V, O.project(U, V, single(cfg.B, 1)))
    h = 1e-6
    fd = (O.completion_loss(O.tt_add(X, O.tt_scale(xi, h)), cfg.idx, y)
          - O.completion_loss(O.tt_add(X, O.tt_scale(xi, -h)), cfg.idx, y)) / (2 * h)
    inner = float(np.sum(O.full(O.tangent_to_tt(U, V, dU)) * O.full(xi)))
    assert np.isclose(fd, inner, rtol=1e-7)


# ---------------------------------------------------------------------------------------
# Tangent-space Gram matrices, projected matvec, linearised Hessian, rounding
# ---------------------------------------------------------------------------------------

def test_tangent_gram_is_the_full_tensor_inner_product():
    # brute force: the tangent vectors as full tensors (their rank-2r TTs), inner products of
    # the dense arrays, and the TT inner product of the same rank-2r TTs
    cfg = S.config1()
    X = single(cfg.X)
    U, V, _ = O.orthogonalize(X)
    dAs = O.project_batch(U, V, [single(cfg.A, b) for b in range(5)], cfg.c[:5])
    dBs = O.project_batch(U, V, [single(cfg.B, b) for b in range(4)])
    G = O.tangent_gram(dAs, dBs)
    FA = [O.full(O.tangent_to_tt(U, V, d)).ravel() for d in dAs]
    FB = [O.full(O.tangent_to_tt(U, V, d)).ravel() for d in dBs]
    np.testing.assert_allclose(G, np.array([[a @ b for b in FB] for a in FA]), rtol=1e-10, atol=1e-10)
    assert np.isclose(G[1, 2], O.dot(O.tangent_to_tt(U, V, dAs[1]), O.tangent_to_tt(U, V, dBs[2])), rtol=1e-10)
    # without the gauge the coordinate sum is not the inner product (the pin can fail)
    raw = O.tangent_coords(U, V, single(cfg.A, 0))
    FR = O.full(O.tangent_to_tt(U, V, raw)).ravel()
    assert not np.isclose(O.tangent_gram([raw], [raw])[0, 0], FR @ FR, rtol=1e-3)


def test_project_batch_scales_and_sums_to_project_sum():
    cfg = S.config1()
    X = single(cfg.X)
    U, V, _ = O.orthogonalize(X)
    Zs = [single(cfg.B, b) for b in range(8)]
    P = O.project_batch(U, V, Zs, cfg.c)
    tot = [sum(p[k] for p in P) for k in range(4)]
    for a, b in zip(tot, O.project_sum(U, V, Zs, cfg.c)):
        np.testing.assert_allclose(a, b, rtol=1e-10, atol=1e-12)
    # each coordinate set is the explicit projector applied to c_j Z_j
    Pm = O.explicit_projector(X)
    np.testing.assert_allclose(O.full(O.tangent_to_tt(U, V, P[3])).ravel(),
                               cfg.c[3] * (Pm @ O.full(Zs[3]).ravel()), rtol=1e-9, atol=1e-10)


def test_project_matvec_is_projected_dense_product():
    rng = np.random.default_rng(41)
    m, n = [2, 3, 2], [3, 2, 2]
    A = single(S.random_ttm(rng, 1, m, n, [1, 2, 3, 1]))
    cs = [rand_tt(rng, n, [1, 2, 2, 1]) for _ in range(3)]
    X = rand_tt(rng, m, [1, 2, 2, 1])
    U, V, _ = O.orthogonalize(X)
    Pm = O.explicit_projector(X)
    M = O.full_matrix(A)
    for c, dU in zip(cs, O.project_matvec(U, V, A, cs)):
        np.testing.assert_allclose(O.full(O.tangent_to_tt(U, V, dU)).ravel(), Pm @ (M @ O.full(c).ravel()),
                                   rtol=1e-9, atol=1e-10)


def test_tangent_gather_is_the_full_tensor_entry():
    cfg = S.config1()
    X = single(cfg.X)
    U, V, _ = O.orthogonalize(X)
    dZ = O.project(U, V, single(cfg.B, 2))
    F = O.full(O.tangent_to_tt(U, V, dZ))
    np.testing.assert_allclose(O.tangent_gather(U, V, dZ, cfg.idx), F[tuple(cfg.idx)], rtol=1e-10, atol=1e-12)
    # d = 1: the tangent vector is dZ itself
    x1 = rand_tt(np.random.default_rng(5), [6], [1, 1])
    U1, V1, _ = O.orthogonalize(x1)
    z = [np.arange(6.0).reshape(1, 6, 1)]
    np.testing.assert_allclose(O.tangent_gather(U1, V1, z, np.array([[0, 3, 5]])), [0.0, 3.0, 5.0])


def test_completion_hvp_is_projected_sampling_operator():
    # dense: P diag(counts) P applied to the dense tangent vector; symmetric; and the second
    # derivative of the (quadratic) loss along xi equals sum_t xi(i_t)^2
    cfg = S.config1()
    X = single(cfg.X)
    U, V, _ = O.orthogonalize(X)
    xi = O.project(U, V, single(cfg.B, 4))
    eta = O.project(U, V, single(cfg.B, 5))
    H = O.completion_hvp(U, V, cfg.idx, xi)
    Pm = O.explicit_projector(X)
    counts = np.zeros(O.full(X).shape)
    np.add.at(counts, tuple(cfg.idx), 1.0)
    xf = O.full(O.tangent_to_tt(U, V, xi)).ravel()
    np.testing.assert_allclose(O.full(O.tangent_to_tt(U, V, H)).ravel(), Pm @ (counts.ravel() * (Pm @ xf)),
                               rtol=1e-9, atol=1e-9)
    He = O.completion_hvp(U, V, cfg.idx, eta)
    assert np.isclose(O.tangent_gram([eta], [H])[0, 0], O.tangent_gram([He], [xi])[0, 0], rtol=1e-10)
    y = O.gather(single(cfg.A, 0), cfg.idx)
    T = O.tangent_to_tt(U, V, xi)
    h = 1e-4
    f = lambda t: O.completion_loss(O.tt_add(X, O.tt_scale(T, t)), cfg.idx, y)
    fd2 = (f(h) - 2 * f(0.0) + f(-h)) / h ** 2
    assert np.isclose(fd2, O.tangent_gram([xi], [H])[0, 0], rtol=1e-5)
    assert np.isclose(fd2, np.sum(O.tangent_gather(U, V, xi, cfg.idx) ** 2), rtol=1e-5)


def test_riemannian_scatter_matches_gradient():
    cfg = S.config1()
    X = single(cfg.X)
    U, V, _ = O.orthogonalize(X)
    y = O.gather(single(cfg.A, 0), cfg.idx) + cfg.noise
    _, dU = O.riemannian_grad_completion(U, V, cfg.idx, y)
    res = O.gather(U, cfg.idx) - y
    for a, b in zip(O.riemannian_scatter(U, V, cfg.idx, res), dU):
        np.testing.assert_allclose(a, b, rtol=1e-12, atol=1e-12)


def test_round_d2_is_truncated_matrix_svd():
    # Eckart-Young: for d = 2 the rounding is the best rank-r approximation of the matrix
    rng = np.random.default_rng(42)
    X = rand_tt(rng, [7, 6], [1, 6, 1])
    Y, disc = O.round_tt(X, 3)
    Mx = O.full(X)
    u, s, vt = np.linalg.svd(Mx)
    np.testing.assert_allclose(O.full(Y), (u[:, :3] * s[:3]) @ vt[:3], rtol=1e-10, atol=1e-10)
    assert np.isclose(disc[0], np.sum(s[3:] ** 2), rtol=1e-10)


def test_round_exact_recompression_and_error_identity():
    rng = np.random.default_rng(43)
    n = [3, 4, 2, 3]
    X = rand_tt(rng, n, [1, 2, 3, 2, 1])
    XX = O.tt_add(X, X)                       # rank 2r, true rank r
    Y, disc = O.round_tt(XX, 3)
    np.testing.assert_allclose(O.full(Y), 2 * O.full(X), rtol=1e-10, atol=1e-10)
    assert O.tt_ranks_of(Y) == O.round_ranks(n, O.tt_ranks_of(XX), 3)
    assert max(disc) < 1e-20 * O.dot(XX, XX) + 1e-24
    # truncation below the true rank: the squared error is the sum of the dropped sigma^2
    Z = rand_tt(rng, n, [1, 3, 5, 3, 1])
    Y2, disc2 = O.round_tt(Z, 2)
    err2 = np.sum((O.full(Z) - O.full(Y2)) ** 2)
    assert np.isclose(err2, sum(disc2), rtol=1e-9)
    # result cores 1..d-1 are left-orthogonal and signs follow the convention
    for k in range(3):
        Ul = Y2[k].reshape(-1, Y2[k].shape[2])
        np.testing.assert_allclose(Ul.T @ Ul, np.eye(Ul.shape[1]), atol=1e-12)
        piv = np.argmax(np.abs(Ul), axis=0)
        assert (Ul[piv, np.arange(Ul.shape[1])] > 0).all()
    assert O.tt_ranks_of(Y2) == O.round_ranks(n, O.tt_ranks_of(Z), 2) == [1, 2, 2, 2, 1]
