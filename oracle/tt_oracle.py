"""FP64 NumPy oracle (test infrastructure; never imported by the library).

Notation follows the paper (Section 1): a TT tensor A has cores G^k of shape
(r_{k-1}, n_k, r_k) with r_0 = r_d = 1, and

    A[i_1, ..., i_d] = G^1[:, i_1, :] G^2[:, i_2, :] ... G^d[:, i_d, :].

A TT object is a Python list of d float64 arrays; a TT-matrix core has shape
(r_{k-1}, m_k, n_k, r_k) (Section 3 and Section 4: TT-matrices of size 10^10 x 10^10).
Indices are 0-based. Every routine works on one object at a time; batches are plain Python
loops over objects, the "batch processing" of Section 3.1 stated without any fusion.

Readings of points the paper leaves open (each also listed in the design notes):
  * merged rank index of a Kronecker core is alpha * r_b + beta (A's rank major);
  * the tangent space at X is parametrised by left-orthogonal cores U_k (k < d) and
    right-orthogonal cores V_k (k > 1) obtained by three Householder sweeps (right-to-left,
    left-to-right, right-to-left), each QR sign-normalised so that diag(R) >= 0;
  * tangent coordinates dU_k satisfy the gauge U_k^L^T dU_k^L = 0 for k < d (Steinlechner
    2016, cited in Section 3.2 for the Riemannian operations).
"""
from __future__ import annotations

import itertools

import numpy as np

__all__ = [
    "tt_ranks_of", "full", "full_brute", "full_matrix", "dot", "gram", "norm",
    "gather", "gather_vjp", "completion_loss", "completion_loss_grad",
    "left_partials", "right_partials", "gram_vjp",
    "matvec", "matvec_vjp",
    "qr_pos", "left_orth_sweep", "right_orth_sweep", "orth_ranks", "orthogonalize",
    "tangent_coords", "gauge_project", "project", "project_sum", "tangent_to_tt",
    "project_sum_vjp", "riemannian_grad_completion", "tangent_basis_jacobian",
    "explicit_projector", "manifold_dim", "tt_add", "tt_scale",
    "project_batch", "tangent_gram", "project_matvec", "tangent_gather",
    "riemannian_scatter", "completion_hvp", "svd_sign", "round_ranks", "round_tt",
]


def _as_list(cores):
    return [np.asarray(c, dtype=np.float64) for c in cores]


def tt_ranks_of(cores) -> list[int]:
    return [int(cores[0].shape[0])] + [int(c.shape[-1]) for c in cores]


# ---------------------------------------------------------------------------------------
# The TT format (Section 1, unnumbered equation for A_{i_1...i_d})
# ---------------------------------------------------------------------------------------

def full(cores) -> np.ndarray:
    """Dense n_1 x ... x n_d tensor: contract the rank indices core by core."""
    cores = _as_list(cores)
    res = cores[0].reshape(cores[0].shape[1], cores[0].shape[2])  # (n_1, r_1)
    for G in cores[1:]:
        res = np.tensordot(res, G, axes=([res.ndim - 1], [0]))
    return res.reshape(res.shape[:-1])


def full_brute(cores) -> np.ndarray:
    """The same tensor from the written-out nested sum over alpha_1..alpha_{d-1}.

    Pure Python loops over every element and every rank index; only for tiny shapes."""
    cores = _as_list(cores)
    d = len(cores)
    n = [c.shape[1] for c in cores]
    r = tt_ranks_of(cores)
    out = np.zeros(n)
    for idx in itertools.product(*[range(v) for v in n]):
        s = 0.0
        for alphas in itertools.product(*[range(r[k]) for k in range(1, d)]):
            a = (0,) + alphas + (0,)
            p = 1.0
            for k in range(d):
                p *= cores[k][a[k], idx[k], a[k + 1]]
            s += p
        out[idx] = s
    return out


def full_matrix(cores) -> np.ndarray:
    """Dense (prod m) x (prod n) matrix of a TT-matrix with cores (r, m_k, n_k, r')."""
    cores = _as_list(cores)
    d = len(cores)
    res = cores[0].reshape(cores[0].shape[1:])  # (m1, n1, r1)
    for G in cores[1:]:
        res = np.tensordot(res, G, axes=([res.ndim - 1], [0]))
    res = res.reshape(res.shape[:-1])  # (m1, n1, m2, n2, ..., md, nd)
    perm = [2 * k for k in range(d)] + [2 * k + 1 for k in range(d)]
    res = res.transpose(perm)
    M = int(np.prod([c.shape[1] for c in cores]))
    N = int(np.prod([c.shape[2] for c in cores]))
    return res.reshape(M, N)


def tt_add(A, B):
    """TT of full(A) + full(B): block-diagonal cores (ranks add)."""
    A, B = _as_list(A), _as_list(B)
    d = len(A)
    if d == 1:
        return [A[0] + B[0]]
    out = []
    for k in range(d):
        a, b = A[k], B[k]
        ra0, n, ra1 = a.shape
        rb0, _, rb1 = b.shape
        if k == 0:
            out.append(np.concatenate([a, b], axis=2))
        elif k == d - 1:
            out.append(np.concatenate([a, b], axis=0))
        else:
            c = np.zeros((ra0 + rb0, n, ra1 + rb1))
            c[:ra0, :, :ra1] = a
            c[ra0:, :, ra1:] = b
            out.append(c)
    return out


def tt_scale(A, s):
    A = _as_list(A)
    return [A[0] * s] + [c.copy() for c in A[1:]]


# ---------------------------------------------------------------------------------------
# Inner products, Gram matrices, norms (Section 4 'norm' and 'gram'; Section 3.1 batches)
# ---------------------------------------------------------------------------------------

def left_partials(A, B):
    """M_0 = [1]; M_k = sum_i A_k[:, i, :]^T M_{k-1} B_k[:, i, :]  (r^A_k x r^B_k).

    Returns [M_0, ..., M_d]; M_d is the 1x1 inner product <A, B>."""
    A, B = _as_list(A), _as_list(B)
    M = [np.ones((1, 1))]
    for a, b in zip(A, B):
        M.append(np.einsum("aib,ac,cid->bd", a, M[-1], b, optimize=True))
    return M


def right_partials(A, B):
    """R_{d+1} = [1]; R_k = sum_i A_k[:, i, :] R_{k+1} B_k[:, i, :]^T  (r^A_{k-1} x r^B_{k-1}).

    Returns a list indexed 1..d+1 (entry 0 unused, None)."""
    A, B = _as_list(A), _as_list(B)
    d = len(A)
    R = [None] * (d + 2)
    R[d + 1] = np.ones((1, 1))
    for k in range(d, 0, -1):
        R[k] = np.einsum("aib,bd,cid->ac", A[k - 1], R[k + 1], B[k - 1], optimize=True)
    return R


def dot(A, B) -> float:
    """<A, B> = sum over all elements of full(A) * full(B), by the left transfer sweep."""
    return float(left_partials(A, B)[-1][0, 0])


def gram(As, Bs) -> np.ndarray:
    """G[a, b] = <A_a, B_b> for every pair (batch x batch broadcasting of Section 3.1)."""
    G = np.zeros((len(As), len(Bs)))
    for a, A in enumerate(As):
        for b, B in enumerate(Bs):
            G[a, b] = dot(A, B)
    return G


def norm(A) -> float:
    """Frobenius norm sqrt(<A, A>) (Table 1 'norm')."""
    return float(np.sqrt(dot(A, A)))


def gram_vjp(As, Bs, Gbar):
    """Cotangents of all cores for the scalar sum_ab Gbar[a,b] <A_a, B_b>.

    d<A,B>/dA_k[:, i, :] = M_{k-1} B_k[:, i, :] R_{k+1}^T and
    d<A,B>/dB_k[:, i, :] = M_{k-1}^T A_k[:, i, :] R_{k+1}, with M, R the left/right
    partials of the pair. Returns (dAs, dBs) as lists of core lists."""
    dAs = [[np.zeros_like(np.asarray(c, float)) for c in A] for A in As]
    dBs = [[np.zeros_like(np.asarray(c, float)) for c in B] for B in Bs]
    for a, A in enumerate(As):
        for b, B in enumerate(Bs):
            g = float(Gbar[a, b])
            if g == 0.0:
                continue
            M = left_partials(A, B)
            R = right_partials(A, B)
            for k in range(len(A)):
                dAs[a][k] += g * np.einsum("ac,cid,bd->aib", M[k], np.asarray(B[k], float), R[k + 2], optimize=True)
                dBs[b][k] += g * np.einsum("ac,aib,bd->cid", M[k], np.asarray(A[k], float), R[k + 2], optimize=True)
    return dAs, dBs


# ---------------------------------------------------------------------------------------
# Element gather and the completion loss (Section 1: completion by minimising the residual
# between the tensor and its known elements)
# ---------------------------------------------------------------------------------------

def _prefixes(cores, idx):
    """l_0 = [1]; l_k = l_{k-1} G^k[:, i_k, :] for every tuple (rows of a (N, r_k) array)."""
    N = idx.shape[1]
    ls = [np.ones((N, 1))]
    for k, G in enumerate(cores):
        S = G[:, idx[k], :].transpose(1, 0, 2)  # (N, r_{k-1}, r_k)
        ls.append(np.einsum("ta,tab->tb", ls[-1], S))
    return ls


def _suffixes(cores, idx):
    """rho_{d+1} = [1]; rho_k = G^k[:, i_k, :] rho_{k+1} (columns of a (N, r_{k-1}) array);
    returned list indexed 1..d+1 (entry 0 unused)."""
    d = len(cores)
    N = idx.shape[1]
    rs = [None] * (d + 2)
    rs[d + 1] = np.ones((N, 1))
    for k in range(d, 0, -1):
        S = cores[k - 1][:, idx[k - 1], :].transpose(1, 0, 2)
        rs[k] = np.einsum("tab,tb->ta", S, rs[k + 1])
    return rs


def _scatter_outer(w, left, right, ik, shape):
    """g[:, i, :] = sum over the tuples t with ik[t] = i of w_t left_t (outer) right_t."""
    g = np.zeros(shape)
    for i in range(shape[1]):
        sel = ik == i
        g[:, i, :] = (w[sel][:, None] * left[sel]).T @ right[sel]
    return g


def gather(cores, idx) -> np.ndarray:
    """X(i_t) for index tuples idx of shape (d, N)."""
    cores = _as_list(cores)
    idx = np.asarray(idx)
    return _prefixes(cores, idx)[-1][:, 0]


def gather_vjp(cores, idx, w):
    """Core cotangents of sum_t w_t X(i_t):  dG^k[:, i, :] = sum_{t: i_{t,k} = i}
    w_t l_{t,k-1} (outer) rho_{t,k+1}."""
    cores = _as_list(cores)
    idx = np.asarray(idx)
    w = np.asarray(w, dtype=np.float64)
    ls = _prefixes(cores, idx)
    rs = _suffixes(cores, idx)
    return [_scatter_outer(w, ls[k], rs[k + 2], idx[k], G.shape) for k, G in enumerate(cores)]


def completion_loss(cores, idx, y) -> float:
    """L = 1/2 sum_t (X(i_t) - y_t)^2 (a sum, not a mean)."""
    res = gather(cores, idx) - np.asarray(y, dtype=np.float64)
    return float(0.5 * np.sum(res * res))


def completion_loss_grad(cores, idx, y):
    """(L, dL/dG^k for every k): the gather adjoint with weights w_t = X(i_t) - y_t."""
    res = gather(cores, idx) - np.asarray(y, dtype=np.float64)
    return float(0.5 * np.sum(res * res)), gather_vjp(cores, idx, res)


# ---------------------------------------------------------------------------------------
# TT-matrix x TT-vector (Section 3 'matmul(tt_matrix, x)', Section 4 'matvec')
# ---------------------------------------------------------------------------------------

def matvec(Acores, xcores):
    """C^k[(a*r_x + b), i, (a'*r_x + b')] = sum_j A^k[a, i, j, a'] x^k[b, j, b']."""
    out = []
    for A, x in zip(_as_list(Acores), _as_list(xcores)):
        ra0, m, n, ra1 = A.shape
        rb0, _, rb1 = x.shape
        C = np.einsum("aijc,bjd->abicd", A, x)
        out.append(C.reshape(ra0 * rb0, m, ra1 * rb1))
    return out


def matvec_vjp(Acores, xcores, dC):
    """Cotangents (dA, dx) of sum_k <dC^k, C^k> with C = matvec(A, x)."""
    dA, dx = [], []
    for A, x, g in zip(_as_list(Acores), _as_list(xcores), _as_list(dC)):
        ra0, m, n, ra1 = A.shape
        rb0, _, rb1 = x.shape
        g5 = g.reshape(ra0, rb0, m, ra1, rb1)
        dA.append(np.einsum("abicd,bjd->aijc", g5, x))
        dx.append(np.einsum("abicd,aijc->bjd", g5, A))
    return dA, dx


# ---------------------------------------------------------------------------------------
# Orthogonalisation (needed by the tangent-space projection of Section 3.2)
# ---------------------------------------------------------------------------------------

def qr_pos(M):
    """Reduced Householder QR (LAPACK via numpy) with the signs fixed so diag(R) >= 0."""
    Q, R = np.linalg.qr(M, mode="reduced")
    s = np.where(np.diag(R) < 0.0, -1.0, 1.0)
    return Q * s[None, :], s[:, None] * R


def left_orth_sweep(cores):
    """Left-to-right: core_k <- Q of its (r_{k-1} n_k) x r_k unfolding, R pushed into
    core_{k+1}; the new rank is min(r_{k-1} n_k, r_k)."""
    cores = [c.copy() for c in _as_list(cores)]
    for k in range(len(cores) - 1):
        r0, n, r1 = cores[k].shape
        Q, R = qr_pos(cores[k].reshape(r0 * n, r1))
        cores[k] = Q.reshape(r0, n, Q.shape[1])
        cores[k + 1] = np.tensordot(R, cores[k + 1], axes=([1], [0]))
    return cores


def right_orth_sweep(cores):
    """Right-to-left: core_k <- Q^T of the QR of its transposed r_{k-1} x (n_k r_k)
    unfolding (an LQ step), R^T pushed into core_{k-1}."""
    cores = [c.copy() for c in _as_list(cores)]
    for k in range(len(cores) - 1, 0, -1):
        r0, n, r1 = cores[k].shape
        Q, R = qr_pos(cores[k].reshape(r0, n * r1).T)
        cores[k] = Q.T.reshape(Q.shape[1], n, r1)
        cores[k - 1] = np.tensordot(cores[k - 1], R.T, axes=([2], [0]))
    return cores


def orth_ranks(n, ranks) -> list[int]:
    """Integer rank bookkeeping of the three sweeps: right-to-left reduction
    r'_{k-1} = min(r_{k-1}, n_k r'_k), then left-to-right r''_k = min(r''_{k-1} n_k, r'_k)."""
    d = len(n)
    r1 = list(ranks)
    for k in range(d - 1, 0, -1):
        r1[k] = min(r1[k], n[k] * r1[k + 1])
    r2 = list(r1)
    for k in range(1, d):
        r2[k] = min(r2[k - 1] * n[k - 1], r1[k])
    return [int(v) for v in r2]


def orthogonalize(cores):
    """(U, V, ranks): U_1..U_{d-1} left-orthogonal with U_d carrying X, V_2..V_d
    right-orthogonal with V_1 carrying X, both representing full(X) with the same ranks.

    Sweeps: right-to-left on X (reduces the ranks from the right), left-to-right on the
    result (gives U), right-to-left on U (gives V)."""
    W = right_orth_sweep(cores)
    U = left_orth_sweep(W)
    V = right_orth_sweep(U)
    ru, rv = tt_ranks_of(U), tt_ranks_of(V)
    if ru != rv:
        raise ValueError(f"orthogonal forms disagree on ranks: {ru} vs {rv}")
    return U, V, ru


# ---------------------------------------------------------------------------------------
# Riemannian projection (Section 3.2: P_B A, project_sum S = P_B(sum_i c_i A_i),
# Riemannian gradient P_X df/dX)
# ---------------------------------------------------------------------------------------

def tangent_coords(U, V, Z):
    """Zhat_k[:, i, :] = L_{k-1} Z_k[:, i, :] R_{k+1}^T, with L the left partials of (U, Z)
    and R the right partials of (V, Z): Zhat_k = (U_{<=k-1}^T (x) I (x) V_{>=k+1}) vec Z."""
    U, V, Z = _as_list(U), _as_list(V), _as_list(Z)
    d = len(Z)
    L = left_partials(U, Z)          # L[k] : r_k x s_k
    R = right_partials(V, Z)         # R[k] : r_{k-1} x s_{k-1}
    return [np.einsum("ac,cid,bd->aib", L[k], Z[k], R[k + 2], optimize=True) for k in range(d)]


def gauge_project(U, Zhat):
    """dU_k = (I - U_k^L U_k^L^T) Zhat_k^L for k < d, dU_d = Zhat_d (left unfoldings)."""
    U = _as_list(U)
    d = len(U)
    out = []
    for k in range(d):
        z = np.asarray(Zhat[k], dtype=np.float64)
        if k < d - 1:
            r0, n, r1 = U[k].shape
            Ul = U[k].reshape(r0 * n, r1)
            zl = z.reshape(r0 * n, z.shape[2])
            z = (zl - Ul @ (Ul.T @ zl)).reshape(z.shape)
        out.append(z)
    return out


def project(U, V, Z):
    """Tangent coordinates dU of P_X Z (X given by its orthogonal forms U, V)."""
    return gauge_project(U, tangent_coords(U, V, Z))


def project_sum(U, V, Zs, c):
    """Coordinates of S = P_X(sum_i c_i Z_i), computed as sum_i c_i P_X Z_i (Section 3.2's
    linearity argument): per-Z coordinates are summed, then gauge-projected."""
    acc = None
    for Z, ci in zip(Zs, c):
        zh = tangent_coords(U, V, Z)
        acc = [ci * z for z in zh] if acc is None else [a + ci * z for a, z in zip(acc, zh)]
    return gauge_project(U, acc)


def tangent_to_tt(U, V, dU):
    """The rank-2r TT of sum_k U_1..U_{k-1} dU_k V_{k+1}..V_d: cores [dU_1, U_1],
    [[V_k, 0], [dU_k, U_k]], [[V_d], [dU_d]]."""
    U, V, dU = _as_list(U), _as_list(V), _as_list(dU)
    d = len(U)
    if d == 1:
        return [dU[0].copy()]
    out = [np.concatenate([dU[0], U[0]], axis=2)]
    for k in range(1, d - 1):
        r0, n, r1 = U[k].shape
        c = np.zeros((2 * r0, n, 2 * r1))
        c[:r0, :, :r1] = V[k]
        c[r0:, :, :r1] = dU[k]
        c[r0:, :, r1:] = U[k]
        out.append(c)
    out.append(np.concatenate([V[d - 1], dU[d - 1]], axis=0))
    return out


def project_sum_vjp(U, V, Zs, c, dUbar):
    """Cotangents (dZ_i cores, dc_i) of phi = sum_k <dUbar_k, dU_k> with
    dU = project_sum(U, V, Zs, c), X held fixed.

    With W = gauge_project(U, dUbar) and T_W the rank-2r TT of (U, V, W):
    dphi/dc_i = <T_W, Z_i>, and dphi/dZ_i = c_i d<T_W, Z_i>/dZ_i, whose core-k slice is
    P_{k-1}^T V_k R_{k+1} + L_{k-1}^T W_k R_{k+1} + L_{k-1}^T U_k Q_{k+1} with L, R the
    U- and V-partials and P, Q the mixed partials of the block cores."""
    U, V = _as_list(U), _as_list(V)
    W = gauge_project(U, dUbar)
    d = len(U)
    dZs, dc = [], []
    for Z, ci in zip(Zs, c):
        Z = _as_list(Z)
        L = left_partials(U, Z)
        R = right_partials(V, Z)
        # P_k = sum_i V_k^T P_{k-1} Z_k + W_k^T L_{k-1} Z_k, P_0 = 0
        P = [np.zeros((1, 1))]
        for k in range(d):
            nxt = np.einsum("aib,ac,cid->bd", W[k], L[k], Z[k], optimize=True)
            if k > 0:
                nxt = nxt + np.einsum("aib,ac,cid->bd", V[k], P[k], Z[k], optimize=True)
            P.append(nxt)
        # Q_k = sum_i U_k Q_{k+1} Z_k^T + W_k R_{k+1} Z_k^T, Q_{d+1} = 0
        Q = [None] * (d + 2)
        Q[d + 1] = np.zeros((1, 1))
        for k in range(d, 0, -1):
            nxt = np.einsum("aib,bd,cid->ac", W[k - 1], R[k + 1], Z[k - 1], optimize=True)
            if k < d:
                nxt = nxt + np.einsum("aib,bd,cid->ac", U[k - 1], Q[k + 1], Z[k - 1], optimize=True)
            Q[k] = nxt
        dZ = []
        for k in range(d):
            g = np.einsum("ac,aib,bd->cid", L[k], W[k], R[k + 2], optimize=True)
            if k > 0:
                g = g + np.einsum("ac,aib,bd->cid", P[k], V[k], R[k + 2], optimize=True)
            if k < d - 1:
                g = g + np.einsum("ac,aib,bd->cid", L[k], U[k], Q[k + 2], optimize=True)
            dZ.append(ci * g)
        dZs.append(dZ)
        dc.append(float(P[d][0, 0]))
    return dZs, np.array(dc)


def riemannian_grad_completion(U, V, idx, y):
    """(L, dU): the loss 1/2 sum_t (X(i_t) - y_t)^2 at X = full(U) and the coordinates of
    P_X of its Euclidean gradient sum_t res_t e_{i_t} (Section 3.2, Riemannian autodiff for
    the completion loss): Zhat_k[:, i, :] = sum_{t: i_{t,k}=i} res_t lU_{t,k-1} (x) rhoV_{t,k+1},
    then the gauge projection."""
    U, V = _as_list(U), _as_list(V)
    idx = np.asarray(idx)
    res = gather(U, idx) - np.asarray(y, dtype=np.float64)
    ls = _prefixes(U, idx)
    rs = _suffixes(V, idx)
    Zhat = [_scatter_outer(res, ls[k], rs[k + 2], idx[k],
                           (U[k].shape[0], U[k].shape[1], V[k].shape[2])) for k in range(len(U))]
    return float(0.5 * np.sum(res * res)), gauge_project(U, Zhat)


# ---------------------------------------------------------------------------------------
# Tailored tangent-space operations (Section 3.2: Gram matrix of tangent vectors of one
# tangent space, projection of a matrix-by-vector product, the linearised Riemannian
# Hessian) and rounding (Section 3, t3f.round)
# ---------------------------------------------------------------------------------------

def project_batch(U, V, Zs, c=None):
    """Coordinates of c_j P_X Z_j for every object of a batch (c_j = 1 when c is None): the
    'project' operation of Table 1 applied to each object separately, without summing."""
    out = []
    for j, Z in enumerate(Zs):
        cj = 1.0 if c is None else float(c[j])
        out.append([cj * x for x in project(U, V, Z)])
    return out


def tangent_gram(dAs, dBs) -> np.ndarray:
    """G[a, b] = <xi_a, eta_b> for tangent vectors of one tangent space given by gauge
    coordinates: the terms U_1..U_{k-1} dU_k V_{k+1}..V_d of different k are mutually
    orthogonal (gauge + orthogonality of U and V), so the inner product is the sum over k of
    the coordinate inner products <dA_k, dB_k>."""
    G = np.zeros((len(dAs), len(dBs)))
    for a, dA in enumerate(dAs):
        for b, dB in enumerate(dBs):
            G[a, b] = sum(float(np.sum(np.asarray(x, float) * np.asarray(y, float))) for x, y in zip(dA, dB))
    return G


def project_matvec(U, V, Acores, cs):
    """Coordinates of P_X (A c_j) for a TT-matrix A and every TT-vector c_j of a batch: the
    projection of the (unrounded, rank r_A r_c) product matvec(A, c_j)."""
    return [project(U, V, matvec(Acores, c)) for c in cs]


def tangent_gather(U, V, dZ, idx) -> np.ndarray:
    """Entries xi(i_t) of the tangent vector xi = sum_k U_1..U_{k-1} dZ_k V_{k+1}..V_d, one
    chain per term k and tuple, summed over k (the definition, term by term)."""
    U, V, dZ = _as_list(U), _as_list(V), _as_list(dZ)
    idx = np.asarray(idx)
    d = len(U)
    N = idx.shape[1]
    out = np.zeros(N)
    for k in range(d):
        chain = [U[j] for j in range(k)] + [dZ[k]] + [V[j] for j in range(k + 1, d)]
        out += _prefixes(chain, idx)[-1][:, 0]
    return out


def riemannian_scatter(U, V, idx, w):
    """Coordinates of P_X (sum_t w_t e_{i_t}): the Euclidean scatter with U-prefixes and
    V-suffixes, then the gauge projection."""
    U, V = _as_list(U), _as_list(V)
    idx = np.asarray(idx)
    w = np.asarray(w, dtype=np.float64)
    ls = _prefixes(U, idx)
    rs = _suffixes(V, idx)
    Zhat = [_scatter_outer(w, ls[k], rs[k + 2], idx[k],
                           (U[k].shape[0], U[k].shape[1], V[k].shape[2])) for k in range(len(U))]
    return gauge_project(U, Zhat)


def completion_hvp(U, V, idx, dZ):
    """Linearised Riemannian Hessian of the completion loss f(X) = 1/2 sum_t (X(i_t) - y_t)^2
    applied to a tangent vector: P_X (grad^2 f) P_X xi, with xi given by its coordinates dZ.
    grad^2 f = sum_t e_{i_t} e_{i_t}^T (tuples counted with multiplicity, independent of X and
    y), so the result is P_X (sum_t xi(i_t) e_{i_t})."""
    return riemannian_scatter(U, V, idx, tangent_gather(U, V, dZ, idx))


def svd_sign(Uk, SVt):
    """Sign convention of the rounding's SVD factors: every left singular vector has its
    entry of largest magnitude positive (the matching row of S V^T flips with it)."""
    piv = np.argmax(np.abs(Uk), axis=0)
    s = np.where(Uk[piv, np.arange(Uk.shape[1])] < 0.0, -1.0, 1.0)
    return Uk * s[None, :], SVt * s[:, None]


def round_ranks(n, ranks, max_rank) -> list[int]:
    """Ranks of round_tt: the right-to-left reduction r'_{k-1} = min(r_{k-1}, n_k r'_k),
    then left to right min(r''_{k-1} n_k, r'_k, max_rank)."""
    d = len(n)
    r1 = list(ranks)
    for k in range(d - 1, 0, -1):
        r1[k] = min(r1[k], n[k] * r1[k + 1])
    r2 = list(r1)
    for k in range(1, d):
        r2[k] = min(r2[k - 1] * n[k - 1], r1[k], int(max_rank))
    return [int(v) for v in r2]


def round_tt(cores, max_rank):
    """TT rounding to TT-ranks <= max_rank (Section 3, t3f.round; the TT-SVD recompression of
    Oseledets 2011): a right-to-left orthogonalisation sweep, then left to right the SVD of
    each (r_{k-1} n_k) x r_k unfolding, truncated to the leading max_rank singular triplets,
    with S V^T pushed into the next core. Returns (cores, discarded), discarded[k] the sum of
    the squared singular values dropped at interface k+1; ||X - round(X)||^2 is their sum."""
    W = right_orth_sweep(cores)
    d = len(W)
    discarded = []
    for k in range(d - 1):
        r0, n, r1 = W[k].shape
        Uk, sv, Vt = np.linalg.svd(W[k].reshape(r0 * n, r1), full_matrices=False)
        keep = min(int(max_rank), len(sv))
        Uk, SVt = svd_sign(Uk[:, :keep], sv[:keep, None] * Vt[:keep])
        discarded.append(float(np.sum(sv[keep:] ** 2)))
        W[k] = Uk.reshape(r0, n, keep)
        W[k + 1] = np.tensordot(SVt, W[k + 1], axes=([1], [0]))
    return W, discarded


# ---------------------------------------------------------------------------------------
# Plain definitions used to pin the sweeps (tiny sizes only)
# ---------------------------------------------------------------------------------------

def tangent_basis_jacobian(cores) -> np.ndarray:
    """Jacobian of the map (G^1, ..., G^d) -> vec full(G) at X: one column per core entry,
    the full tensor of X with that core replaced by the matching unit tensor. Its range is
    the tangent space of the fixed-rank manifold at X."""
    cores = _as_list(cores)
    cols = []
    for k, G in enumerate(cores):
        for pos in itertools.product(*[range(s) for s in G.shape]):
            E = np.zeros_like(G)
            E[pos] = 1.0
            cols.append(full(cores[:k] + [E] + cores[k + 1:]).ravel())
    return np.stack(cols, axis=1)


def explicit_projector(cores, tol: float = 1e-10) -> np.ndarray:
    """Orthogonal projector onto the tangent space: J J^+ from the SVD of the Jacobian."""
    J = tangent_basis_jacobian(cores)
    Uj, s, _ = np.linalg.svd(J, full_matrices=False)
    rank = int(np.sum(s > tol * s[0]))
    Q = Uj[:, :rank]
    return Q @ Q.T


def manifold_dim(n, ranks) -> int:
    """sum_k r_{k-1} n_k r_k - sum_{k=1}^{d-1} r_k^2 (dimension of the TT manifold)."""
    d = len(n)
    return int(sum(ranks[k] * n[k] * ranks[k + 1] for k in range(d))
               - sum(ranks[k] ** 2 for k in range(1, d)))
