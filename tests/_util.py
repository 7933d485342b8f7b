"""Helpers shared by the tests: batch <-> per-object core lists, FP32 rounding of inputs,
and the error measures used for parity (normwise relative error of each output array; Gram
matrices of one collection scored per group, separately over diagonal and off-diagonal
entries)."""
import numpy as np

# Stated tolerances against the FP64 oracle (relative, normwise per output array).
TOL = {"fp32": 1e-5, "tf32": 5e-3, "bf16": 2e-2}


def objects(cores_batched):
    """[(batch, ...) per core] -> list of per-object core lists."""
    b = cores_batched[0].shape[0]
    return [[np.asarray(c[i], dtype=np.float64) for c in cores_batched] for i in range(b)]


def batched(objs):
    """list of per-object core lists -> [(batch, ...) per core]."""
    return [np.stack([o[k] for o in objs]) for k in range(len(objs[0]))]


def round32(cores):
    return [np.asarray(c, dtype=np.float32).astype(np.float64) for c in cores]


def round_bf16(cores):
    import torch
    return [torch.as_tensor(np.asarray(c)).to(torch.bfloat16).to(torch.float64).numpy() for c in cores]


def rel_err(y, y_ref) -> float:
    y = np.asarray(y, dtype=np.float64).ravel()
    y_ref = np.asarray(y_ref, dtype=np.float64).ravel()
    den = np.linalg.norm(y_ref)
    num = np.linalg.norm(y - y_ref)
    return float(num / den) if den > 0 else float(num)


def rel_err_cores(a, b) -> float:
    return rel_err(np.concatenate([np.asarray(x).ravel() for x in a]),
                   np.concatenate([np.asarray(x).ravel() for x in b]))


def gram_block_errs(G, G_ref, sizes):
    """Normwise errors of concatenated square group matrices, per group and separately over
    the diagonal (squared norms) and the off-diagonal entries (inner products of distinct
    objects). Random TT pairs are nearly orthogonal, so in a self-Gram matrix the diagonal
    dominates the norm by many orders of magnitude and one normwise error over the whole
    matrix could not see a wrong off-diagonal block. Returns [(diag_err, offdiag_err)]."""
    G = np.asarray(G, dtype=np.float64).ravel()
    G_ref = np.asarray(G_ref, dtype=np.float64).ravel()
    out, off = [], 0
    for s in sizes:
        M = G[off:off + s * s].reshape(s, s)
        R = G_ref[off:off + s * s].reshape(s, s)
        off += s * s
        mask = ~np.eye(s, dtype=bool)
        out.append((rel_err(np.diag(M), np.diag(R)), rel_err(M[mask], R[mask]) if s > 1 else 0.0))
    return out


def assert_gram_blocks(G, G_ref, sizes, tol):
    for g, (ed, eo) in enumerate(gram_block_errs(G, G_ref, sizes)):
        assert ed < tol and eo < tol, (g, ed, eo, tol)


def sampled_gram_errs(got, want, is_diag):
    """(diag_err, offdiag_err) of sampled entries of one group matrix."""
    got, want, is_diag = np.asarray(got, float), np.asarray(want, float), np.asarray(is_diag, bool)
    ed = rel_err(got[is_diag], want[is_diag]) if is_diag.any() else 0.0
    eo = rel_err(got[~is_diag], want[~is_diag]) if (~is_diag).any() else 0.0
    return ed, eo
