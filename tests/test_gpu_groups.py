"""Grouped Gram matrices over ragged collections (uneven d, n and r per object) against the
FP64 oracle: forward, FP64 norms, adjoint, BF16 storage, the tile autotuner and CUDA-graph
replay of the prepared persistent launch."""
import numpy as np
import pytest

import oracle as O
import synth as S
from tests._util import TOL, assert_gram_blocks, rel_err, rel_err_cores, round32, round_bf16, sampled_gram_errs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def ragged_case(seed=400):
    rng = np.random.default_rng(seed)
    groups = []
    for d, n, S_, rlo, rhi in ((4, [3, 2, 4, 3], 9, 1, 12), (3, [5, 4, 2], 6, 2, 40), (5, [2, 3, 2, 2, 3], 5, 3, 64)):
        objs = []
        for _ in range(S_):
            r = int(rng.integers(rlo, rhi + 1))
            ranks = [1] + [r] * (d - 1) + [1]
            objs.append([c[0] for c in S.random_tt(rng, 1, n, ranks, 1.0 / np.sqrt(r))])
        groups.append(objs)
    gstart = [0]
    for objs in groups:
        gstart.append(gstart[-1] + len(objs))
    return [o for objs in groups for o in objs], gstart


def as_f32(objs):
    return [round32(o) for o in objs]


def sizes_of(gstart):
    return [gstart[g + 1] - gstart[g] for g in range(len(gstart) - 1)]


def oracle_groups(objs, gstart):
    out = []
    for g in range(len(gstart) - 1):
        grp = objs[gstart[g]:gstart[g + 1]]
        out.append(O.gram(grp, grp).ravel())
    return np.concatenate(out)


def test_gram_groups_forward_norms_backward(lib):
    objs, gstart = ragged_case()
    objs = as_f32(objs)
    X = lib.RaggedTT.from_objects([[np.asarray(c, np.float32) for c in o] for o in objs])
    ws = lib.gram_groups_prepare(X, gstart)
    G, nrm = lib.gram_groups(X, gstart, ws)
    ref = oracle_groups(objs, gstart)
    assert_gram_blocks(G.cpu().numpy(), ref, sizes_of(gstart), TOL["fp32"])
    assert rel_err(nrm.cpu().numpy(), [O.norm(o) for o in objs]) < TOL["fp32"]
    rng = np.random.default_rng(401)
    dout = rng.normal(size=G.numel()).astype(np.float32)
    dX = lib.gram_groups_backward(X, gstart, ws, torch.tensor(dout, device="cuda"))
    off = 0
    for g in range(len(gstart) - 1):
        grp = objs[gstart[g]:gstart[g + 1]]
        Sg = len(grp)
        dG = dout[off:off + Sg * Sg].reshape(Sg, Sg).astype(np.float64)
        off += Sg * Sg
        dA, dB = O.gram_vjp(grp, grp, dG)
        for j in range(Sg):
            o = gstart[g] + j
            got = [c.double().cpu().numpy() for c in
                   lib.RaggedTT(dX, X.dims, X.modes, X.ranks, X.offsets).object_cores(o)]
            want = [a + b for a, b in zip(dA[j], dB[j])]
            assert rel_err_cores(got, want) < TOL["fp32"], (g, j)


def test_gram_groups_varying_core_ranks(lib):
    # interior ranks that change from core to core (and d = 1, n_k = 1 groups): the kernels
    # bound each core's products by the tile's largest ranks on either side of that core
    rng = np.random.default_rng(402)
    groups = []
    for d, n, S_ in ((1, [5], 3), (2, [1, 3], 4), (4, [3, 1, 2, 4], 7), (5, [2, 3, 2, 2, 3], 6)):
        objs = []
        for _ in range(S_):
            ranks = [1] + [int(rng.integers(1, 40)) for _ in range(d - 1)] + [1]
            objs.append([c[0] for c in S.random_tt(rng, 1, n, ranks, 0.3)])
        groups.append(objs)
    gstart = [0]
    for objs in groups:
        gstart.append(gstart[-1] + len(objs))
    objs = as_f32([o for g in groups for o in g])
    X = lib.RaggedTT.from_objects([[np.asarray(c, np.float32) for c in o] for o in objs])
    ws = lib.gram_groups_prepare(X, gstart)
    G, nrm = lib.gram_groups(X, gstart, ws)
    assert_gram_blocks(G.cpu().numpy(), oracle_groups(objs, gstart), sizes_of(gstart), TOL["fp32"])
    assert rel_err(nrm.cpu().numpy(), [O.norm(o) for o in objs]) < TOL["fp32"]
    dout = rng.normal(size=G.numel()).astype(np.float32)
    dX = lib.gram_groups_backward(X, gstart, ws, torch.tensor(dout, device="cuda"))
    view = lib.RaggedTT(dX, X.dims, X.modes, X.ranks, X.offsets)
    off = 0
    for g in range(len(gstart) - 1):
        grp = objs[gstart[g]:gstart[g + 1]]
        Sg = len(grp)
        dG = dout[off:off + Sg * Sg].reshape(Sg, Sg).astype(np.float64)
        off += Sg * Sg
        dA, dB = O.gram_vjp(grp, grp, dG)
        for j in range(Sg):
            got = [c.double().cpu().numpy() for c in view.object_cores(gstart[g] + j)]
            assert rel_err_cores(got, [a + b for a, b in zip(dA[j], dB[j])]) < TOL["fp32"], (g, j)


def test_gram_groups_bf16_storage(lib):
    objs, gstart = ragged_case(402)
    objs_b = [round_bf16(o) for o in objs]
    X = lib.RaggedTT.from_objects([[torch.tensor(np.asarray(c)) for c in o] for o in objs_b], dtype=torch.bfloat16)
    ws = lib.gram_groups_prepare(X, gstart)
    G, nrm = lib.gram_groups(X, gstart, ws)
    ref = oracle_groups(objs_b, gstart)
    assert rel_err(nrm.cpu().numpy(), [O.norm(o) for o in objs_b]) < TOL["bf16"]
    # the arithmetic is FP32 on the rounded inputs: inside the FP32 tolerance
    assert_gram_blocks(G.cpu().numpy(), ref, sizes_of(gstart), TOL["fp32"])


def test_gram_groups_autotune_and_graph_replay(lib):
    objs, gstart = ragged_case(403)
    objs = as_f32(objs)
    X = lib.RaggedTT.from_objects([[np.asarray(c, np.float32) for c in o] for o in objs])
    tiles, _ = lib.autotune_gram_groups(X, gstart, candidates=(1, 2, 4, 8), reps=1)
    assert len(tiles) == 4 and all(1 <= t <= 16 for t in tiles)
    ws = lib.gram_groups_prepare(X, gstart, tiles)
    G0, n0 = lib.gram_groups(X, gstart, ws, tiles)
    dout = torch.randn(G0.numel(), device="cuda")
    d0 = lib.gram_groups_backward(X, gstart, ws, dout, tiles)
    G, nrm, dX = torch.empty_like(G0), torch.empty_like(n0), torch.empty_like(d0)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        lib.gram_groups(X, gstart, ws, tiles, out=G, norms=nrm)  # warm-up on the capture stream
        lib.gram_groups_backward(X, gstart, ws, dout, tiles, dcores=dX)
    torch.cuda.current_stream().wait_stream(s)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        lib.gram_groups(X, gstart, ws, tiles, out=G, norms=nrm)
        lib.gram_groups_backward(X, gstart, ws, dout, tiles, dcores=dX)
    G.zero_()
    dX.zero_()
    graph.replay()
    torch.cuda.synchronize()
    assert_gram_blocks(G.cpu().numpy(), G0.cpu().numpy(), sizes_of(gstart), 1e-6)
    assert rel_err(dX.cpu().numpy(), d0.cpu().numpy()) < 1e-5
    assert_gram_blocks(G.cpu().numpy(), oracle_groups(objs, gstart), sizes_of(gstart), TOL["fp32"])


def _config4_sampled_check(G, objs, gstart, rng, tol):
    # per group: both end diagonals and 10 distinct-object pairs, scored separately (the
    # off-diagonal inner products are 1e-8..1e-2 of the diagonal ones)
    off = 0
    for g in range(len(gstart) - 1):
        Sg = gstart[g + 1] - gstart[g]
        pairs = [(0, 0), (Sg - 1, Sg - 1)]
        while len(pairs) < 12:
            a, b = (int(v) for v in rng.integers(0, Sg, 2))
            if a != b:
                pairs.append((a, b))
        got = [G[off + a * Sg + b] for a, b in pairs]
        want = [O.dot(objs[gstart[g] + a], objs[gstart[g] + b]) for a, b in pairs]
        ed, eo = sampled_gram_errs(got, want, [a == b for a, b in pairs])
        assert ed < tol and eo < tol, (g, ed, eo)
        off += Sg * Sg


def test_gram_groups_config4_sampled(lib):
    cfg = S.config4()
    objs, gstart = [], [0]
    for grp in cfg.groups:
        objs += [round32(o) for o in grp.cores]
        gstart.append(len(objs))
    X = lib.RaggedTT.from_objects([[np.asarray(c, np.float32) for c in o] for o in objs])
    ws = lib.gram_groups_prepare(X, gstart)
    G, nrm = lib.gram_groups(X, gstart, ws)
    _config4_sampled_check(G.cpu().numpy(), objs, gstart, np.random.default_rng(404), TOL["fp32"])


def test_gram_groups_config4_backward_sampled(lib):
    # the full uneven batch (8 groups x 64 TTs, ranks up to 64) through the persistent adjoint;
    # one sampled object per group (the highest rank and a random one alternately) against the
    # oracle's cotangent of sum_ab dG_ab <X_a, X_b>: object a collects (dG_ab + dG_ba) times
    # the derivative of <X_a, X_b> in its first argument
    cfg = S.config4()
    objs, gstart = [], [0]
    for grp in cfg.groups:
        objs += [round32(o) for o in grp.cores]
        gstart.append(len(objs))
    X = lib.RaggedTT.from_objects([[np.asarray(c, np.float32) for c in o] for o in objs])
    ws = lib.gram_groups_prepare(X, gstart)
    G, _ = lib.gram_groups(X, gstart, ws)
    rng = np.random.default_rng(405)
    dout = rng.normal(size=G.numel()).astype(np.float32)
    dX = lib.gram_groups_backward(X, gstart, ws, torch.tensor(dout, device="cuda"))
    view = lib.RaggedTT(dX, X.dims, X.modes, X.ranks, X.offsets)
    off = 0
    for g in range(len(gstart) - 1):
        grp = objs[gstart[g]:gstart[g + 1]]
        Sg = len(grp)
        dG = dout[off:off + Sg * Sg].reshape(Sg, Sg).astype(np.float64)
        off += Sg * Sg
        ranks = [max(np.asarray(c).shape[0] for c in o) for o in grp]
        a = int(np.argmax(ranks)) if g % 2 == 0 else int(rng.integers(0, Sg))
        w = (dG[a, :] + dG[:, a])[None, :]
        dA, _ = O.gram_vjp([grp[a]], grp, w)
        got = [c.double().cpu().numpy() for c in view.object_cores(gstart[g] + a)]
        assert rel_err_cores(got, dA[0]) < TOL["fp32"], (g, a)


@pytest.mark.parametrize("math_", ["tf32", "bf16"])
def test_gram_groups_tensor_cores(lib, math_):
    # every pair on the tensor cores in (128/RA) x (128/RB) tiles (RA, RB in 16/32/64 by rank
    # bucket); one result matrix per group
    objs, gstart = ragged_case(405)
    if math_ == "tf32":
        objs, dt = as_f32(objs), torch.float32
    else:
        objs, dt = [round_bf16(o) for o in objs], torch.bfloat16
    X = lib.RaggedTT.from_objects([[torch.tensor(np.asarray(c)) for c in o] for o in objs], dtype=dt)
    ws = lib.gram_groups_prepare(X, gstart)
    G, nrm = lib.gram_groups(X, gstart, ws, math=math_)
    torch.cuda.synchronize()
    assert lib.device_status(ws) == 0
    ref = oracle_groups(objs, gstart)
    assert np.isfinite(G.cpu().numpy()).all()
    assert_gram_blocks(G.cpu().numpy(), ref, sizes_of(gstart), TOL[math_])
    assert rel_err(nrm.cpu().numpy(), [O.norm(o) for o in objs]) < TOL[math_]
    # each group matrix is symmetric up to the operand rounding
    off = 0
    Gh = G.cpu().numpy()
    for g in range(len(gstart) - 1):
        S_ = gstart[g + 1] - gstart[g]
        M = Gh[off:off + S_ * S_].reshape(S_, S_)
        assert rel_err(M, M.T) < TOL[math_]
        off += S_ * S_


def test_gram_groups_config4_bf16_sampled(lib):
    cfg = S.config4()
    objs, gstart = [], [0]
    for grp in cfg.groups:
        objs += [round_bf16(o) for o in grp.cores]
        gstart.append(len(objs))
    X = lib.RaggedTT.from_objects([[torch.tensor(np.asarray(c)) for c in o] for o in objs], dtype=torch.bfloat16)
    ws = lib.gram_groups_prepare(X, gstart)
    G, nrm = lib.gram_groups(X, gstart, ws, math="bf16")
    _config4_sampled_check(G.cpu().numpy(), objs, gstart, np.random.default_rng(406), TOL["bf16"])
    assert rel_err(nrm.cpu().numpy()[[0, 100, 511]], [O.norm(objs[i]) for i in (0, 100, 511)]) < TOL["bf16"]


def test_gram_groups_config4_bf16_backward_sampled(lib):
    # the uneven adjoint on BF16-stored cores (FP32 arithmetic): sampled objects of every group
    # against the oracle's cotangent on the same BF16-rounded cores
    cfg = S.config4()
    objs, gstart = [], [0]
    for grp in cfg.groups:
        objs += [round_bf16(o) for o in grp.cores]
        gstart.append(len(objs))
    X = lib.RaggedTT.from_objects([[torch.tensor(np.asarray(c)) for c in o] for o in objs], dtype=torch.bfloat16)
    ws = lib.gram_groups_prepare(X, gstart)
    G, _ = lib.gram_groups(X, gstart, ws)
    rng = np.random.default_rng(407)
    dout = rng.normal(size=G.numel()).astype(np.float32)
    dX = lib.gram_groups_backward(X, gstart, ws, torch.tensor(dout, device="cuda"))
    view = lib.RaggedTT(dX, X.dims, X.modes, X.ranks, X.offsets)
    off = 0
    for g in range(len(gstart) - 1):
        grp = objs[gstart[g]:gstart[g + 1]]
        Sg = len(grp)
        dG = dout[off:off + Sg * Sg].reshape(Sg, Sg).astype(np.float64)
        off += Sg * Sg
        a = int(rng.integers(0, Sg))
        dA, _ = O.gram_vjp([grp[a]], grp, (dG[a, :] + dG[:, a])[None, :])
        got = [c.double().cpu().numpy() for c in view.object_cores(gstart[g] + a)]
        assert rel_err_cores(got, dA[0]) < TOL["bf16"], (g, a)
