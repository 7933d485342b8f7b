"""Tensor-core Gram adjoint (TF32 / BF16 operands, FP32 accumulation in tensor memory) against
the FP64 oracle's cotangents: uniform batches of every padded tile shape, exchanged sides
(A of the larger rank), ragged batch tails, d = 1, BF16-stored cores, the grouped ragged
collections and sampled objects of the uneven 8 x 64 batch. Every object's gradient is scored
on its own (normwise over its cores) at the math's stated tolerance."""
import numpy as np
import pytest

import oracle as O
import synth as S
from tests._util import TOL, objects, rel_err_cores, round32, round_bf16

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def dev_tt(t3f, cores, dtype=torch.float32):
    return t3f.TT.from_cores([torch.tensor(np.asarray(c)) for c in cores], dtype=dtype, device="cuda")


def host_objects(tt):
    return objects([c.detach().double().cpu().numpy() for c in tt.cores()])


# (seed, bA, bB, modes, A ranks, B ranks): padded tile shapes 16 x 16, 32 x 64, exchanged sides
# (A's padded rank above B's), rank-changing interiors, d = 1 and d = 2 at rank 64
UNIFORM = [
    (1100, 11, 9, [3, 4, 2, 3, 5], [1, 3, 4, 2, 3, 1], [1, 2, 3, 5, 2, 1]),
    (1101, 9, 5, [2, 3, 4, 2], [1, 20, 17, 24, 1], [1, 40, 33, 48, 1]),
    (1102, 5, 17, [3, 2, 3], [1, 50, 37, 1], [1, 12, 9, 1]),
    (1103, 6, 4, [7], [1, 1], [1, 1]),
    (1104, 3, 4, [4, 3], [1, 64, 1], [1, 61, 1]),
    (1105, 20, 13, [4, 4, 4, 4, 4, 4], [1, 10, 10, 10, 10, 10, 1], [1, 10, 10, 10, 10, 10, 1]),
]


@pytest.mark.parametrize("math_", ["tf32", "bf16"])
@pytest.mark.parametrize("case", UNIFORM, ids=[str(c[0]) for c in UNIFORM])
def test_gram_backward_tensor_cores(lib, case, math_):
    seed, bA, bB, n, rA, rB = case
    rng = np.random.default_rng(seed)
    A = round32(S.random_tt(rng, bA, n, rA, 1.0 / np.sqrt(max(rA))))
    B = round32(S.random_tt(rng, bB, n, rB, 1.0 / np.sqrt(max(rB))))
    dG = rng.normal(size=(bA, bB)).astype(np.float32)
    tA, tB = dev_tt(lib, A), dev_tt(lib, B)
    ws = lib.workspace("gram_bwd_tc", tA, tB)
    dA, dB = lib.gram_backward(tA, tB, torch.tensor(dG, device="cuda"), math=math_, ws=ws)
    assert lib.device_status(ws) == 0
    oa, ob = objects(A), objects(B)
    rA_, rB_ = O.gram_vjp(oa, ob, dG.astype(np.float64))
    hA, hB = host_objects(dA), host_objects(dB)
    for a in range(bA):
        assert rel_err_cores(hA[a], rA_[a]) < TOL[math_], ("A", a)
    for b in range(bB):
        assert rel_err_cores(hB[b], rB_[b]) < TOL[math_], ("B", b)


def test_gram_backward_tensor_cores_bf16_storage_and_one_side(lib):
    # BF16-stored cores (the BF16 operands are then exact) and only dA requested
    rng = np.random.default_rng(1110)
    n = [3, 4, 3, 2]
    A = round_bf16(S.random_tt(rng, 7, n, [1, 30, 22, 28, 1], 0.2))
    B = round_bf16(S.random_tt(rng, 10, n, [1, 14, 16, 9, 1], 0.25))
    dG = rng.normal(size=(7, 10)).astype(np.float32)
    tA, tB = dev_tt(lib, A, torch.bfloat16), dev_tt(lib, B, torch.bfloat16)
    dA, dB = lib.gram_backward(tA, tB, torch.tensor(dG, device="cuda"), need_B=False, math="bf16")
    assert dB is None
    rA_, _ = O.gram_vjp(objects(A), objects(B), dG.astype(np.float64))
    hA = host_objects(dA)
    for a in range(7):
        assert rel_err_cores(hA[a], rA_[a]) < TOL["bf16"], a


def test_gram_backward_tensor_cores_config3a_sampled(lib):
    # the 100 x 100 Gram adjoint of the batched-Gram workload (d = 10, n = 10, r = 10)
    cfg = S.config3a()
    A, B = round32(cfg.A), round32(cfg.B)
    dG = np.random.default_rng(1111).normal(size=(100, 100)).astype(np.float32)
    tA, tB = dev_tt(lib, A), dev_tt(lib, B)
    for math_ in ("tf32", "bf16"):
        dA, dB = lib.gram_backward(tA, tB, torch.tensor(dG, device="cuda"), math=math_)
        hA, hB = host_objects(dA), host_objects(dB)
        oa, ob = objects(A), objects(B)
        for a in (0, 57, 99):
            rA_, _ = O.gram_vjp([oa[a]], ob, dG[a:a + 1].astype(np.float64))
            assert rel_err_cores(hA[a], rA_[0]) < TOL[math_], (math_, a)
        for b in (3, 64):
            _, rB_ = O.gram_vjp(oa, [ob[b]], dG[:, b:b + 1].astype(np.float64))
            assert rel_err_cores(hB[b], rB_[0]) < TOL[math_], (math_, b)


def test_gram_backward_tensor_cores_rejects(lib):
    rng = np.random.default_rng(1112)
    A = round32(S.random_tt(rng, 2, [3, 3], [1, 70, 1], 0.1))  # rank above 64
    tA = dev_tt(lib, A)
    with pytest.raises(lib.T3FError):
        lib.gram_backward(tA, tA, torch.ones(2, 2, device="cuda"), math="tf32",
                          ws=torch.empty(1 << 20, dtype=torch.uint8, device="cuda"))
    Ab = round_bf16(S.random_tt(rng, 2, [3, 3], [1, 5, 1], 0.1))
    tb = dev_tt(lib, Ab, torch.bfloat16)
    with pytest.raises(lib.T3FError):  # TF32 needs F32 cores
        lib.gram_backward(tb, tb, torch.ones(2, 2, device="cuda"), math="tf32")


def _group_case(seed):
    from tests.test_gpu_groups import ragged_case
    return ragged_case(seed)


def _check_groups(lib, X, objs, gstart, dout, dX, tol, sample=None, rng=None):
    view = lib.RaggedTT(dX, X.dims, X.modes, X.ranks, X.offsets)
    off = 0
    for g in range(len(gstart) - 1):
        grp = objs[gstart[g]:gstart[g + 1]]
        Sg = len(grp)
        dG = dout[off:off + Sg * Sg].reshape(Sg, Sg).astype(np.float64)
        off += Sg * Sg
        js = range(Sg) if sample is None else [int(rng.integers(0, Sg)) for _ in range(sample)]
        for j in js:
            want, _ = O.gram_vjp([grp[j]], grp, (dG[j, :] + dG[:, j])[None, :])
            got = [c.double().cpu().numpy() for c in view.object_cores(gstart[g] + j)]
            assert rel_err_cores(got, want[0]) < tol, (g, j)


@pytest.mark.parametrize("math_", ["tf32", "bf16"])
def test_gram_groups_backward_tensor_cores(lib, math_):
    objs, gstart = _group_case(1120)
    objs = [round32(o) for o in objs]
    X = lib.RaggedTT.from_objects([[np.asarray(c, np.float32) for c in o] for o in objs])
    ws = lib.gram_groups_prepare(X, gstart, backward_math=math_)
    G, _ = lib.gram_groups(X, gstart, ws, math=math_)
    dout = np.random.default_rng(1121).normal(size=G.numel()).astype(np.float32)
    dX = lib.gram_groups_backward(X, gstart, ws, torch.tensor(dout, device="cuda"), math=math_)
    assert lib.device_status(ws) == 0
    _check_groups(lib, X, objs, gstart, dout, dX, TOL[math_])


def test_gram_groups_backward_tensor_cores_varying_ranks(lib):
    # interior ranks that change from core to core, d = 1 and n_k = 1 groups
    rng = np.random.default_rng(1122)
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
    objs = [round32(o) for g in groups for o in g]
    X = lib.RaggedTT.from_objects([[np.asarray(c, np.float32) for c in o] for o in objs])
    ws = lib.gram_groups_prepare(X, gstart, backward_math="tf32")
    G, _ = lib.gram_groups(X, gstart, ws, math="tf32")
    dout = rng.normal(size=G.numel()).astype(np.float32)
    dX = lib.gram_groups_backward(X, gstart, ws, torch.tensor(dout, device="cuda"), math="tf32")
    _check_groups(lib, X, objs, gstart, dout, dX, TOL["tf32"])


@pytest.mark.parametrize("math_", ["bf16", "tf32"])
def test_gram_groups_config4_backward_tensor_cores_sampled(lib, math_):
    # the uneven batch (8 groups x 64 ragged TTs): BF16 cores for BF16, F32 cores for TF32
    cfg = S.config4()
    objs, gstart = [], [0]
    rnd = round_bf16 if math_ == "bf16" else round32
    for grp in cfg.groups:
        objs += [rnd(o) for o in grp.cores]
        gstart.append(len(objs))
    dt = torch.bfloat16 if math_ == "bf16" else torch.float32
    X = lib.RaggedTT.from_objects([[torch.tensor(np.asarray(c)) for c in o] for o in objs], dtype=dt)
    ws = lib.gram_groups_prepare(X, gstart, backward_math=math_)
    G, _ = lib.gram_groups(X, gstart, ws, math=math_)
    rng = np.random.default_rng(1123)
    dout = rng.normal(size=G.numel()).astype(np.float32)
    dX = lib.gram_groups_backward(X, gstart, ws, torch.tensor(dout, device="cuda"), math=math_)
    assert lib.device_status(ws) == 0
    _check_groups(lib, X, objs, gstart, dout, dX, TOL[math_], sample=2, rng=rng)
