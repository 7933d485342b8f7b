"""torch.autograd wrappers: gradients of the completion loss, the Gram matrix and project_sum
against the FP64 oracle's analytic gradients (FP32 tolerance) and against central finite
differences of the CUDA forward along a random direction."""
import numpy as np
import pytest

import oracle as O
import synth as S
from tests._util import TOL, batched, objects, rel_err, rel_err_cores, round32

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _tt(lib, cores):
    return lib.TT.from_cores([np.asarray(c, np.float32) for c in cores], device="cuda")


def _host_cores(lib, data, like):
    t = lib.TT(data.detach(), like.n, like.ranks, like.batch, like.m)
    return [c.double().cpu().numpy() for c in t.cores()]


def _fd(f, data, direction, h):
    """Five-point central difference (truncation O(h^4)) of t -> f(data + t direction) at 0."""
    with torch.no_grad():
        v = [float(f(data + t * h * direction)) for t in (-2, -1, 1, 2)]
    return (v[0] - 8 * v[1] + 8 * v[2] - v[3]) / (12 * h)


def test_completion_loss_autograd(lib):
    from paper_1801_01928_gb300 import autograd as AG
    torch.manual_seed(500)
    rng = np.random.default_rng(500)
    n, r = [4, 3, 5, 3, 4], [1, 3, 4, 4, 2, 1]
    X = round32(S.random_tt(rng, 1, n, r, 0.6))
    idx = S.random_indices(rng, 3000, n)
    y = rng.normal(size=3000).astype(np.float32)
    Xt = _tt(lib, X)
    Xt.data.requires_grad_(True)
    idx_d, y_d = torch.tensor(idx, device="cuda"), torch.tensor(y, device="cuda")
    loss = AG.completion_loss(Xt, idx_d, y_d)
    assert loss.dtype == torch.float64 and loss.dim() == 0
    (3.0 * loss).backward()
    Xo = objects(X)[0]
    ref_loss = O.completion_loss(Xo, idx, y.astype(np.float64))
    _, ref_grad = O.completion_loss_grad(Xo, idx, y.astype(np.float64))
    assert abs(float(loss.detach()) - ref_loss) / abs(ref_loss) < TOL["fp32"]
    got = _host_cores(lib, Xt.data.grad, Xt)
    assert rel_err_cores([g[0] for g in got], [3.0 * g for g in ref_grad]) < TOL["fp32"]
    # central differences of the CUDA forward along a random direction
    D = torch.randn_like(Xt.data)
    f = lambda d: AG.completion_loss(lib.TT(d, Xt.n, Xt.ranks, 1), idx_d, y_d)
    fd = _fd(f, Xt.data.detach(), D, 1e-2)
    ad = float((Xt.data.grad.double() * D.double()).sum()) / 3.0
    assert abs(fd - ad) / abs(ad) < 1e-3


def test_completion_loss_no_grad_matches(lib):
    from paper_1801_01928_gb300 import autograd as AG
    cfg = S.config1()
    X = round32(cfg.X)
    Xt = _tt(lib, X)
    idx = torch.tensor(cfg.idx, device="cuda")
    y = torch.zeros(cfg.idx.shape[1], device="cuda")
    loss = AG.completion_loss(Xt, idx, y)
    ref = 0.5 * float(np.sum(O.gather(objects(X)[0], cfg.idx) ** 2))
    assert abs(float(loss) - ref) / ref < TOL["fp32"]


@pytest.mark.parametrize("same", [False, True])
def test_gram_autograd(lib, same):
    from paper_1801_01928_gb300 import autograd as AG
    torch.manual_seed(501)
    rng = np.random.default_rng(501)
    n = [3, 4, 2, 5]
    A = round32(S.random_tt(rng, 7, n, [1, 3, 5, 2, 1], 0.5))
    Bc = A if same else round32(S.random_tt(rng, 5, n, [1, 2, 4, 3, 1], 0.5))
    At = _tt(lib, A)
    At.data.requires_grad_(True)
    if same:
        Bt = At
    else:
        Bt = _tt(lib, Bc)
        Bt.data.requires_grad_(True)
    W = torch.randn(At.batch, Bt.batch, device="cuda")
    G = AG.gram(At, Bt)
    (G * W).sum().backward()
    dA, dB = O.gram_vjp(objects(A), objects(Bc), W.double().cpu().numpy())
    if same:
        want = [[a + b for a, b in zip(x, y)] for x, y in zip(dA, dB)]
        assert rel_err_cores(_host_cores(lib, At.data.grad, At), batched(want)) < TOL["fp32"]
    else:
        assert rel_err_cores(_host_cores(lib, At.data.grad, At), batched(dA)) < TOL["fp32"]
        assert rel_err_cores(_host_cores(lib, Bt.data.grad, Bt), batched(dB)) < TOL["fp32"]
    # full(A) is multilinear in A's cores, so f is a polynomial of degree d (2d for B = A)
    # along DA; the five-point difference keeps its truncation far below the tolerance
    DA = torch.randn_like(At.data)
    if same:
        f = lambda d: (AG.gram(lib.TT(d, At.n, At.ranks, At.batch), lib.TT(d, At.n, At.ranks, At.batch)).double()
                       * W.double()).sum()
        fd = _fd(f, At.data.detach(), DA, 1e-2)
        ad = float((At.data.grad.double() * DA.double()).sum())
    else:
        f = lambda d: (AG.gram(lib.TT(d, At.n, At.ranks, At.batch), Bt).double() * W.double()).sum()
        fd = _fd(f, At.data.detach(), DA, 1e-2)
        ad = float((At.data.grad.double() * DA.double()).sum())
    assert abs(fd - ad) / abs(ad) < 1e-3


def test_project_sum_autograd(lib):
    from paper_1801_01928_gb300 import autograd as AG
    torch.manual_seed(502)
    cfg = S.config5(batch=23, d=5, n=4, rX=5, rZ=3, seed=502)
    X, Z = round32(cfg.X), round32(cfg.Z)
    c = cfg.c.astype(np.float32)
    U, V = lib.orthogonalize(_tt(lib, X))
    Zt = _tt(lib, Z)
    Zt.data.requires_grad_(True)
    ct = torch.tensor(c, device="cuda", requires_grad=True)
    dU = AG.project_sum(U, V, Zt, ct)
    Uo, Vo, _ = O.orthogonalize(objects(X)[0])
    ref = O.project_sum(Uo, Vo, objects(Z), c.astype(np.float64))
    assert rel_err_cores([x[0] for x in _host_cores(lib, dU.data, dU)], ref) < TOL["fp32"]
    Rbar = torch.randn_like(dU.data)
    (dU.data * Rbar).sum().backward()
    rb = lib.TT(Rbar, U.n, U.ranks, 1)
    rZ, rc = O.project_sum_vjp(Uo, Vo, objects(Z), c.astype(np.float64),
                               [x.double().cpu().numpy()[0] for x in rb.cores()])
    assert rel_err_cores(_host_cores(lib, Zt.data.grad, Zt), batched(rZ)) < TOL["fp32"]
    assert rel_err(ct.grad.cpu().numpy(), rc) < TOL["fp32"]
    # project_sum is linear in each Z_j as a tensor, i.e. multilinear in its cores
    DZ = torch.randn_like(Zt.data)
    f = lambda d: (AG.project_sum(U, V, lib.TT(d, Zt.n, Zt.ranks, Zt.batch), ct.detach()).data.double()
                   * Rbar.double()).sum()
    fd = _fd(f, Zt.data.detach(), DZ, 1e-2)
    ad = float((Zt.data.grad.double() * DZ.double()).sum())
    assert abs(fd - ad) / abs(ad) < 1e-3


@pytest.mark.parametrize("math_", ["tf32", "bf16"])
def test_gram_autograd_tensor_cores(lib, math_):
    # the tensor-core forward and adjoint behind torch.autograd, against the oracle's
    # cotangents at the math's tolerance (A and B distinct, both requiring gradients)
    from paper_1801_01928_gb300 import autograd as AG
    torch.manual_seed(502)
    rng = np.random.default_rng(502)
    n = [3, 4, 2, 5]
    A = round32(S.random_tt(rng, 9, n, [1, 6, 20, 9, 1], 0.3))
    Bc = round32(S.random_tt(rng, 6, n, [1, 4, 12, 30, 1], 0.3))
    At, Bt = _tt(lib, A), _tt(lib, Bc)
    At.data.requires_grad_(True)
    Bt.data.requires_grad_(True)
    W = torch.randn(At.batch, Bt.batch, device="cuda")
    G = AG.gram(At, Bt, math=math_)
    Gref = O.gram(objects(A), objects(Bc))
    assert rel_err(G.detach().double().cpu().numpy(), Gref) < TOL[math_]
    (G * W).sum().backward()
    dA, dB = O.gram_vjp(objects(A), objects(Bc), W.double().cpu().numpy())
    assert rel_err_cores(_host_cores(lib, At.data.grad, At), batched(dA)) < TOL[math_]
    assert rel_err_cores(_host_cores(lib, Bt.data.grad, Bt), batched(dB)) < TOL[math_]
