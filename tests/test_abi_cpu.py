"""CPU checks of the C ABI: the library builds and loads, exports every declared symbol,
validates descriptors (statuses only, no launches) and does the integer rank bookkeeping
exactly as the oracle does."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle as O
import synth as S

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "t3f.h")


@pytest.fixture(scope="module")
def clib():
    from paper_1801_01928_gb300 import build
    path = build.build()
    import paper_1801_01928_gb300 as t3f
    return t3f.load(path)


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\**\s+\**(t3f_[a-z0-9_]+)\s*\(",
                                 src, flags=re.M)))


def test_every_declared_symbol_is_exported(clib):
    names = declared_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(clib, n), n
    import paper_1801_01928_gb300 as t3f
    assert set(t3f.EXPORTS) <= set(names)


def test_status_strings(clib):
    for st in range(-7, 1):
        assert clib.t3f_status_string(st).decode().startswith("T3F_")
    assert clib.t3f_version() >= 100


def _desc(t3f, n, ranks, batch=1, m=None, dtype=0, ptr=0x1000):
    class _T:
        pass
    keep = []
    arr = lambda v: (ctypes.c_int32 * len(v))(*v)
    nn, rr = arr(n), arr(ranks)
    mm = arr(m) if m is not None else None
    keep += [nn, rr, mm]
    d = t3f._binding._Desc(batch, len(n), mm, nn, rr, ctypes.c_void_p(ptr), dtype)
    d._keep = keep
    return d


def test_descriptor_validation_statuses(clib):
    import paper_1801_01928_gb300 as t3f
    A = _desc(t3f, [3, 3, 3], [1, 2, 2, 1])
    B = _desc(t3f, [3, 4, 3], [1, 2, 2, 1])
    G = ctypes.c_void_p(0x2000)
    s = ctypes.c_void_p(0)
    assert clib.t3f_gram(ctypes.byref(A), ctypes.byref(B), G, 0, None, 0, s) == -2  # shape
    bad = _desc(t3f, [3, 3, 3], [2, 2, 2, 1])
    assert clib.t3f_gram(ctypes.byref(bad), ctypes.byref(A), G, 0, None, 0, s) == -2
    nul = _desc(t3f, [3, 3, 3], [1, 2, 2, 1], ptr=0)
    assert clib.t3f_gram(ctypes.byref(nul), ctypes.byref(A), G, 0, None, 0, s) == -1
    assert clib.t3f_gram(ctypes.byref(A), ctypes.byref(A), None, 0, None, 0, s) == -1
    assert clib.t3f_gram(ctypes.byref(A), ctypes.byref(A), G, 7, None, 0, s) == -1
    f64 = _desc(t3f, [3, 3, 3], [1, 2, 2, 1], dtype=1)
    assert clib.t3f_gram(ctypes.byref(f64), ctypes.byref(f64), G, 0, None, 0, s) == -3
    big = _desc(t3f, [3, 3, 3], [1, 65, 2, 1])
    assert clib.t3f_gram(ctypes.byref(big), ctypes.byref(big), G, 0, None, 0, s) == -7
    # gather: batch must be 1, workspace checked before any launch
    X2 = _desc(t3f, [3, 3, 3], [1, 2, 2, 1], batch=2)
    assert clib.t3f_gather(ctypes.byref(X2), G, 10, None, G, None, None, 0, s) == -2
    assert clib.t3f_gather(ctypes.byref(A), G, 10, None, G, None, None, 0, s) == -4
    assert clib.t3f_gather(ctypes.byref(A), G, -1, None, G, None, None, 0, s) == -1
    # matvec: A must be a TT-matrix whose column modes match x
    M = _desc(t3f, [3, 3, 3], [1, 2, 2, 1], m=[2, 2, 2])
    C = _desc(t3f, [2, 2, 2], [1, 4, 4, 1])
    Cbad = _desc(t3f, [2, 2, 2], [1, 4, 3, 1])
    assert clib.t3f_matvec(ctypes.byref(A), ctypes.byref(A), ctypes.byref(C), None, 0, s) == -2
    assert clib.t3f_matvec(ctypes.byref(M), ctypes.byref(A), ctypes.byref(Cbad), None, 0, s) == -2
    # project_sum: U, V must be single objects
    U2 = _desc(t3f, [3, 3, 3], [1, 2, 2, 1], batch=2)
    assert clib.t3f_project_sum(ctypes.byref(U2), ctypes.byref(U2), ctypes.byref(A), G,
                                ctypes.byref(U2), 0, None, 0, s) == -2


def test_orth_ranks_bit_exact_against_oracle(clib):
    import paper_1801_01928_gb300 as t3f
    rng = np.random.default_rng(7)
    for _ in range(200):
        d = int(rng.integers(1, 12))
        n = [int(v) for v in rng.integers(1, 9, size=d)]
        ranks = [1] + [int(v) for v in rng.integers(1, 70, size=d - 1)] + [1]
        assert t3f.orth_ranks(n, ranks) == O.orth_ranks(n, ranks)
    assert t3f.orth_ranks([16] * 20, S.tt_ranks(20, 32)) == [1, 16] + [32] * 17 + [16, 1]


def test_packed_size_and_workspace(clib):
    import paper_1801_01928_gb300 as t3f
    n, r = [4, 5, 6], [1, 3, 2, 1]
    A = _desc(t3f, n, r, batch=7)
    assert clib.t3f_packed_size(ctypes.byref(A)) == t3f.TT.numel(n, r, 7)
    M = _desc(t3f, n, r, batch=2, m=[2, 3, 2])
    assert clib.t3f_packed_size(ctypes.byref(M)) == t3f.TT.numel(n, r, 2, [2, 3, 2])
    X = _desc(t3f, n, r)
    assert clib.t3f_workspace_size(4, ctypes.byref(X), None, 1000) >= 256
    assert clib.t3f_workspace_size(5, ctypes.byref(X), None, 1000) > clib.t3f_workspace_size(4, ctypes.byref(X), None, 1000)
    assert clib.t3f_workspace_size(10, ctypes.byref(X), ctypes.byref(A), 0) > 0
    assert clib.t3f_workspace_size(99, ctypes.byref(X), None, 0) == 0


def _ragged_meta(t3f, shapes):
    """A RaggedTT descriptor for the given (modes, ranks) per object over a dummy host buffer:
    the grouped-Gram planner reads shapes only."""
    torch = pytest.importorskip("torch")
    dims = [len(m) for m, _ in shapes]
    modes = [list(m) for m, _ in shapes]
    ranks = [list(r) for _, r in shapes]
    offs, o = [], 0
    for m, r in shapes:
        offs.append(o)
        o += sum(r[k] * m[k] * r[k + 1] for k in range(len(m)))
    return t3f.RaggedTT(torch.zeros(1), dims, modes, ranks, offs)


def test_gram_groups_planner_on_host(clib):
    # the whole work-list planner (rank-adaptive forward tiles, the adjoint's two lists) runs
    # on the host: the bench-size uneven batch, per-core varying ranks, d = 1 and n = 1 groups,
    # every tile-side cap; an out-of-range cap is rejected (size 0)
    import paper_1801_01928_gb300 as t3f
    cfg = S.config4()
    shapes, gstart = [], [0]
    for grp in cfg.groups:
        for r in grp.ranks:
            shapes.append(([grp.n] * grp.d, S.tt_ranks(grp.d, int(r))))
        gstart.append(len(shapes))
    rng = np.random.default_rng(7)
    for d, n in ((1, [5]), (2, [1, 3]), (5, [2, 3, 2, 2, 3])):
        for _ in range(9):
            shapes.append((n, [1] + [int(rng.integers(1, 65)) for _ in range(d - 1)] + [1]))
        gstart.append(len(shapes))
    X = _ragged_meta(t3f, shapes)
    gs = (ctypes.c_int32 * len(gstart))(*gstart)
    sizes = []
    for tiles in (None, (16, 10, 4, 8), (1, 1, 1, 1), (16, 16, 16, 16)):
        tl = None if tiles is None else (ctypes.c_int32 * 4)(*tiles)
        ws = clib.t3f_gram_groups_workspace_size(ctypes.byref(X.desc()), len(gstart) - 1, gs, tl)
        assert ws > 0, tiles
        sizes.append(ws)
    assert len(set(sizes)) > 1  # the caps change the forward work list
    bad = (ctypes.c_int32 * 4)(16, 0, 4, 8)
    assert clib.t3f_gram_groups_workspace_size(ctypes.byref(X.desc()), len(gstart) - 1, gs, bad) == 0
