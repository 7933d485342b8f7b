"""Benchmark of the TT-sweep hot path on one GB300 (or N independent replicas under torchrun).

One step = one pass of every hot-path operation over its synthetic workload:
  completion   gather loss + adjoint, 1e6 int32 tuples, d=10, n=10, model rank 8
  rgrad        FP64 orthogonalisation of that X + Riemannian gradient of the same loss
  gram         100 x 100 Gram matrix, d=10, n=10, r=10, forward + adjoint, norms
  matvec       100 TT-matrices (4x4 modes, r=10) zip 100 TT-vectors (r=10), fwd + adjoint
  psum         FP64 orthogonalisation of X (d=20, n=16, r=32) + project_sum of 1000 rank-8
               TTs and the adjoint of ||project_sum||^2
  uneven       512 ragged TTs in 8 groups of 64 (d in [4,16], n in [2,16], r in [2,64]): all
               pairwise inner products within groups + FP64 norms + adjoint, one persistent
               work-queue launch with autotuned rank-bucket tiles, replayed as a CUDA graph
value = algorithmic FLOPs of the step / device time of the step (GFLOP/s, FP32).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

# the CPU baseline is the oracle as it stands: pin its BLAS to one thread and report 1 core
for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import numpy as np  # noqa: E402

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth as S  # noqa: E402

METRIC = "TT-sweep GFLOP/s and % roofline (Gram, gather fwd+bwd, project_sum) vs plain FP32"
WORKLOAD = ("t3f-hot-path: completion(N=1e6,d=10,n=10,r=8)+rgrad + gram(100x100,d=10,n=10,r=10)"
            "+bwd+norm + matvec(100,d=10,4x4,r=10)+bwd + orth+project_sum(1000,d=20,n=16,rX=32,rZ=8)+bwd"
            " + uneven(8x64 ragged TTs, d 4-16, n 2-16, r 2-64: grouped gram+norms+bwd, graph replay)")
L2_BYTES = 129 * 1024 * 1024
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12   # SMs x FP32 lanes x FMA x max SM clock


# ---------------------------------------------------------------------------------------
# algorithmic FLOP counts (shape arithmetic only)
# ---------------------------------------------------------------------------------------

def f_left_sweep(n, ra, rb):
    """T_i = M B_i (2 ra0 rb0 rb1), M' += A_i^T T_i (2 ra1 ra0 rb1), per slice."""
    return sum(2 * n[k] * ra[k] * rb[k + 1] * (rb[k] + ra[k + 1]) for k in range(len(n)))


def f_right_sweep(n, ra, rb):
    """T_i = A_i R (2 ra0 ra1 rb1), R' += T_i B_i^T (2 ra0 rb1 rb0), per slice."""
    return sum(2 * n[k] * ra[k] * rb[k + 1] * (ra[k + 1] + rb[k]) for k in range(len(n)))


def f_gram_bwd(n, ra, rb):
    g = sum(2 * n[k] * ra[k + 1] * rb[k] * (rb[k + 1] + ra[k])        # dA: B_i R^T, M (.)
            + 2 * n[k] * rb[k] * ra[k] * rb[k + 1] for k in range(len(n)))  # dB: M^T (A_i R)
    return f_left_sweep(n, ra, rb) + f_right_sweep(n, ra, rb) + g


def f_chain(r):
    return sum(2 * r[k] * r[k + 1] for k in range(1, len(r) - 1))


def f_completion(r):
    """value chain + second chain + outer products, per tuple (fwd 1040 + bwd 2096 at r=8)."""
    d = len(r) - 1
    outer = sum(2 * r[k] * r[k + 1] for k in range(d))
    return 2 * f_chain(r) + outer


def f_gauge(n, r):
    return sum(4 * r[k] * n[k] * r[k + 1] * r[k + 1] for k in range(len(n) - 1))


def f_qr(m, c):
    k = min(m, c)
    fac = 2 * m * c * k - (m + c) * k * k + 2 * k ** 3 / 3
    form_q = 4 * m * k * k - 2 * (m + k) * k * k + 4 * k ** 3 / 3
    return fac + form_q


def f_orth(n, ranks):
    """three Householder sweeps (right-left, left-right, right-left) with the R products."""
    d = len(n)
    r = list(ranks)
    tot = 0.0

    def rl(r):
        nonlocal tot
        r = list(r)
        for k in range(d - 1, 0, -1):
            m, c = n[k] * r[k + 1], r[k]
            kk = min(m, c)
            tot += f_qr(m, c) + 2 * r[k - 1] * n[k - 1] * c * kk
            r[k] = kk
        return r

    def lr(r):
        nonlocal tot
        r = list(r)
        for k in range(d - 1):
            m, c = r[k] * n[k], r[k + 1]
            kk = min(m, c)
            tot += f_qr(m, c) + 2 * kk * c * n[k + 1] * r[k + 2]
            r[k + 1] = kk
        return r

    r = lr(rl(r))
    rl(r)
    return tot


def f_matvec(m, n, ra, rx):
    return sum(2 * n[k] * ra[k] * rx[k] * m[k] * ra[k + 1] * rx[k + 1] for k in range(len(n)))


def f_psum_fwd(n, ru, rz, batch):
    asm = sum(2 * n[k] * ru[k] * rz[k + 1] * (rz[k] + ru[k + 1]) for k in range(len(n)))
    return batch * (f_left_sweep(n, ru, rz) + f_right_sweep(n, ru, rz) + asm) + f_gauge(n, ru)


def f_psum_bwd(n, ru, rz, batch):
    d = len(n)
    P = 2 * f_left_sweep(n, ru, rz)                                   # V- and W-terms
    Q = sum(2 * n[k] * (2 * ru[k] * ru[k + 1] * rz[k + 1] + ru[k] * rz[k + 1] * rz[k]) for k in range(d))
    G = sum(2 * n[k] * (3 * rz[k] * ru[k] * ru[k + 1] + 2 * rz[k] * ru[k + 1] * rz[k + 1]) for k in range(d))
    return batch * (f_left_sweep(n, ru, rz) + f_right_sweep(n, ru, rz) + P + Q + G) + f_gauge(n, ru)


def f_project_batch(n, ru, rz, batch):
    """per object: both sweeps, the per-slice assembly and the per-object gauge projection."""
    asm = sum(2 * n[k] * ru[k] * rz[k + 1] * (rz[k] + ru[k + 1]) for k in range(len(n)))
    return batch * (f_left_sweep(n, ru, rz) + f_right_sweep(n, ru, rz) + asm + f_gauge(n, ru))


def f_project_matvec(m, n, rx, ra, rc, batch):
    """per object: left and right Kronecker sweeps (c-step, A-step, X-step) and the assembly."""
    d = len(n)
    tot = 0.0
    for k in range(d):
        x0, x1, a0, a1, b0, b1 = rx[k], rx[k + 1], ra[k], ra[k + 1], rc[k], rc[k + 1]
        left = 2 * x0 * a0 * n[k] * b1 * b0 + 2 * x0 * m[k] * a1 * b1 * a0 * n[k] + 2 * x1 * a1 * b1 * x0 * m[k]
        right = 2 * x1 * a1 * n[k] * b0 * b1 + 2 * x1 * m[k] * a0 * b0 * a1 * n[k] + 2 * x0 * a0 * b0 * x1 * m[k]
        asm = 2 * x0 * a0 * n[k] * b1 * b0 + 2 * x0 * m[k] * a1 * b1 * a0 * n[k] + 2 * x0 * m[k] * x1 * a1 * b1
        tot += left + right + asm
    return batch * (tot + f_gauge(m, rx))


def f_round(n, ranks, maxr):
    """TT rounding, non-iterative part: the right-to-left Householder QRs (factor + form Q)
    with the R products, then per interface the Gram matrix of the smaller side, the left
    singular vectors (when formed from M V) and the S V^T product into the next core (the
    Jacobi sweeps, an iteration, are not counted)."""
    d = len(n)
    r = list(ranks)
    tot = 0.0
    for k in range(d - 1, 0, -1):
        m, c = n[k] * r[k + 1], r[k]
        q = min(m, c)
        tot += f_qr(m, c) + 2 * r[k - 1] * n[k - 1] * c * q
        r[k] = q
    rr = [1] + [0] * d
    for k in range(d - 1):
        m, c = rr[k] * n[k], r[k + 1]
        s = min(m, c)
        p = min(maxr, s)
        tot += 2 * s * s * max(m, c) + (2 * m * c * p if m > c else 2 * p * m * c) + 2 * p * c * n[k + 1] * r[k + 2]
        rr[k + 1] = p
    return tot


def f_hvp(r, n, N):
    """tangent-vector gather (three chains of r x r products per core) + the Riemannian scatter."""
    d = len(r) - 1
    gather = sum(3 * 2 * r[k] * r[k + 1] for k in range(d))
    return N * (gather + f_completion(r)) + f_gauge(n, r)


# ---------------------------------------------------------------------------------------
# workload
# ---------------------------------------------------------------------------------------

class Workload:
    """Host (pinned) and device copies of every input of one step."""

    def __init__(self, t3f, torch, dev, seed_offset=0):
        self.t3f, self.torch, self.dev = t3f, torch, dev
        f32 = lambda cs: [np.asarray(c, np.float32) for c in cs]
        c2 = S.config2(seed=2 + seed_offset)
        c3 = S.config3a(seed=3 + seed_offset)
        c3b = S.config3b(seed=4 + seed_offset)
        c5 = S.config5(seed=6 + seed_offset)
        rng = np.random.default_rng(1000 + seed_offset)
        self.shapes = dict(c2=c2, c3=c3, c3b=c3b, c5=c5)
        host = {}
        # completion targets y = T(i) + noise, with T(i) from the library's own gather
        T = t3f.TT.from_cores(f32(c2.T), device=dev)
        idx_d = torch.tensor(c2.idx, device=dev)
        tv, _ = t3f.gather(T, idx_d)
        host["y"] = (tv.cpu().double().numpy() + c2.noise).astype(np.float32)
        host["idx"] = c2.idx
        host["X2"] = np.concatenate([c.ravel() for c in f32(c2.X)])
        host["A3"] = np.concatenate([c.ravel() for c in f32(c3.A)])
        host["B3"] = np.concatenate([c.ravel() for c in f32(c3.B)])
        host["dG"] = rng.normal(size=(100, 100)).astype(np.float32)
        host["Am"] = np.concatenate([c.ravel() for c in f32(c3b.A)])
        host["xv"] = np.concatenate([c.ravel() for c in f32(c3b.x)])
        host["X5"] = np.concatenate([c.ravel() for c in f32(c5.X)])
        host["Z5"] = np.concatenate([c.ravel() for c in f32(c5.Z)])
        host["c5"] = c5.c.astype(np.float32)
        self.meta = {
            "X2": ([c.shape[2] for c in c2.X], [1] + [c.shape[3] for c in c2.X], 1, None),
            "A3": ([10] * 10, S.tt_ranks(10, 10), 100, None),
            "B3": ([10] * 10, S.tt_ranks(10, 10), 100, None),
            "Am": ([4] * 10, S.tt_ranks(10, 10), 100, [4] * 10),
            "xv": ([4] * 10, S.tt_ranks(10, 10), 100, None),
            "X5": ([16] * 20, S.tt_ranks(20, 32), 1, None),
            "Z5": ([16] * 20, S.tt_ranks(20, 8), 1000, None),
        }
        # matvec cotangent: one fixed random TT of the product's shape
        rc = [a * b for a, b in zip(S.tt_ranks(10, 10), S.tt_ranks(10, 10))]
        dC = np.concatenate([rng.normal(size=(100, rc[k], 4, rc[k + 1])).astype(np.float32).ravel() for k in range(10)])
        host["dC"] = dC
        self.meta["dC"] = ([4] * 10, rc, 100, None)
        # uneven batches: 8 groups of 64 ragged TTs, stored back to back
        c4 = S.config4(seed=5 + seed_offset)
        objs = [[np.asarray(c, np.float32) for c in o] for grp in c4.groups for o in grp.cores]
        self.gstart = [0]
        for grp in c4.groups:
            self.gstart.append(self.gstart[-1] + len(grp.cores))
        r4 = t3f.RaggedTT.from_objects(objs, device="cpu")
        host["X4"] = r4.data.numpy()
        self.r4meta = (r4.dims, r4.modes, r4.ranks, r4.offsets)
        self.shapes["c4"] = c4
        ntot = sum((self.gstart[g + 1] - self.gstart[g]) ** 2 for g in range(len(self.gstart) - 1))
        host["dG4"] = rng.normal(size=ntot).astype(np.float32)
        self.host = {k: torch.from_numpy(np.ascontiguousarray(v)).pin_memory() for k, v in host.items()}
        # inputs of the tangent-space rows measured beside the step: the first 100 TTs of the
        # projection batch, the first TT-matrix of the matvec batch and a rank-10 point (d=10, n=4)
        Z100 = [np.asarray(cz[:100], np.float32) for cz in c5.Z]
        A1 = [np.asarray(ca[:1], np.float32) for ca in c3b.A]
        Xp = S.random_tt(np.random.default_rng(7 + seed_offset), 1, 4, S.tt_ranks(10, 10), 1 / math.sqrt(10))
        self.next_dev = {
            "Z100": torch.tensor(np.concatenate([c.ravel() for c in Z100]), device=dev),
            "A1": torch.tensor(np.concatenate([c.ravel() for c in A1]), device=dev),
            "Xp": torch.tensor(np.concatenate([np.asarray(c, np.float32).ravel() for c in Xp]), device=dev),
        }
        self.h2d_bytes = sum(v.numel() * v.element_size() for v in self.host.values())
        self.devbuf = {k: torch.empty_like(v, device=dev) for k, v in self.host.items()}
        self.upload(torch.cuda.current_stream(dev))
        torch.cuda.synchronize(dev)

    def upload(self, stream):
        for k, v in self.host.items():
            self.devbuf[k].copy_(v, non_blocking=True)

    # inputs in the order the step first reads them: the main stream starts with the Gram
    # matrix and norms (8 MB of inputs), then takes the completion loss, the uneven batch, the
    # Gram adjoint and the matvec calls; the side stream reaches orth5 (the X5 group) after a
    # few milliseconds, and dC (128 MB) is read last
    UPLOAD_GROUPS = (("A3", "B3", "dG"), ("X2", "idx", "y"), ("X4", "dG4"), ("X5", "Z5", "c5"),
                     ("Am", "xv", "dC"))

    def upload_async(self, copy_stream):
        """Every input copied from pinned host memory on `copy_stream`, one group at a time;
        returns input name -> CUDA event recorded after its group, so each operation waits
        for its own inputs only and the copies of later groups overlap earlier compute."""
        torch = self.torch
        ready = {}
        with torch.cuda.stream(copy_stream):
            for grp in self.UPLOAD_GROUPS:
                for k in grp:
                    self.devbuf[k].copy_(self.host[k], non_blocking=True)
                ev = torch.cuda.Event()
                ev.record(copy_stream)
                for k in grp:
                    ready[k] = ev
        assert set(ready) == set(self.host), "every input belongs to one upload group"
        return ready

    def ragged(self):
        return self.t3f.RaggedTT(self.devbuf["X4"], *self.r4meta)

    def prepare_uneven(self):
        """Autotune the rank-bucket tiles, prepare the work list and capture the grouped
        forward + adjoint in a CUDA graph (all outside the timed region)."""
        t3f, torch = self.t3f, self.torch
        X4 = self.ragged()
        self.tiles4, _ = t3f.autotune_gram_groups(X4, self.gstart, reps=2)
        self.ws4 = t3f.gram_groups_prepare(X4, self.gstart, self.tiles4)
        total = self.devbuf["dG4"].numel()
        self.G4 = torch.empty(total, dtype=torch.float32, device=self.dev)
        self.n4 = torch.empty(X4.count, dtype=torch.float64, device=self.dev)
        self.dX4 = torch.empty(X4.data.numel(), dtype=torch.float32, device=self.dev)
        side = torch.cuda.Stream(self.dev)
        side.wait_stream(torch.cuda.current_stream(self.dev))
        with torch.cuda.stream(side):
            t3f.gram_groups(X4, self.gstart, self.ws4, self.tiles4, out=self.G4, norms=self.n4)
            t3f.gram_groups_backward(X4, self.gstart, self.ws4, self.devbuf["dG4"], self.tiles4, dcores=self.dX4)
        torch.cuda.current_stream(self.dev).wait_stream(side)
        # kernels per replay: the library's launch counter advances during capture
        n0 = t3f.launch_count()
        self.graph4f = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph4f):
            t3f.gram_groups(X4, self.gstart, self.ws4, self.tiles4, out=self.G4, norms=self.n4)
        n1 = t3f.launch_count()
        self.graph4b = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph4b):
            t3f.gram_groups_backward(X4, self.gstart, self.ws4, self.devbuf["dG4"], self.tiles4, dcores=self.dX4)
        self.graph_kernels = (n1 - n0) + (t3f.launch_count() - n1)
        torch.cuda.synchronize(self.dev)

    def tt(self, key):
        n, r, b, m = self.meta[key]
        return self.t3f.TT(self.devbuf[key], n, r, b, m)

    def flops(self):
        c2 = self.shapes["c2"]
        r2 = S.tt_ranks(10, 8)
        n10 = [10] * 10
        ru2 = self.t3f.orth_ranks(n10, r2)
        r10 = S.tt_ranks(10, 10)
        n16 = [16] * 20
        ru5 = self.t3f.orth_ranks(n16, S.tt_ranks(20, 32))
        rz5 = S.tt_ranks(20, 8)
        N = c2.idx.shape[1]
        return {
            "completion": N * f_completion(r2),
            "orth2": f_orth(n10, r2),
            "rgrad": N * f_completion(ru2) + f_gauge(n10, ru2),
            "gram": 100 * 100 * f_left_sweep(n10, r10, r10),
            "gram_bwd": 100 * 100 * f_gram_bwd(n10, r10, r10),
            "norm": 100 * f_left_sweep(n10, r10, r10),
            "matvec": 100 * f_matvec([4] * 10, [4] * 10, r10, r10),
            "matvec_bwd": 2 * 100 * f_matvec([4] * 10, [4] * 10, r10, r10),
            "orth5": f_orth(n16, S.tt_ranks(20, 32)),
            "psum": f_psum_fwd(n16, ru5, rz5, 1000),
            "psum_bwd": f_psum_bwd(n16, ru5, rz5, 1000),
            "uneven": self.uneven_flops(False),
            "uneven_bwd": self.uneven_flops(True),
        }

    def uneven_flops(self, bwd):
        """Unique pairs (a <= b) of every group: the left sweep (forward) or the adjoint."""
        dims, modes, ranks, _ = self.r4meta
        tot = 0.0
        for g in range(len(self.gstart) - 1):
            for a in range(self.gstart[g], self.gstart[g + 1]):
                for b in range(a, self.gstart[g + 1]):
                    f = f_gram_bwd if bwd else f_left_sweep
                    tot += f(modes[a], ranks[a], ranks[b])
        return tot


def combine_ranks(dev_ms, e2e_ms, world, step_flops, device):
    """Whole-job numbers of `world` replicas: the per-rank step times are reduced with MAX
    (the slowest replica sets the step time) and the job processes `world` steps' FLOPs per
    step. Returns (dev_ms, e2e_ms, value GFLOP/s, e2e GFLOP/s)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([dev_ms, e2e_ms], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dev_ms, e2e_ms = float(t[0]), float(t[1])
    return (dev_ms, e2e_ms, world * step_flops / (dev_ms * 1e-3) / 1e9,
            world * step_flops / (e2e_ms * 1e-3) / 1e9)


def op_graph_times(w, flush, stream):
    """Device time of every operation of the step on its own: each one (with the inputs the
    step gives it) captured as a CUDA graph and timed by replay with L2 flushed before every
    replay, so operations shorter than their host-side call are timed on the device. The
    uneven batch is already a graph and is replayed as it stands."""
    t3f, torch = w.t3f, w.torch
    X2, idx, y = w.tt("X2"), w.devbuf["idx"], w.devbuf["y"]
    U2, V2 = t3f.orthogonalize(X2)
    X5, Z5, c5 = w.tt("X5"), w.tt("Z5"), w.devbuf["c5"]
    U5, V5 = t3f.orthogonalize(X5)
    dU5 = t3f.project_sum(U5, V5, Z5, c5)
    A3, B3, dG = w.tt("A3"), w.tt("B3"), w.devbuf["dG"]
    Am, xv, dC = w.tt("Am"), w.tt("xv"), w.tt("dC")
    fns = {
        "completion": lambda: t3f.gather_backward(X2, idx, y=y, want_loss=True),
        "orth2": lambda: t3f.orthogonalize(X2),
        "rgrad": lambda: t3f.gather_backward(None, idx, y=y, riemannian=True, U=U2, V=V2),
        "orth5": lambda: t3f.orthogonalize(X5),
        "psum": lambda: t3f.project_sum(U5, V5, Z5, c5),
        "psum_bwd": lambda: t3f.project_sum_backward(U5, V5, Z5, c5, dU5),
        "gram": lambda: t3f.gram(A3, B3),
        "gram_bwd": lambda: t3f.gram_backward(A3, B3, dG),
        "norm": lambda: t3f.norm(A3),
        "matvec": lambda: t3f.matvec(Am, xv),
        "matvec_bwd": lambda: t3f.matvec_backward(Am, xv, dC),
    }
    out = {k: graph_time(torch, f, flush, stream, reps=5) for k, f in fns.items()}
    for key, g in (("uneven", w.graph4f), ("uneven_bwd", w.graph4b)):
        out[key] = event_time(torch, g.replay, flush, stream)
    return out


def run_step(w, timers=None, stream=None, side=None, ready=None, emit=None):
    """All hot-path operations once; returns the outputs a user reads back.

    With `side` (a second CUDA stream) the orthogonalisation chain (orth2 -> Riemannian
    gradient, orth5 -> project_sum -> its adjoint), which does not depend on the other
    operations, is issued first on `side` and runs concurrently with the rest on the main
    stream: the FP64 orthogonalisation is a chain of small QR steps on one 16-CTA cluster, so
    the other SMs take the independent work meanwhile. Without `side` every operation runs
    in order on the main stream (the per-operation timings come from that form). With
    `ready` (input name -> event of its host-to-device copy) each operation first waits for
    the copies of its own inputs; with `emit` (name, tensor, stream) each result is handed
    over as soon as the operation that writes it has been issued (for the read-back). The
    main stream starts with the Gram matrix and norms, whose inputs are small, while the
    completion inputs are still being copied; the uneven batch runs after the completion loss,
    so the Gram adjoint and matvec calls that follow it overlap the read-back of its
    gradient."""
    t3f, torch = w.t3f, w.torch
    out = {}
    main = stream if stream is not None else torch.cuda.current_stream(w.dev)

    def need(st, *keys):
        if ready is not None:
            for ev in {id(ready[k]): ready[k] for k in keys}.values():
                st.wait_event(ev)

    def give(st, **kv):
        if emit is not None:
            for k, v in kv.items():
                emit(k, v, st)

    def timed(name, fn, st):
        if timers is not None:
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(st)
            r = fn()
            e1.record(st)
            timers.setdefault(name, []).append((e0, e1))
            return r
        return fn()

    X2 = w.tt("X2")
    idx = w.devbuf["idx"]
    y = w.devbuf["y"]
    X5, Z5 = w.tt("X5"), w.tt("Z5")
    c5 = w.devbuf["c5"]
    res = {}

    def orth_chain(st):
        need(st, "X2", "idx", "y")
        U2, V2 = timed("orth2", lambda: t3f.orthogonalize(X2), st)
        res["dU2"], _ = timed("rgrad", lambda: t3f.gather_backward(None, idx, y=y, riemannian=True, U=U2, V=V2), st)
        give(st, dU2=res["dU2"].data)
        need(st, "X5", "Z5", "c5")
        U5, V5 = timed("orth5", lambda: t3f.orthogonalize(X5), st)
        res["dU5"] = timed("psum", lambda: t3f.project_sum(U5, V5, Z5, c5), st)
        give(st, dU5=res["dU5"].data)
        # adjoint of 1/2 ||project_sum||^2: the cotangent of the coordinates is dU5 itself
        res["dZ"], res["dc"] = timed("psum_bwd", lambda: t3f.project_sum_backward(U5, V5, Z5, c5, res["dU5"]), st)
        give(st, dc=res["dc"])

    if side is not None:
        side.wait_stream(main)
        with torch.cuda.stream(side):
            orth_chain(side)
    A3, B3 = w.tt("A3"), w.tt("B3")
    need(main, "A3", "B3", "dG")
    G = timed("gram", lambda: t3f.gram(A3, B3), main)
    nrm = timed("norm", lambda: t3f.norm(A3), main)
    give(main, G=G, norm=nrm)
    need(main, "X2", "idx", "y")
    dX, loss = timed("completion", lambda: t3f.gather_backward(X2, idx, y=y, want_loss=True), main)
    give(main, loss=loss, dX=dX.data)
    if side is None:
        orth_chain(main)
    need(main, "X4", "dG4")
    timed("uneven", lambda: w.graph4f.replay(), main)
    give(main, G4=w.G4, n4=w.n4)
    timed("uneven_bwd", lambda: w.graph4b.replay(), main)
    give(main, dX4=w.dX4)
    dA, dB = timed("gram_bwd", lambda: t3f.gram_backward(A3, B3, w.devbuf["dG"]), main)
    give(main, dA=dA.data, dB=dB.data)
    Am, xv = w.tt("Am"), w.tt("xv")
    need(main, "Am", "xv", "dC")
    C = timed("matvec", lambda: t3f.matvec(Am, xv), main)
    dAm, dxv = timed("matvec_bwd", lambda: t3f.matvec_backward(Am, xv, w.tt("dC")), main)
    give(main, dAm=dAm.data, dxv=dxv.data)
    if side is not None:
        main.wait_stream(side)
    out.update(loss=loss, dX=dX.data, dU2=res["dU2"].data, G=G, dA=dA.data, dB=dB.data, norm=nrm,
               dAm=dAm.data, dxv=dxv.data, dU5=res["dU5"].data, dc=res["dc"], G4=w.G4, n4=w.n4,
               dX4=w.dX4)
    out["_bulk"] = (C, res["dZ"])  # stay on the device
    return out


def tensor_peaks():
    """Dense tensor peaks (TFLOP/s) for a kernel timed alone: the measured cuBLAS BF16 burst
    figure, and TF32 at NVIDIA's nominal TF32/BF16 ratio (1.1 / 2.25) of it."""
    src, bf16 = "fallback", 1900.0
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            bf16 = float(json.load(f)["bf16_tflops"])
            src = "measured"
    except (OSError, ValueError, KeyError):
        pass
    return {"bf16": bf16, "tf32": bf16 * 1.1 / 2.25}, src


def reduced_precision(w, flops, flush, stream, reps=5):
    """TF32 / BF16 tensor-core Gram and Gram adjoint of config 3a and of the uneven batch (BF16
    on BF16 cores), the FP32 paths on BF16 cores and the TF32 project_sum of config 5, each
    timed by CUDA-graph replay (L2 flushed before every replay) and compared with the FP32
    result of the same inputs (normwise relative difference)."""
    t3f, torch = w.t3f, w.torch
    A3, B3 = w.tt("A3"), w.tt("B3")
    G32 = t3f.gram(A3, B3).double()
    X4 = w.ragged()
    X4b = t3f.RaggedTT(X4.data.to(torch.bfloat16), X4.dims, X4.modes, X4.ranks, X4.offsets)
    ws4b = t3f.gram_groups_prepare(X4b, w.gstart, w.tiles4)
    G4_32 = w.G4.double()

    def timed(fn):
        # device time by CUDA-graph replay (L2 flushed before each replay), as for the step's
        # own uneven batch: the per-call host planning of the grouped calls is not device work
        return graph_time(torch, fn, flush, stream, reps)

    def rel(x, y):
        return float((x.double() - y).norm() / y.norm())

    out = {}
    peaks, psrc = tensor_peaks()

    def roof(gflops, kind):
        return {"bound": "tensor", "achieved": round(gflops / 1e3, 3), "peak": round(peaks[kind], 1),
                "unit": "TFLOP/s", "frac": round(gflops / 1e3 / peaks[kind], 5), "peak_source": psrc,
                "flops": "algorithmic (unpadded ranks)"}

    keep = {}
    for math_ in ("tf32", "bf16"):
        ms = timed(lambda: t3f.gram(A3, B3, math=math_))
        G = t3f.gram(A3, B3, math=math_)
        keep[f"gram_{math_}"] = (G, 5e-3 if math_ == "tf32" else 2e-2)
        gf = flops["gram"] / (ms * 1e-3) / 1e9
        out[f"gram_{math_}"] = {"ms": round(ms, 4), "gflops": round(gf, 1),
                                "diff_vs_fp32": round(rel(G, G32), 6), "roofline": roof(gf, math_),
                                "path": "tcgen05 " + math_ + " products, FP32 accumulation in TMEM"}
    # the uneven adjoint on BF16-stored cores (FP32 arithmetic) next to the FP32 one
    dX32 = w.dX4.double()
    ms = timed(lambda: t3f.gram_groups_backward(X4b, w.gstart, ws4b, w.devbuf["dG4"], w.tiles4))
    dXb = t3f.gram_groups_backward(X4b, w.gstart, ws4b, w.devbuf["dG4"], w.tiles4)
    keep["uneven_bwd_bf16_cores"] = (dXb, 1e-5)
    gf = flops["uneven_bwd"] / (ms * 1e-3) / 1e9
    out["uneven_bwd_bf16_cores"] = {"ms": round(ms, 4), "gflops": round(gf, 1), "diff_vs_fp32": round(rel(dXb, dX32), 6),
                                    "path": "BF16 cores, FP32 CUDA-core arithmetic (adjoint work lists)"}
    # tensor-core adjoints: the uniform Gram (100 x 100) and the uneven batch. Sweeps in both
    # directions store every interface's partials, then (tile, core, side) items run
    # T = gM Y_i and dX_i = T R^T on the tensor cores
    dG3 = w.devbuf["dG"]
    dA32, _ = t3f.gram_backward(A3, B3, dG3)
    for math_ in ("tf32", "bf16"):
        ws3 = t3f.workspace("gram_bwd_tc", A3, B3)
        ms = timed(lambda: t3f.gram_backward(A3, B3, dG3, math=math_, ws=ws3))
        dAx, dBx = t3f.gram_backward(A3, B3, dG3, math=math_, ws=ws3)
        tol = 5e-3 if math_ == "tf32" else 2e-2
        keep[f"gram_bwd_{math_}"] = ((dAx, dBx), tol)
        gf = flops["gram_bwd"] / (ms * 1e-3) / 1e9
        out[f"gram_bwd_{math_}"] = {"ms": round(ms, 4), "gflops": round(gf, 1),
                                    "diff_vs_fp32": round(rel(dAx.data, dA32.data.double()), 6),
                                    "roofline": roof(gf, math_),
                                    "path": "tcgen05 " + math_ + " sweeps storing partials + gradient products"}
        del ws3
    for key, X_, math_ in (("uneven_bwd_tf32", X4, "tf32"), ("uneven_bwd_bf16_tc", X4b, "bf16")):
        ws_ = t3f.gram_groups_prepare(X_, w.gstart, w.tiles4, backward_math=math_)
        dXx = torch.empty(X_.data.numel(), dtype=torch.float32, device=X_.data.device)
        ms = timed(lambda: t3f.gram_groups_backward(X_, w.gstart, ws_, w.devbuf["dG4"], w.tiles4, dcores=dXx,
                                                    math=math_))
        t3f.gram_groups_backward(X_, w.gstart, ws_, w.devbuf["dG4"], w.tiles4, dcores=dXx, math=math_)
        keep[key] = (dXx.clone(), 5e-3 if math_ == "tf32" else 2e-2)
        gf = flops["uneven_bwd"] / (ms * 1e-3) / 1e9
        out[key] = {"ms": round(ms, 4), "gflops": round(gf, 1), "diff_vs_fp32": round(rel(dXx, dX32), 6),
                    "roofline": roof(gf, math_), "workspace_mb": round(ws_.numel() / 1e6, 1),
                    "path": ("F32" if math_ == "tf32" else "BF16") + " cores; tcgen05 " + math_ +
                            " sweeps storing partials + (tile, core, side) gradient items"}
        del ws_, dXx
    # project_sum of config 5 with the U- and V-side sweep contractions on the tensor cores
    X5, Z5, c5 = w.tt("X5"), w.tt("Z5"), w.devbuf["c5"]
    U5, V5 = t3f.orthogonalize(X5)
    P32 = t3f.project_sum(U5, V5, Z5, c5).data.double()
    ms = timed(lambda: t3f.project_sum(U5, V5, Z5, c5, math="tf32"))
    Ptf = t3f.project_sum(U5, V5, Z5, c5, math="tf32")
    keep["psum_tf32"] = (Ptf.data, 5e-3)
    gf = flops["psum"] / (ms * 1e-3) / 1e9
    out["psum_tf32"] = {"ms": round(ms, 4), "gflops": round(gf, 1), "diff_vs_fp32": round(rel(Ptf.data, P32), 6),
                        "roofline": roof(gf, "tf32"),
                        "path": "sweeps: CUDA-core L Z_i factor + tcgen05 TF32 products against U_k / V_k "
                                "(M = 128, N = 32, K = r n), TMA bulk Z staging; FP32 assembly and gauge"}
    for key, X_, ws_, math_, path in (
            ("uneven_bf16_cores", X4b, ws4b, "fp32", "BF16 cores, FP32 CUDA-core arithmetic (grouped work list)"),
            ("uneven_tf32", X4, w.ws4, "tf32", "F32 cores; tcgen05 TF32 tiles, FP32 accumulation"),
            ("uneven_bf16_tc", X4b, ws4b, "bf16", "BF16 cores; tcgen05 BF16 tiles, FP32 accumulation")):
        ms = timed(lambda: t3f.gram_groups(X_, w.gstart, ws_, w.tiles4, math=math_))
        Gx, _ = t3f.gram_groups(X_, w.gstart, ws_, w.tiles4, math=math_)
        keep[key] = (Gx, {"fp32": 2e-2, "tf32": 5e-3, "bf16": 2e-2}[math_])
        gf = flops["uneven"] / (ms * 1e-3) / 1e9
        out[key] = {"ms": round(ms, 4), "gflops": round(gf, 1), "diff_vs_fp32": round(rel(Gx, G4_32), 6),
                    "path": path}
        if math_ != "fp32":
            out[key]["roofline"] = roof(gf, math_)
    return out, keep


def event_time(torch, fn, flush, stream, reps=5):
    """Mean CUDA-event time (ms) of fn on `stream`, L2 flushed (untimed) before each rep."""
    fn()
    torch.cuda.synchronize()
    tot = 0.0
    for _ in range(reps):
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        tot += e0.elapsed_time(e1)
    return tot / reps


def graph_time(torch, fn, flush, stream, reps=10):
    """Mean CUDA-event time (ms) of one replay of fn captured as a CUDA graph, L2 flushed
    (untimed) before each replay: the device time of operations whose host-side call would
    otherwise be longer than their kernels."""
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        fn()
        fn()
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        fn()
    torch.cuda.synchronize()
    tot = 0.0
    for _ in range(reps):
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        g.replay()
        e1.record(stream)
        torch.cuda.synchronize()
        tot += e0.elapsed_time(e1)
    del g
    return tot / reps


def measured_fp64_peak(t3f, torch, dev):
    """FP64 FMA rate of this GPU from the library's FP64 probe (same shape as the FP32 one)."""
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    grid, iters = sms * 4, 400
    t3f.fma_probe(grid, iters, dev, fp64=True)
    torch.cuda.synchronize(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(3):
        flops, _ = t3f.fma_probe(grid, iters, dev, fp64=True)
    e1.record()
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / 3
    return {"tflops": round(flops / (ms * 1e-3) / 1e12, 3), "ms_per_launch": round(ms, 3),
            "how": f"t3f_fma_probe_f64: {grid} CTAs x 256 threads x 8 DFMA chains, CUDA events"}


def measured_fp32_peak(t3f, torch, dev, gpu_index):
    """FP32 FMA rate of this GPU from the library's FMA probe (8 independent chains per
    thread, 4 CTAs of 256 threads per SM), with the SM clock sampled while it runs."""
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    grid, iters = sms * 4, 20000
    t3f.fma_probe(grid, iters, dev)
    torch.cuda.synchronize(dev)
    reps = 8
    with ClockSampler(gpu_index) as clk:
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            flops, _ = t3f.fma_probe(grid, iters, dev)
        e1.record()
        torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / reps
    c = clk.summary()
    return {"tflops": round(flops / (ms * 1e-3) / 1e12, 2), "ms_per_launch": round(ms, 3),
            "sm_mhz": c["sm_mhz"], "sm_max_mhz": c["sm_max_mhz"], "reasons": c["reasons"],
            "derived_at_max_clock": round(FP32_PEAK_TFLOPS, 2),
            "how": f"t3f_fma_probe: {grid} CTAs x 256 threads x 8 FMA chains, CUDA events"}


def next_rows(w, flush, stream, fp32_peak, fp64_peak=None):
    """The tangent-space rows beyond the step (Section 3.2), each timed on its own (CUDA-graph
    replay, L2 flushed before each):
    batched projection of 100 config-5 TTs + the Gram matrix of their tangent vectors (FP32
    CUDA cores and TF32 tensor cores via TMA), the projected matvec P_X(A x_j) at config-3b
    shapes, and the completion loss's linearised Riemannian Hessian applied to its Riemannian
    gradient (config 2)."""
    t3f, torch = w.t3f, w.torch
    out = {}
    hbm = hbm_peak()
    X5 = w.tt("X5")
    U5, V5 = t3f.orthogonalize(X5)
    Z = t3f.TT(w.next_dev["Z100"], [16] * 20, S.tt_ranks(20, 8), 100)
    c100 = w.devbuf["c5"][:100]
    ru5 = t3f.orth_ranks([16] * 20, S.tt_ranks(20, 32))
    rz5 = S.tt_ranks(20, 8)

    def row(name, ms, flops, extra=None):
        gf = flops / (ms * 1e-3) / 1e9
        out[name] = {"ms": round(ms, 4), "gflop": round(flops / 1e9, 4), "gflops": round(gf, 1),
                     "roofline": {"bound": "alu", "achieved": round(gf / 1e3, 3), "peak": fp32_peak, "unit": "TFLOP/s",
                                  "frac": round(gf / 1e3 / fp32_peak, 4), "peak_source": "measured FMA probe"}}
        if extra:
            out[name].update(extra)

    ms = graph_time(torch, lambda: t3f.project(U5, V5, Z, c100), flush, stream)
    row("project_batch", ms, f_project_batch([16] * 20, ru5, rz5, 100))
    dU = t3f.project(U5, V5, Z, c100)
    K = dU.data.numel() // 100
    gflop = 2 * 100 * 100 * K
    ms = graph_time(torch, lambda: t3f.tangent_gram(dU, dU), flush, stream)
    row("tangent_gram_fp32", ms, gflop)
    ms = graph_time(torch, lambda: t3f.tangent_gram(dU, dU, math="tf32"), flush, stream)
    G32 = t3f.tangent_gram(dU, dU).double()
    Gtf = t3f.tangent_gram(dU, dU, math="tf32").double()
    nbytes = dU.data.numel() * 4
    gbs = nbytes / (ms * 1e-3) / 1e9
    out["tangent_gram_tf32"] = {
        "ms": round(ms, 4), "gflops": round(gflop / (ms * 1e-3) / 1e9, 1),
        "diff_vs_fp32": round(float((Gtf - G32).norm() / G32.norm()), 6),
        "path": "TMA (2D, 128-byte swizzle) + tcgen05 kind::tf32, FP32 accumulation in TMEM, split-K",
        "roofline": {"bound": "hbm", "achieved": round(gbs, 1), "peak": hbm, "unit": "GB/s", "frac": round(gbs / hbm, 4),
                     "traffic": None, "bytes": "coordinates read once (self Gram: one operand per diagonal tile)"}}
    # projected matvec at config-3b shapes: A = the first TT-matrix, 100 TT-vectors, X rank 10
    A1 = t3f.TT(w.next_dev["A1"], [4] * 10, S.tt_ranks(10, 10), 1, [4] * 10)
    xv = w.tt("xv")
    Xp = t3f.TT(w.next_dev["Xp"], [4] * 10, S.tt_ranks(10, 10), 1)
    Up, Vp = t3f.orthogonalize(Xp)
    rxp = t3f.orth_ranks([4] * 10, S.tt_ranks(10, 10))
    ms = graph_time(torch, lambda: t3f.project_matvec(Up, Vp, A1, xv), flush, stream)
    row("project_matvec", ms, f_project_matvec([4] * 10, [4] * 10, rxp, S.tt_ranks(10, 10), S.tt_ranks(10, 10), 100))
    # linearised Riemannian Hessian of the completion loss along its Riemannian gradient
    X2 = w.tt("X2")
    U2, V2 = t3f.orthogonalize(X2)
    idx, y = w.devbuf["idx"], w.devbuf["y"]
    g2, _ = t3f.gather_backward(None, idx, y=y, riemannian=True, U=U2, V=V2)
    ms = graph_time(torch, lambda: t3f.completion_hvp(U2, V2, idx, g2), flush, stream)
    ru2 = t3f.orth_ranks([10] * 10, S.tt_ranks(10, 8))
    row("completion_hvp", ms, f_hvp(ru2, [10] * 10, idx.shape[1]))
    # TT rounding (FP64 TT-SVD) of the 100 rank-100 matvec products of config 3b to rank 10
    C = t3f.matvec(w.tt("Am"), xv)
    ms = event_time(torch, lambda: t3f.round_tt(C, 10), flush, stream, reps=3)
    fl = 100 * f_round([4] * 10, C.ranks, 10)
    gf = fl / (ms * 1e-3) / 1e9
    out["round"] = {"ms": round(ms, 4), "gflop": round(fl / 1e9, 4), "gflops": round(gf, 2),
                    "what": "100 TT-vectors of rank 100 (d=10, n=4) rounded to rank 10, FP64",
                    "roofline": {"bound": "alu", "achieved": round(gf / 1e3, 4),
                                 "peak": fp64_peak, "unit": "TFLOP/s (FP64)",
                                 "frac": round(gf / 1e3 / fp64_peak, 4) if fp64_peak else None,
                                 "peak_source": "measured FP64 FMA probe",
                                 "flops": "QR, Gram, singular-vector and S V^T products; Jacobi sweeps not counted"}}
    return out


def hbm_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"])
    except (OSError, ValueError, KeyError):
        return 6800.0


def bucket_comparator(w):
    """The single-shape FP32 comparator of the uneven batch without cubic padding: within each
    group the objects are split by rank bucket (<= 8, 16, 32, 64), each bucket padded to its
    own largest rank, and every bucket pair runs as one uniform Gram + adjoint launch pair
    (per-group sequential launches, no work queue, no graph)."""
    t3f, torch = w.t3f, w.torch
    dims, modes, ranks, offs = w.r4meta
    rg = t3f.RaggedTT(w.host["X4"], dims, modes, ranks, offs)
    launches = []
    for g in range(len(w.gstart) - 1):
        objs = list(range(w.gstart[g], w.gstart[g + 1]))
        d, n = dims[objs[0]], modes[objs[0]]
        buckets = {}
        for o in objs:
            r = max(ranks[o][1:-1], default=1)
            b = 0 if r <= 8 else 1 if r <= 16 else 2 if r <= 32 else 3
            buckets.setdefault(b, []).append(o)
        tts = {}
        for b, os_ in buckets.items():
            R = max(max(ranks[o][1:-1], default=1) for o in os_)
            rk = [1] + [R] * (d - 1) + [1]
            cores = []
            for k in range(d):
                blk = np.zeros((len(os_), rk[k], n[k], rk[k + 1]), np.float32)
                for j, o in enumerate(os_):
                    cc = rg.object_cores(o)[k].numpy()
                    blk[j, :cc.shape[0], :, :cc.shape[2]] = cc
                cores.append(blk)
            tts[b] = t3f.TT.from_cores(cores, device=w.dev)
        keys = sorted(tts)
        for i, p in enumerate(keys):
            for q in keys[i:]:
                dG = torch.randn(tts[p].batch, tts[q].batch, device=w.dev)
                launches.append((tts[p], tts[q], dG))
    return launches


# ---------------------------------------------------------------------------------------
# clocks
# ---------------------------------------------------------------------------------------

class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            p = [x.strip() for x in l.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx = float(p[2])
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------------------
# CPU oracle (baseline and the reference arm)
# ---------------------------------------------------------------------------------------

def oracle_sample(frac: float, seed: int = 0):
    """Run the FP64 oracle on a bounded sample of the step's workload.

    Returns (algorithmic FLOPs of the sample, seconds, description)."""
    import oracle as O
    t_start = time.perf_counter()
    flops = 0.0
    obj = lambda cs: [[np.asarray(c[i], np.float64) for c in cs] for i in range(cs[0].shape[0])]
    # completion on a prefix of the tuples
    c2 = S.config2(N=max(1000, int(1_000_000 * frac)), seed=2 + seed)
    X = obj([np.asarray(c, np.float32) for c in c2.X])[0]
    T = obj([np.asarray(c, np.float32) for c in c2.T])[0]
    y = O.gather(T, c2.idx) + c2.noise
    N = c2.idx.shape[1]
    t0 = time.perf_counter()
    O.completion_loss_grad(X, c2.idx, y)
    U, V, ru = O.orthogonalize(X)
    O.riemannian_grad_completion(U, V, c2.idx, y)
    r2 = S.tt_ranks(10, 8)
    flops += N * f_completion(r2) + f_orth([10] * 10, r2) + N * f_completion(ru) + f_gauge([10] * 10, ru)
    tcomp = time.perf_counter() - t0
    # gram on a subset of rows
    nA = max(1, int(round(100 * frac)))
    c3 = S.config3a(bA=nA, seed=3 + seed)
    A, B = obj(c3.A), obj(c3.B)
    r10, n10 = S.tt_ranks(10, 10), [10] * 10
    G = O.gram(A, B)
    O.gram_vjp(A, B, np.ones_like(G))
    for a in A:
        O.norm(a)
    flops += nA * 100 * (f_left_sweep(n10, r10, r10) + f_gram_bwd(n10, r10, r10)) + nA * f_left_sweep(n10, r10, r10)
    # matvec on a subset of pairs
    nm = max(1, int(round(100 * frac)))
    c3b = S.config3b(batch=nm, seed=4 + seed)
    Am, xv = obj(c3b.A), obj(c3b.x)
    for a, x in zip(Am, xv):
        Cm = O.matvec(a, x)
        O.matvec_vjp(a, x, Cm)
    flops += 3 * nm * f_matvec([4] * 10, [4] * 10, r10, r10)
    # project_sum on a subset of the batch
    nz = max(1, int(round(1000 * frac)))
    c5 = S.config5(batch=nz, seed=6 + seed)
    X5 = obj(c5.X)[0]
    Z = obj(c5.Z)
    U5, V5, ru5 = O.orthogonalize(X5)
    Sg = O.project_sum(U5, V5, Z, c5.c)
    O.project_sum_vjp(U5, V5, Z, c5.c, Sg)
    n16, rz5 = [16] * 20, S.tt_ranks(20, 8)
    flops += f_orth(n16, S.tt_ranks(20, 32)) + f_psum_fwd(n16, ru5, rz5, nz) + f_psum_bwd(n16, ru5, rz5, nz)
    secs = time.perf_counter() - t_start
    desc = (f"FP64 NumPy oracle, 1 thread: completion+rgrad on {N} tuples, gram+bwd {nA}x100 pairs, "
            f"matvec+bwd {nm} pairs, orth+project_sum+bwd of {nz} TTs (fraction {frac:g} of the step)")
    return flops, secs, desc, tcomp


def oracle_errors(w, out, extra=None):
    """Error of every output of one step against the FP64 oracle on the same (FP32-rounded)
    inputs, on sampled objects / rows / pairs the oracle computes one by one (the loss, the
    completion gradient, the Riemannian gradient and project_sum in full). Each entry gives
    the max and median over its samples of the normwise relative error (Gram matrices of one
    collection: diagonal and off-diagonal entries separately) and the stated tolerance."""
    import oracle as O
    t3f = w.t3f
    t0 = time.perf_counter()
    res = {}

    def rel(a, b):
        a = np.concatenate([np.asarray(x, np.float64).ravel() for x in a]) if isinstance(a, list) else np.ravel(a)
        b = np.concatenate([np.asarray(x, np.float64).ravel() for x in b]) if isinstance(b, list) else np.ravel(b)
        nb = np.linalg.norm(b)
        return float(np.linalg.norm(a - b) / nb) if nb > 0 else float(np.linalg.norm(a - b))

    def rec(name, errs, tol):
        res[name] = {"max": float(max(errs)), "median": float(np.median(errs)), "samples": len(errs), "tol": tol}

    def objs(key, data=None, ranks=None):
        n, r, b, m = w.meta[key]
        r = ranks or r
        src = w.host[key] if data is None else data.detach().cpu()
        tt = t3f.TT(src.double(), n, r, b, m)
        cores = [c.numpy() for c in tt.cores()]
        return [[c[i] for c in cores] for i in range(b)]

    # completion loss and gradient, Riemannian gradient (all 10^6 tuples)
    X2 = objs("X2")[0]
    idx = w.host["idx"].numpy()
    y = w.host["y"].double().numpy()
    L, g = O.completion_loss_grad(X2, idx, y)
    rec("completion.loss", [abs(float(out["loss"].item()) - L) / abs(L)], 1e-5)
    rec("completion.dX", [rel(objs("X2", out["dX"])[0], g)], 1e-5)
    U2, V2, ru2 = O.orthogonalize(X2)
    _, dU2 = O.riemannian_grad_completion(U2, V2, idx, y)
    rec("rgrad.dU", [rel(objs("X2", out["dU2"], ranks=ru2)[0], dU2)], 1e-5)
    # Gram, adjoint, norms (sampled rows and objects)
    A, B = objs("A3"), objs("B3")
    dG = w.host["dG"].double().numpy()
    G = out["G"].double().cpu().numpy()
    rec("gram.G", [rel(G[a], [O.dot(A[a], Bb) for Bb in B]) for a in (0, 57, 99)], 1e-5)
    dA, dB = objs("A3", out["dA"]), objs("B3", out["dB"])
    rec("gram_bwd.dA", [rel(dA[a], O.gram_vjp([A[a]], B, dG[a:a + 1])[0][0]) for a in (0, 99)], 1e-5)
    rec("gram_bwd.dB", [rel(dB[b], O.gram_vjp(A, [B[b]], dG[:, b:b + 1])[1][0]) for b in (3,)], 1e-5)
    nrm = out["norm"].double().cpu().numpy()
    rec("norm", [abs(nrm[a] - O.norm(A[a])) / O.norm(A[a]) for a in range(0, 100, 11)], 1e-5)
    # matvec and its adjoint (sampled pairs)
    Am, xv = objs("Am"), objs("xv")
    C = w.t3f.TT(out["_bulk"][0].data.detach().cpu().double(), [4] * 10,
                 [a * b for a, b in zip(S.tt_ranks(10, 10), S.tt_ranks(10, 10))], 100)
    Cc = [c.numpy() for c in C.cores()]
    rec("matvec.C", [rel([c[p] for c in Cc], O.matvec(Am[p], xv[p])) for p in (0, 99)], 1e-5)
    dC = objs("dC")
    dAm, dxv = objs("Am", out["dAm"]), objs("xv", out["dxv"])
    ea, ex = [], []
    for p in (0, 99):
        ra, rx = O.matvec_vjp(Am[p], xv[p], dC[p])
        ea.append(rel(dAm[p], ra))
        ex.append(rel(dxv[p], rx))
    rec("matvec_bwd.dA", ea, 1e-5)
    rec("matvec_bwd.dx", ex, 1e-5)
    # project_sum (all 1000 TTs) and its adjoint (sampled TTs, the step's own cotangent)
    X5 = objs("X5")[0]
    Z5 = objs("Z5")
    c5 = w.host["c5"].double().numpy()
    U5, V5, ru5 = O.orthogonalize(X5)
    dU5 = objs("X5", out["dU5"], ranks=ru5)[0]
    psum_ref = O.project_sum(U5, V5, Z5, c5)
    rec("psum.dU", [rel(dU5, psum_ref)], 1e-5)
    if extra and "psum_tf32" in extra:
        rec("psum_tf32.dU", [rel(objs("X5", extra["psum_tf32"][0], ranks=ru5)[0], psum_ref)], extra["psum_tf32"][1])
    dZ = w.t3f.TT(out["_bulk"][1].data.detach().cpu().double(), [16] * 20, S.tt_ranks(20, 8), 1000)
    dZc = [c.numpy() for c in dZ.cores()]
    dc = out["dc"].double().cpu().numpy()
    ez, ec = [], []
    for j in (0, 500, 999):
        rz, rc = O.project_sum_vjp(U5, V5, [Z5[j]], [c5[j]], dU5)
        ez.append(rel([c[j] for c in dZc], rz[0]))
        ec.append(abs(dc[j] - rc[0]) / abs(rc[0]))
    rec("psum_bwd.dZ", ez, 1e-5)
    rec("psum_bwd.dc", ec, 1e-5)
    # uneven batch: sampled pairs of every group, first norm of every group, one adjoint object
    dims, modes, ranks, offs = w.r4meta
    rg = t3f.RaggedTT(w.host["X4"], dims, modes, ranks, offs)
    ob = lambda o, src=rg: [c.double().numpy() for c in src.object_cores(o)]
    G4 = out["G4"].double().cpu().numpy()
    n4 = out["n4"].double().cpu().numpy()
    gd = t3f.RaggedTT(out["dX4"].detach().cpu(), dims, modes, ranks, offs)
    dG4 = w.host["dG4"].double().numpy()
    rng = np.random.default_rng(77)
    ediag, eoff, enorm, ebwd = [], [], [], []
    off = 0
    for gi in range(len(w.gstart) - 1):
        g0, Sg = w.gstart[gi], w.gstart[gi + 1] - w.gstart[gi]
        pairs = [(0, 0), (Sg - 1, Sg - 1)]
        while len(pairs) < 12:
            a, b = (int(v) for v in rng.integers(0, Sg, 2))
            if a != b:
                pairs.append((a, b))
        got = np.array([G4[off + a * Sg + b] for a, b in pairs])
        want = np.array([O.dot(ob(g0 + a), ob(g0 + b)) for a, b in pairs])
        ediag.append(rel(got[:2], want[:2]))
        eoff.append(rel(got[2:], want[2:]))
        enorm.append(abs(n4[g0] - O.norm(ob(g0))) / O.norm(ob(g0)))
        a = int(rng.integers(0, Sg))
        M = dG4[off:off + Sg * Sg].reshape(Sg, Sg)
        grp = [ob(g0 + j) for j in range(Sg)]
        ref = O.gram_vjp([grp[a]], grp, (M[a, :] + M[:, a])[None, :])[0][0]
        ebwd.append(rel(ob(g0 + a, gd), ref))
        off += Sg * Sg
    rec("uneven.G.diag", ediag, 1e-5)
    rec("uneven.G.offdiag", eoff, 1e-5)
    rec("uneven.norms", enorm, 1e-5)
    rec("uneven_bwd.dX", ebwd, 1e-5)
    for key, (G_, tol) in (extra or {}).items():
        if key == "psum_tf32":
            continue
        if key.startswith("gram_bwd_"):
            dAo, dBo = objs("A3", G_[0].data), objs("B3", G_[1].data)
            rec(key + ".dA", [rel(dAo[a], O.gram_vjp([A[a]], B, dG[a:a + 1])[0][0]) for a in (0, 99)], tol)
            rec(key + ".dB", [rel(dBo[b], O.gram_vjp(A, [B[b]], dG[:, b:b + 1])[1][0]) for b in (3,)], tol)
        elif key.startswith("uneven_bwd_"):
            rg_x = rg
            if "bf16" in key:
                import torch as _t
                rg_x = t3f.RaggedTT(w.host["X4"].to(_t.bfloat16).to(_t.float64), dims, modes, ranks, offs)
            obx = lambda o: [c.double().numpy() for c in rg_x.object_cores(o)]
            gx = t3f.RaggedTT(G_.detach().cpu(), dims, modes, ranks, offs)
            eb, off = [], 0
            rng_b = np.random.default_rng(78)
            for gi in range(len(w.gstart) - 1):
                g0, Sg = w.gstart[gi], w.gstart[gi + 1] - w.gstart[gi]
                a = int(rng_b.integers(0, Sg))
                M = dG4[off:off + Sg * Sg].reshape(Sg, Sg)
                grp = [obx(g0 + j) for j in range(Sg)]
                ref = O.gram_vjp([grp[a]], grp, (M[a, :] + M[:, a])[None, :])[0][0]
                eb.append(rel([c.double().numpy() for c in gx.object_cores(g0 + a)], ref))
                off += Sg * Sg
            rec(key + ".dX", eb, tol)
        elif key.startswith("gram_"):
            Gx = G_.double().cpu().numpy()
            rec(key + ".G", [rel(Gx[a], [O.dot(A[a], Bb) for Bb in B]) for a in (0, 57, 99)], tol)
        elif key.startswith("uneven_"):
            Gx = G_.double().cpu().numpy()
            rg_x = rg
            if "bf16" in key:
                import torch as _t
                rg_x = t3f.RaggedTT(w.host["X4"].to(_t.bfloat16).to(_t.float64), dims, modes, ranks, offs)
            obx = lambda o: [c.double().numpy() for c in rg_x.object_cores(o)]
            ed, eo, off = [], [], 0
            for gi in range(len(w.gstart) - 1):
                g0, Sg = w.gstart[gi], w.gstart[gi + 1] - w.gstart[gi]
                pairs = [(0, 0), (Sg - 1, Sg - 1), (0, Sg - 1), (1, 2), (3, Sg - 2), (Sg // 2, 5)]
                got = np.array([Gx[off + a * Sg + b] for a, b in pairs])
                want = np.array([O.dot(obx(g0 + a), obx(g0 + b)) for a, b in pairs])
                ed.append(rel(got[:2], want[:2]))
                eo.append(rel(got[2:], want[2:]))
                off += Sg * Sg
            rec(key + ".G.diag", ed, tol)
            rec(key + ".G.offdiag", eo, tol)
    res["_seconds"] = round(time.perf_counter() - t0, 2)
    return res


def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    total_steps = args.steps + args.warmup
    budget = min(8.0, 150.0 / max(1, total_steps))     # seconds per step
    f0, s0, _, _ = oracle_sample(0.01)
    frac = max(0.002, min(0.2, 0.01 * budget / max(s0, 1e-3)))
    for i in range(args.warmup):
        oracle_sample(frac, seed=0)
    rates, secs, flops_tot, desc = [], 0.0, 0.0, ""
    for i in range(args.steps):
        f, s, desc, _ = oracle_sample(frac, seed=0)
        rates.append(f / s)
        secs += s
        flops_tot += f
    value = flops_tot / secs / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "GFLOP/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": secs / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample_fraction": frac},
        "cpu_baseline": {"value": value, "unit": "GFLOP/s", "cores": 1, "kind": "oracle", "sample": desc},
        "e2e": {"value": value, "unit": "GFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------------------

def gpu_arm(args):
    import torch
    import torch.distributed as dist

    import paper_1801_01928_gb300 as t3f

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    t3f.load()

    def barrier():
        if world > 1:
            dist.barrier()

    w = Workload(t3f, torch, dev, seed_offset=rank)
    w.prepare_uneven()
    flops = w.flops()
    step_flops = sum(flops.values())
    stream = torch.cuda.current_stream(dev)
    side = torch.cuda.Stream(dev)
    copy_stream = torch.cuda.Stream(dev)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)

    for _ in range(args.warmup):
        run_step(w, stream=stream, side=side)
        run_step(w, stream=stream)
    torch.cuda.synchronize(dev)

    # device-timed region: K steps (orthogonalisation chain on the side stream), L2 flushed
    # (untimed) before each
    step_ev = []
    launches0 = t3f.launch_count()
    barrier()
    torch.cuda.synchronize(dev)
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            run_step(w, None, stream, side)
            e1.record(stream)
            step_ev.append((e0, e1))
        torch.cuda.synchronize(dev)
        barrier()
    # library launches issued in the timed steps, plus the kernels the graph replays launch
    launches = t3f.launch_count() - launches0 + args.steps * w.graph_kernels
    step_ms = [a.elapsed_time(b) for a, b in step_ev]
    dev_ms = sum(step_ms) / args.steps

    # the same K steps with every operation in order on one stream (no overlap)
    seq_ev = []
    torch.cuda.synchronize(dev)
    for _ in range(args.steps):
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        run_step(w, None, stream)
        e1.record(stream)
        seq_ev.append((e0, e1))
    torch.cuda.synchronize(dev)
    seq_ms = sum(a.elapsed_time(b) for a, b in seq_ev) / args.steps
    # per-operation device times (each operation replayed as its own CUDA graph)
    op_ms = op_graph_times(w, flush, stream)

    # end-to-end: pinned host inputs copied in, results read back, every step. Each result is
    # copied into pinned host memory on its own stream as soon as the operation writing it has
    # been issued; the step ends when the last copy has landed. The pinned result buffers are
    # sized by one untimed step.
    d2h_stream = torch.cuda.Stream(dev)
    copy_stream.wait_stream(stream)
    out0 = run_step(w, None, stream, side, w.upload_async(copy_stream))
    host_out = {k: torch.empty(v.shape, dtype=v.dtype).pin_memory() for k, v in out0.items() if k != "_bulk"}
    del out0
    d2h = sum(v.numel() * v.element_size() for v in host_out.values())

    def emit(name, t, st):
        ev = torch.cuda.Event()
        ev.record(st)
        d2h_stream.wait_event(ev)
        t.record_stream(d2h_stream)
        with torch.cuda.stream(d2h_stream):
            host_out[name].copy_(t, non_blocking=True)

    e2e_ev = []
    barrier()
    torch.cuda.synchronize(dev)
    for _ in range(args.steps):
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        copy_stream.wait_stream(stream)
        d2h_stream.wait_stream(stream)
        ready = w.upload_async(copy_stream)
        run_step(w, None, stream, side, ready, emit)
        stream.wait_stream(d2h_stream)
        e1.record(stream)
        e2e_ev.append((e0, e1))
    torch.cuda.synchronize(dev)
    barrier()
    e2e_ms = sum(a.elapsed_time(b) for a, b in e2e_ev) / args.steps

    dev_ms, e2e_ms, value, e2e_value = combine_ranks(dev_ms, e2e_ms, world, step_flops, dev)

    # FP32 FMA peak measured on this GPU (the ALU roofline's denominator)
    fp32 = measured_fp32_peak(t3f, torch, dev, local)
    peak32 = fp32["tflops"]
    # dominant operation and its roofline (FP32 CUDA-core pipe)
    dom = max(op_ms, key=op_ms.get)
    ach = flops[dom] / (op_ms[dom] * 1e-3) / 1e12
    per_op = {k: {"ms": round(op_ms[k], 4), "gflop": round(flops[k] / 1e9, 4),
                  "gflops": round(flops[k] / (op_ms[k] * 1e-3) / 1e9, 1),
                  "frac_fp32": round(flops[k] / (op_ms[k] * 1e-3) / 1e12 / peak32, 4)}
              for k in op_ms}
    traffic = None
    prof = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(prof):
        try:
            tj = json.load(open(prof))
            traffic = tj.get(dom, {}).get("dram_bytes")
        except (OSError, ValueError):
            traffic = None
    line = {
        "metric": METRIC, "value": round(value, 2), "unit": "GFLOP/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dev_ms, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "l2": "flushed before every timed step (256 MiB write)",
                   "parallelism": f"replicas{world}", "step_gflop": round(step_flops / 1e9, 3),
                   "streams": "2: orthogonalisation chain (orth2, rgrad, orth5, project_sum, adjoint) "
                              "on a side stream, concurrent with the rest",
                   "ms_per_step_one_stream": round(seq_ms, 4),
                   "uneven_tiles": list(w.tiles4)},
        "roofline": {"bound": "alu", "kernel_op": dom, "achieved": round(ach, 3),
                     "peak": peak32, "unit": "TFLOP/s",
                     "frac": round(ach / peak32, 4), "traffic": traffic,
                     "peak_source": "measured: FP32 FMA probe on this GPU (fp32_peak)",
                     "frac_of_derived": round(ach / FP32_PEAK_TFLOPS, 4)},
        "fp32_peak": fp32,
        "e2e": {"value": round(e2e_value, 2), "unit": "GFLOP/s", "h2d_bytes_per_step": w.h2d_bytes,
                "d2h_bytes_per_step": d2h, "ms_per_step": round(e2e_ms, 4)},
        "gpu_launches": launches,
        "clocks": clk.summary(),
        "ops": per_op,
    }
    # single-shape FP32 comparator for the uneven batch (outside the timed step)
    if not args.no_comparator:
        groups = bucket_comparator(w)
        def plain():
            for A, B, dG in groups:
                t3f.gram(A, B)
                t3f.gram_backward(A, B, dG)
        plain()
        torch.cuda.synchronize(dev)
        reps = 2
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            plain()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        pm = e0.elapsed_time(e1) / reps
        um = op_ms["uneven"] + op_ms["uneven_bwd"]
        uf = flops["uneven"] + flops["uneven_bwd"]
        line["comparators"] = {"uneven_plain_fp32": {
            "what": "per group and rank-bucket pair (<= 8, 16, 32, 64) one uniform FP32 Gram + adjoint "
                    "launch pair, each bucket padded to its own largest rank; no work queue, no graph",
            "launches": 2 * len(groups),
            "ms": round(pm, 3), "gflops_same_work": round(uf / (pm * 1e-3) / 1e9, 1),
            "uneven_ms": round(um, 3), "uneven_speedup": round(pm / um, 2)}}
        del groups
    # reduced-precision forms of the same work (outside the timed step; FP32 step above)
    line["reduced_precision"], rp_out = reduced_precision(w, flops, flush, stream)
    # tangent-space rows measured beside the step
    fp64 = measured_fp64_peak(t3f, torch, dev)
    line["fp64_peak"] = fp64
    line["next_rows"] = next_rows(w, flush, stream, peak32, fp64["tflops"])
    # error of every output against the FP64 oracle (one step's outputs, sampled)
    if rank == 0 and not args.no_oracle_check:
        out = run_step(w, None, stream, side)
        torch.cuda.synchronize(dev)
        line["oracle_err"] = oracle_errors(w, out, rp_out)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        f, s, desc, _ = oracle_sample(args.cpu_fraction)
        line["cpu_baseline"] = {"value": round(f / s / 1e9, 4), "unit": "GFLOP/s", "cores": 1,
                                "kind": "oracle", "sample": desc, "seconds": round(s, 2)}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--cpu-fraction", type=float, default=0.15)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-comparator", action="store_true")
    ap.add_argument("--no-oracle-check", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return reference_arm(args)
    return gpu_arm(args)


if __name__ == "__main__":
    sys.exit(main())
