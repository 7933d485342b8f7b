"""ctypes binding of libt3f (argument marshalling only).

Every function here validates nothing beyond Python types, allocates the outputs and the
workspace with torch on the operands' device, passes raw device pointers and the current
CUDA stream to the C ABI declared in include/t3f.h, and raises T3FError on a non-zero
status. All arithmetic runs in the library's CUDA kernels; there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libt3f.so")

# t3f_dtype / t3f_math / t3f_op values (include/t3f.h)
F32, F64, BF16 = 0, 1, 2
MATH = {"fp32": 0, "tf32": 1, "bf16": 2}
OP = dict(gram=1, gram_bwd=2, norm=3, gather=4, gather_bwd=5, rgather_bwd=6, matvec=7,
          matvec_bwd=8, orth=9, psum=10, psum_bwd=11, project=12, tangent_gram=13, completion_hvp=14,
          round=15, gram_bwd_tc=16)
_TORCH_DTYPE = {F32: torch.float32, F64: torch.float64, BF16: torch.bfloat16}
_CODE = {v: k for k, v in _TORCH_DTYPE.items()}


class T3FError(RuntimeError):
    def __init__(self, status: int, where: str):
        msg = _lib().t3f_status_string(status).decode() if _LIB is not None else str(status)
        super().__init__(f"{where}: {msg}")
        self.status = status


class _Desc(ctypes.Structure):
    _fields_ = [("batch", ctypes.c_int32), ("d", ctypes.c_int32),
                ("m", ctypes.POINTER(ctypes.c_int32)), ("n", ctypes.POINTER(ctypes.c_int32)),
                ("ranks", ctypes.POINTER(ctypes.c_int32)), ("cores", ctypes.c_void_p),
                ("dtype", ctypes.c_int32)]


_LIB: Optional[ctypes.CDLL] = None
_P = ctypes.POINTER(_Desc)
_VP = ctypes.c_void_p
_SZ = ctypes.c_size_t

_SIGS = {
    "t3f_status_string": (ctypes.c_char_p, [ctypes.c_int32]),
    "t3f_version": (ctypes.c_int32, []),
    "t3f_launch_count": (ctypes.c_int64, []),
    "t3f_packed_size": (ctypes.c_int64, [_P]),
    "t3f_workspace_size": (ctypes.c_size_t, [ctypes.c_int32, _P, _P, ctypes.c_int64]),
    "t3f_gram": (ctypes.c_int32, [_P, _P, _VP, ctypes.c_int32, _VP, _SZ, _VP]),
    "t3f_norm": (ctypes.c_int32, [_P, _VP, _VP, _SZ, _VP]),
    "t3f_gram_backward": (ctypes.c_int32, [_P, _P, _VP, _P, _P, ctypes.c_int32, _VP, _SZ, _VP]),
    "t3f_gather": (ctypes.c_int32, [_P, _VP, ctypes.c_int64, _VP, _VP, _VP, _VP, _SZ, _VP]),
    "t3f_gather_noalloc": (ctypes.c_int32, [_P, _VP, ctypes.c_int64, _VP, _VP, _VP, _VP]),
    "t3f_gather_noalloc_status": (ctypes.c_int32, [_VP]),
    "t3f_gather_backward": (ctypes.c_int32, [_P, _VP, ctypes.c_int64, _VP, _VP, _VP, _P,
                                             ctypes.c_int32, _P, _P, _VP, _SZ, _VP]),
    "t3f_matvec": (ctypes.c_int32, [_P, _P, _P, _VP, _SZ, _VP]),
    "t3f_matvec_backward": (ctypes.c_int32, [_P, _P, _P, _P, _P, _VP, _SZ, _VP]),
    "t3f_orth_ranks": (ctypes.c_int32, [ctypes.c_int32, ctypes.POINTER(ctypes.c_int32),
                                        ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)]),
    "t3f_orthogonalize": (ctypes.c_int32, [_P, _P, _P, _VP, _SZ, _VP]),
    "t3f_project_sum": (ctypes.c_int32, [_P, _P, _P, _VP, _P, ctypes.c_int32, _VP, _SZ, _VP]),
    "t3f_project_sum_backward": (ctypes.c_int32, [_P, _P, _P, _VP, _P, _P, _VP, _VP, _SZ, _VP]),
    "t3f_device_status": (ctypes.c_int32, [_VP, _VP]),
    "t3f_project": (ctypes.c_int32, [_P, _P, _P, _VP, _P, _VP, _SZ, _VP]),
    "t3f_tangent_gram": (ctypes.c_int32, [_P, _P, _VP, ctypes.c_int32, _VP, _SZ, _VP]),
    "t3f_project_matvec_workspace_size": (ctypes.c_size_t, [_P, _P, _P]),
    "t3f_project_matvec": (ctypes.c_int32, [_P, _P, _P, _P, _P, _VP, _SZ, _VP]),
    "t3f_completion_hvp": (ctypes.c_int32, [_P, _P, _VP, ctypes.c_int64, _P, _P, _VP, _SZ, _VP]),
    "t3f_fma_probe": (ctypes.c_int32, [ctypes.c_int32, ctypes.c_int64, _VP, _VP]),
    "t3f_fma_probe_flops": (ctypes.c_double, [ctypes.c_int32, ctypes.c_int64]),
    "t3f_fma_probe_f64": (ctypes.c_int32, [ctypes.c_int32, ctypes.c_int64, _VP, _VP]),
    "t3f_round_ranks": (ctypes.c_int32, [ctypes.c_int32, ctypes.POINTER(ctypes.c_int32),
                                         ctypes.POINTER(ctypes.c_int32), ctypes.c_int32,
                                         ctypes.POINTER(ctypes.c_int32)]),
    "t3f_round": (ctypes.c_int32, [_P, ctypes.c_int32, _P, _VP, _SZ, _VP]),
}
EXPORTS = tuple(_SIGS)


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libt3f.so (built in-tree); raises if it is missing -- there is no fallback."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(path):
        raise RuntimeError(f"libt3f.so not found at {path}; build it with "
                           "`python -m paper_1801_01928_gb300.build`")
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _LIB = lib
    return lib


def _lib() -> ctypes.CDLL:
    return _LIB if _LIB is not None else load()


def _check(status: int, where: str):
    if status != 0:
        raise T3FError(status, where)


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(device: torch.device):
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def _i32(vals: Sequence[int]):
    return (ctypes.c_int32 * len(vals))(*[int(v) for v in vals])


class TT:
    """A batch of TT-vectors (m is None) or TT-matrices in the library's packed layout.

    Core k of all objects is one contiguous block [batch][r_{k-1}][m_k][n_k][r_k]; the
    blocks follow each other in one flat device tensor ``data``."""

    def __init__(self, data: torch.Tensor, n, ranks, batch: int, m=None):
        self.n = [int(v) for v in n]
        self.ranks = [int(v) for v in ranks]
        self.m = None if m is None else [int(v) for v in m]
        self.batch = int(batch)
        self.d = len(self.n)
        if len(self.ranks) != self.d + 1:
            raise ValueError("ranks must have d+1 entries")
        if data.dim() != 1 or data.numel() != self.numel(self.n, self.ranks, self.batch, self.m):
            raise ValueError("data does not match the packed size")
        self.data = data
        self._keep = None

    @staticmethod
    def core_numel(n, ranks, m, k):
        return ranks[k] * (1 if m is None else m[k]) * n[k] * ranks[k + 1]

    @classmethod
    def numel(cls, n, ranks, batch, m=None):
        return batch * sum(cls.core_numel(n, ranks, m, k) for k in range(len(n)))

    @classmethod
    def empty(cls, n, ranks, batch, m=None, dtype=torch.float32, device="cuda"):
        return cls(torch.empty(cls.numel(n, ranks, batch, m), dtype=dtype, device=device), n, ranks, batch, m)

    @classmethod
    def zeros(cls, n, ranks, batch, m=None, dtype=torch.float32, device="cuda"):
        return cls(torch.zeros(cls.numel(n, ranks, batch, m), dtype=dtype, device=device), n, ranks, batch, m)

    def empty_like(self, dtype=None, ranks=None):
        return TT.empty(self.n, ranks or self.ranks, self.batch, self.m, dtype or self.data.dtype, self.data.device)

    @classmethod
    def from_cores(cls, cores, dtype=torch.float32, device="cuda"):
        """cores: list of arrays/tensors shaped (batch, r0, [m], n, r1)."""
        ts = [torch.as_tensor(c) for c in cores]
        batch = ts[0].shape[0]
        is_matrix = ts[0].dim() == 5
        n = [t.shape[-2] for t in ts]
        m = [t.shape[2] for t in ts] if is_matrix else None
        ranks = [ts[0].shape[1]] + [t.shape[-1] for t in ts]
        flat = torch.cat([t.reshape(-1) for t in ts]).to(dtype=dtype)
        return cls(flat.to(device), n, ranks, batch, m)

    def core(self, k: int) -> torch.Tensor:
        off = self.batch * sum(self.core_numel(self.n, self.ranks, self.m, j) for j in range(k))
        sz = self.batch * self.core_numel(self.n, self.ranks, self.m, k)
        shape = [self.batch, self.ranks[k]] + ([] if self.m is None else [self.m[k]]) + [self.n[k], self.ranks[k + 1]]
        return self.data[off:off + sz].view(shape)

    def cores(self):
        return [self.core(k) for k in range(self.d)]

    @property
    def dtype_code(self) -> int:
        return _CODE[self.data.dtype]

    def desc(self) -> _Desc:
        n, r = _i32(self.n), _i32(self.ranks)
        m = _i32(self.m) if self.m is not None else None
        self._keep = (n, r, m)
        return _Desc(self.batch, self.d, m if m is not None else None, n, r,
                     ctypes.c_void_p(self.data.data_ptr()), self.dtype_code)


def _ref(t: Optional[TT]):
    return None if t is None else ctypes.byref(t.desc())


def _ws(op: str, a: TT, b: Optional[TT], n_items: int, device) -> torch.Tensor:
    nbytes = _lib().t3f_workspace_size(OP[op], ctypes.byref(a.desc()), _ref(b), int(n_items))
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)


def workspace(op: str, a: TT, b: Optional[TT] = None, n_items: int = 0) -> torch.Tensor:
    """A device workspace of t3f_workspace_size(op) bytes (op: a key of OP)."""
    return _ws(op, a, b, n_items, a.data.device)


# ---------------------------------------------------------------------------------------
# Operations (names follow include/t3f.h)
# ---------------------------------------------------------------------------------------

def gram(A: TT, B: TT, math: str = "fp32") -> torch.Tensor:
    dev = A.data.device
    G = torch.empty(A.batch, B.batch, dtype=torch.float32, device=dev)
    ws = _ws("gram", A, B, 0, dev)
    _check(_lib().t3f_gram(_ref(A), _ref(B), _ptr(G), MATH[math], _ptr(ws), ws.numel(), _stream(dev)), "t3f_gram")
    return G


def norm(A: TT) -> torch.Tensor:
    dev = A.data.device
    out = torch.empty(A.batch, dtype=torch.float64, device=dev)
    ws = _ws("norm", A, None, 0, dev)
    _check(_lib().t3f_norm(_ref(A), _ptr(out), _ptr(ws), ws.numel(), _stream(dev)), "t3f_norm")
    return out


def gram_backward(A: TT, B: TT, dG: torch.Tensor, need_A=True, need_B=True, math: str = "fp32",
                  ws: Optional[torch.Tensor] = None):
    """Cotangents of sum_ab dG[a,b] <A_a, B_b>; math "tf32" / "bf16" runs the tensor-core
    adjoint (its workspace holds the stored partials; pass `ws` to reuse one)."""
    dev = A.data.device
    dA = A.empty_like(torch.float32) if need_A else None
    dB = B.empty_like(torch.float32) if need_B else None
    if ws is None:
        ws = _ws("gram_bwd" if math == "fp32" else "gram_bwd_tc", A, B, 0, dev)
    dG = dG.contiguous().to(torch.float32)
    _check(_lib().t3f_gram_backward(_ref(A), _ref(B), _ptr(dG), _ref(dA), _ref(dB), MATH[math], _ptr(ws),
                                    ws.numel(), _stream(dev)), "t3f_gram_backward")
    return dA, dB


def gather(X: TT, idx: torch.Tensor, y: Optional[torch.Tensor] = None, want_vals: bool = True,
           want_loss: bool = False):
    """idx: int32 [d][N] on the device. Returns (vals or None, loss or None)."""
    dev = X.data.device
    N = idx.shape[1]
    vals = torch.empty(N, dtype=torch.float32, device=dev) if want_vals else None
    loss = torch.empty(1, dtype=torch.float64, device=dev) if want_loss else None
    ws = _ws("gather", X, None, N, dev)
    _check(_lib().t3f_gather(_ref(X), _ptr(idx), N, _ptr(y), _ptr(vals), _ptr(loss), _ptr(ws),
                             ws.numel(), _stream(dev)), "t3f_gather")
    return vals, loss


def gather_backward(X: Optional[TT], idx: torch.Tensor, w: Optional[torch.Tensor] = None,
                    y: Optional[torch.Tensor] = None, want_loss: bool = False,
                    riemannian: bool = False, U: Optional[TT] = None, V: Optional[TT] = None,
                    return_ws: bool = False):
    """Core cotangents (riemannian=False) or tangent coordinates dU (riemannian=True)."""
    base = U if riemannian else X
    dev = base.data.device
    N = idx.shape[1]
    dX = base.empty_like(torch.float32)
    loss = torch.empty(1, dtype=torch.float64, device=dev) if want_loss else None
    if riemannian:
        ws = _ws("rgather_bwd", U, V, N, dev)
    else:
        ws = _ws("gather_bwd", X, None, N, dev)
    _check(_lib().t3f_gather_backward(_ref(X) if not riemannian else None, _ptr(idx), N, _ptr(w), _ptr(y),
                                      _ptr(loss), _ref(dX), int(bool(riemannian)), _ref(U), _ref(V),
                                      _ptr(ws), ws.numel(), _stream(dev)), "t3f_gather_backward")
    if return_ws:
        return dX, loss, ws
    return dX, loss


def matvec(A: TT, x: TT) -> TT:
    dev = A.data.device
    P = max(A.batch, x.batch)
    ranks = [a * b for a, b in zip(A.ranks, x.ranks)]
    C = TT.empty(A.m, ranks, P, None, torch.float32, dev)
    ws = _ws("matvec", A, x, 0, dev)
    _check(_lib().t3f_matvec(_ref(A), _ref(x), _ref(C), _ptr(ws), ws.numel(), _stream(dev)), "t3f_matvec")
    return C


def matvec_backward(A: TT, x: TT, dC: TT, need_A=True, need_x=True):
    dev = A.data.device
    dA = A.empty_like(torch.float32) if need_A else None
    dx = x.empty_like(torch.float32) if need_x else None
    _check(_lib().t3f_matvec_backward(_ref(A), _ref(x), _ref(dC), _ref(dA), _ref(dx), None, 0,
                                      _stream(dev)), "t3f_matvec_backward")
    return dA, dx


def orth_ranks(n, ranks):
    out = (ctypes.c_int32 * (len(n) + 1))()
    _check(_lib().t3f_orth_ranks(len(n), _i32(n), _i32(ranks), out), "t3f_orth_ranks")
    return [int(v) for v in out]


def orthogonalize(X: TT, dtype=torch.float32):
    dev = X.data.device
    r = orth_ranks(X.n, X.ranks)
    U = TT.empty(X.n, r, X.batch, None, dtype, dev)
    V = TT.empty(X.n, r, X.batch, None, dtype, dev)
    ws = _ws("orth", X, None, 0, dev)
    _check(_lib().t3f_orthogonalize(_ref(X), _ref(U), _ref(V), _ptr(ws), ws.numel(), _stream(dev)),
           "t3f_orthogonalize")
    return U, V


def project_sum(U: TT, V: TT, Z: TT, c: torch.Tensor, math: str = "fp32") -> TT:
    dev = U.data.device
    dU = U.empty_like(torch.float32)
    ws = _ws("psum", U, Z, 0, dev)
    c = c.contiguous().to(torch.float32)
    _check(_lib().t3f_project_sum(_ref(U), _ref(V), _ref(Z), _ptr(c), _ref(dU), MATH[math], _ptr(ws),
                                  ws.numel(), _stream(dev)), "t3f_project_sum")
    return dU


def project_sum_backward(U: TT, V: TT, Z: TT, c: torch.Tensor, dUbar: TT, need_Z=True, need_c=True):
    dev = U.data.device
    dZ = Z.empty_like(torch.float32) if need_Z else None
    dc = torch.empty(Z.batch, dtype=torch.float32, device=dev) if need_c else None
    ws = _ws("psum_bwd", U, Z, 0, dev)
    c = c.contiguous().to(torch.float32)
    _check(_lib().t3f_project_sum_backward(_ref(U), _ref(V), _ref(Z), _ptr(c), _ref(dUbar), _ref(dZ),
                                           _ptr(dc), _ptr(ws), ws.numel(), _stream(dev)),
           "t3f_project_sum_backward")
    return dZ, dc


def project(U: TT, V: TT, Z: TT, c: Optional[torch.Tensor] = None) -> TT:
    """Tangent coordinates of c_j P_X Z_j for every object of Z (batch Z.batch, U's shape)."""
    dev = U.data.device
    dU = TT.empty(U.n, U.ranks, Z.batch, None, torch.float32, dev)
    ws = _ws("project", U, Z, 0, dev)
    c = None if c is None else c.contiguous().to(torch.float32)
    _check(_lib().t3f_project(_ref(U), _ref(V), _ref(Z), _ptr(c), _ref(dU), _ptr(ws), ws.numel(), _stream(dev)),
           "t3f_project")
    return dU


def tangent_gram(dA: TT, dB: TT, math: str = "fp32") -> torch.Tensor:
    """G[a, b] = <xi_a, eta_b> for tangent vectors of one tangent space (gauge coordinates)."""
    dev = dA.data.device
    G = torch.empty(dA.batch, dB.batch, dtype=torch.float32, device=dev)
    ws = _ws("tangent_gram", dA, dB, 0, dev)
    _check(_lib().t3f_tangent_gram(_ref(dA), _ref(dB), _ptr(G), MATH[math], _ptr(ws), ws.numel(), _stream(dev)),
           "t3f_tangent_gram")
    return G


def project_matvec(U: TT, V: TT, A: TT, x: TT) -> TT:
    """Tangent coordinates of P_X (A x_j) for every x_j (the product is never formed)."""
    dev = U.data.device
    dU = TT.empty(U.n, U.ranks, x.batch, None, torch.float32, dev)
    nbytes = _lib().t3f_project_matvec_workspace_size(_ref(U), _ref(A), _ref(x))
    ws = torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=dev)
    _check(_lib().t3f_project_matvec(_ref(U), _ref(V), _ref(A), _ref(x), _ref(dU), _ptr(ws), ws.numel(),
                                     _stream(dev)), "t3f_project_matvec")
    return dU


def completion_hvp(U: TT, V: TT, idx: torch.Tensor, dZ: TT, return_ws: bool = False):
    """Coordinates of P_X (sum_t xi(i_t) e_{i_t}) for the tangent vector with coordinates dZ."""
    dev = U.data.device
    N = idx.shape[1]
    out = U.empty_like(torch.float32)
    ws = _ws("completion_hvp", U, V, N, dev)
    _check(_lib().t3f_completion_hvp(_ref(U), _ref(V), _ptr(idx), N, _ref(dZ), _ref(out), _ptr(ws), ws.numel(),
                                     _stream(dev)), "t3f_completion_hvp")
    return (out, ws) if return_ws else out


def round_ranks(n, ranks, max_rank):
    out = (ctypes.c_int32 * (len(n) + 1))()
    _check(_lib().t3f_round_ranks(len(n), _i32(n), _i32(ranks), int(max_rank), out), "t3f_round_ranks")
    return [int(v) for v in out]


def round_tt(X: TT, max_rank: int) -> TT:
    """TT rounding of every object of X to ranks <= max_rank (FP64 TT-SVD, F32 output)."""
    dev = X.data.device
    Y = TT.empty(X.n, round_ranks(X.n, X.ranks, max_rank), X.batch, None, torch.float32, dev)
    ws = _ws("round", X, None, 0, dev)
    _check(_lib().t3f_round(_ref(X), int(max_rank), _ref(Y), _ptr(ws), ws.numel(), _stream(dev)), "t3f_round")
    return Y


def fma_probe(grid: int, iters: int, device="cuda", fp64: bool = False):
    """Launch the FP32 (or FP64) FMA probe once; returns (FLOPs of the launch, its output)."""
    out = torch.empty(grid * 256, dtype=torch.float64 if fp64 else torch.float32, device=device)
    fn = _lib().t3f_fma_probe_f64 if fp64 else _lib().t3f_fma_probe
    _check(fn(grid, iters, _ptr(out), _stream(torch.device(device))), "t3f_fma_probe")
    return float(_lib().t3f_fma_probe_flops(grid, iters)), out


def device_status(ws: torch.Tensor) -> int:
    return int(_lib().t3f_device_status(_ptr(ws), _stream(ws.device)))


def launch_count() -> int:
    """Kernels launched by libt3f in this process so far."""
    return int(_lib().t3f_launch_count())


# ---------------------------------------------------------------------------------------
# Ragged collections and grouped Gram matrices
# ---------------------------------------------------------------------------------------

class _RDesc(ctypes.Structure):
    _fields_ = [("count", ctypes.c_int32), ("d", ctypes.POINTER(ctypes.c_int32)),
                ("n", ctypes.POINTER(ctypes.c_int32)), ("ranks", ctypes.POINTER(ctypes.c_int32)),
                ("obj_off", ctypes.POINTER(ctypes.c_int64)), ("cores", ctypes.c_void_p),
                ("dtype", ctypes.c_int32)]


_RP = ctypes.POINTER(_RDesc)
_I32P = ctypes.POINTER(ctypes.c_int32)
_SIGS.update({
    "t3f_gram_groups_workspace_size": (ctypes.c_size_t, [_RP, ctypes.c_int32, _I32P, _I32P]),
    "t3f_gram_groups_prepare": (ctypes.c_int32, [_RP, ctypes.c_int32, _I32P, _I32P, _VP, _SZ, _VP]),
    "t3f_gram_groups": (ctypes.c_int32, [_RP, ctypes.c_int32, _I32P, _I32P, ctypes.c_int32, _VP, _VP, _VP, _SZ,
                                         _VP]),
    "t3f_gram_groups_backward": (ctypes.c_int32, [_RP, ctypes.c_int32, _I32P, _I32P, ctypes.c_int32, _VP, _VP, _VP,
                                                  _SZ, _VP]),
    "t3f_gram_groups_backward_workspace_size": (ctypes.c_size_t, [_RP, ctypes.c_int32, _I32P, _I32P, ctypes.c_int32]),
})
EXPORTS = tuple(_SIGS)


class RaggedTT:
    """TT-vectors of different d, modes and ranks stored back to back in one flat tensor:
    object o's cores (r_{k-1}, n_k, r_k) follow each other starting at element offsets[o]."""

    def __init__(self, data: torch.Tensor, dims, modes, ranks, offsets):
        self.data = data
        self.dims = [int(v) for v in dims]
        self.modes = [[int(v) for v in m] for m in modes]
        self.ranks = [[int(v) for v in r] for r in ranks]
        self.offsets = [int(v) for v in offsets]
        self.count = len(self.dims)
        self._keep = None

    @staticmethod
    def object_numel(modes, ranks):
        return sum(ranks[k] * modes[k] * ranks[k + 1] for k in range(len(modes)))

    @classmethod
    def from_objects(cls, objects, dtype=torch.float32, device="cuda"):
        """objects: list of per-object core lists, core k shaped (r_{k-1}, n_k, r_k)."""
        flat, dims, modes, ranks, offs, o = [], [], [], [], [], 0
        for cores in objects:
            ts = [torch.as_tensor(c) for c in cores]
            dims.append(len(ts))
            modes.append([t.shape[1] for t in ts])
            ranks.append([ts[0].shape[0]] + [t.shape[2] for t in ts])
            offs.append(o)
            for t in ts:
                flat.append(t.reshape(-1))
                o += t.numel()
        data = torch.cat(flat).to(dtype=dtype).to(device)
        return cls(data, dims, modes, ranks, offs)

    def object_cores(self, o):
        out, off = [], self.offsets[o]
        for k in range(self.dims[o]):
            r0, n, r1 = self.ranks[o][k], self.modes[o][k], self.ranks[o][k + 1]
            out.append(self.data[off:off + r0 * n * r1].view(r0, n, r1))
            off += r0 * n * r1
        return out

    def desc(self) -> _RDesc:
        d = _i32(self.dims)
        n = _i32([v for m in self.modes for v in m])
        r = _i32([v for rr in self.ranks for v in rr])
        off = (ctypes.c_int64 * self.count)(*self.offsets)
        self._keep = (d, n, r, off)
        return _RDesc(self.count, d, n, r, off, ctypes.c_void_p(self.data.data_ptr()), _CODE[self.data.dtype])


def _tiles_arg(tiles):
    return None if tiles is None else _i32(tiles)


def gram_groups_prepare(X: RaggedTT, gstart, tiles=None, backward_math: str = "fp32") -> torch.Tensor:
    """Workspace holding the work list and object tables of the grouped Gram (host copies),
    sized for the adjoint in `backward_math` too (the tensor-core adjoint stores its partials
    there)."""
    gs = _i32(gstart)
    tl = _tiles_arg(tiles)
    nbytes = _lib().t3f_gram_groups_backward_workspace_size(ctypes.byref(X.desc()), len(gstart) - 1, gs, tl,
                                                            MATH[backward_math])
    if nbytes == 0:
        raise T3FError(-2, "t3f_gram_groups_workspace_size")
    ws = torch.empty(int(nbytes), dtype=torch.uint8, device=X.data.device)
    _check(_lib().t3f_gram_groups_prepare(ctypes.byref(X.desc()), len(gstart) - 1, gs, tl, _ptr(ws), ws.numel(),
                                          _stream(X.data.device)), "t3f_gram_groups_prepare")
    return ws


def gram_groups(X: RaggedTT, gstart, ws: torch.Tensor, tiles=None, want_norms=True, out=None, norms=None,
                math: str = "fp32"):
    """Concatenated per-group Gram matrices (and FP64 norms) from a prepared workspace;
    math "tf32" / "bf16" puts the pairs of rank > 8 objects on the tensor cores."""
    dev = X.data.device
    total = sum((gstart[g + 1] - gstart[g]) ** 2 for g in range(len(gstart) - 1))
    out = torch.empty(total, dtype=torch.float32, device=dev) if out is None else out
    if want_norms and norms is None:
        norms = torch.empty(X.count, dtype=torch.float64, device=dev)
    _check(_lib().t3f_gram_groups(ctypes.byref(X.desc()), len(gstart) - 1, _i32(gstart), _tiles_arg(tiles),
                                  MATH[math], _ptr(out),
                                  _ptr(norms) if want_norms else None, _ptr(ws), ws.numel(), _stream(dev)),
           "t3f_gram_groups")
    return out, (norms if want_norms else None)


def gram_groups_backward(X: RaggedTT, gstart, ws: torch.Tensor, dout: torch.Tensor, tiles=None, dcores=None,
                         math: str = "fp32"):
    """Core cotangents of the grouped Gram; math "tf32" / "bf16" needs a workspace prepared
    with the same backward_math."""
    dev = X.data.device
    dcores = torch.empty(X.data.numel(), dtype=torch.float32, device=dev) if dcores is None else dcores
    _check(_lib().t3f_gram_groups_backward(ctypes.byref(X.desc()), len(gstart) - 1, _i32(gstart), _tiles_arg(tiles),
                                           MATH[math], _ptr(dout), _ptr(dcores), _ptr(ws), ws.numel(),
                                           _stream(dev)),
           "t3f_gram_groups_backward")
    return dcores


DEFAULT_TILES = (10, 6, 3, 1)


def autotune_gram_groups(X: RaggedTT, gstart, candidates=(1, 2, 3, 4, 6, 8, 10, 12, 16), reps=3):
    """Rank-bucket tile sides chosen by timing the grouped forward sweep on X itself:
    coordinate search over the four buckets, starting from the defaults. Returns a tuple of
    four tile sides; infeasible candidates (tiles that do not fit one CTA) are skipped."""
    dev = X.data.device

    def time_tiles(tl):
        try:
            ws = gram_groups_prepare(X, gstart, tl)
        except T3FError:
            return float("inf")
        gram_groups(X, gstart, ws, tl, want_norms=False)
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            gram_groups(X, gstart, ws, tl, want_norms=False)
        e1.record()
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1) / reps

    best = list(DEFAULT_TILES)
    best_t = time_tiles(tuple(best))
    for b in (3, 2, 1, 0):
        for c in candidates:
            if c == best[b]:
                continue
            trial = list(best)
            trial[b] = c
            t = time_tiles(tuple(trial))
            if t < best_t:
                best, best_t = trial, t
    return tuple(best), best_t
