"""Helpers shared by the tests: batch <-> per-object core lists, FP32 rounding of inputs,
and the error measure used for parity (normwise relative error of each output array)."""
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
