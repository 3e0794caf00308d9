"""Helpers shared by the GPU tests (no method arithmetic here)."""
import numpy as np


def require_cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return torch


def to_dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def to_bf16_rne(x):
    """Round float64 values to bfloat16 (8 significant bits, ties to even)
    directly from FP64, returned as float64 (normal range only)."""
    x = np.asarray(x, dtype=np.float64)
    mant, ex = np.frexp(x)                  # x = mant * 2**ex, 0.5 <= |mant| < 1
    q = np.rint(mant * 256.0)               # 8 significant bits, half to even
    return np.ldexp(q / 256.0, ex)
