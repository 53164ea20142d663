"""Helpers for GPU tests: numpy <-> CUDA tensors by bit pattern, key-type codes."""
from __future__ import annotations

import numpy as np

KT = {"u32": 0, "u64": 1, "f32": 2, "i32": 3, "i64": 4, "f64": 5, "u16": 6, "i16": 7}


def to_dev(a: np.ndarray, dev="cuda:0"):
    import torch

    view = {2: np.int16, 4: np.int32, 8: np.int64}[a.dtype.itemsize]
    return torch.from_numpy(np.ascontiguousarray(a).view(view)).to(dev)


def from_dev(t, like: np.dtype) -> np.ndarray:
    a = t.cpu().numpy()
    return a.view(np.dtype(like))


def kt_of(a: np.ndarray) -> int:
    return {np.dtype(np.uint32): 0, np.dtype(np.uint64): 1, np.dtype(np.float32): 2,
            np.dtype(np.int32): 3, np.dtype(np.int64): 4, np.dtype(np.float64): 5,
            np.dtype(np.uint16): 6, np.dtype(np.int16): 7}[a.dtype]


def bits(a: np.ndarray) -> np.ndarray:
    """Bit patterns as unsigned integers of the key width (exact comparison)."""
    return a.view({2: np.uint16, 4: np.uint32, 8: np.uint64}[a.dtype.itemsize])
