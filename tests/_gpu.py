"""Helpers for the GPU tests: numpy <-> torch CUDA copies of uint32 data."""
import numpy as np


def to_dev(a: np.ndarray):
    import torch
    a = np.ascontiguousarray(a)
    if a.dtype == np.uint32:
        a = a.view(np.int32)
    elif a.dtype == np.uint64:
        a = a.view(np.int64)
    return torch.from_numpy(a).cuda()


def to_host_u32(t) -> np.ndarray:
    return t.cpu().numpy().view(np.uint32)


def to_host_u64(t) -> np.ndarray:
    return t.cpu().numpy().view(np.uint64)
