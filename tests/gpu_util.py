"""Helpers for the GPU parity tests (torch for device memory only)."""
import numpy as np


def rel_fro(a, b) -> float:
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def to_dev(A):
    import torch
    return torch.from_numpy(np.ascontiguousarray(A, dtype=np.float64)).cuda()


def empty_like_dev(n):
    import torch
    return torch.empty((n, n), dtype=torch.float64, device="cuda")


def to_host(t):
    import torch
    torch.cuda.synchronize()
    return t.cpu().numpy()
