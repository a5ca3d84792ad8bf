"""Helpers for the GPU parity tests: move seeded numpy inputs to the device and
results back. The library is called through the C ABI binding."""
import numpy as np


def dev_u64(a: np.ndarray):
    import torch

    a = np.ascontiguousarray(a, dtype=np.uint64)
    return torch.from_numpy(a.view(np.int64).copy()).cuda()


def zeros_u8(n):
    import torch

    return torch.zeros(n, dtype=torch.uint8, device="cuda")


def zeros_u64(n):
    import torch

    return torch.zeros(n, dtype=torch.int64, device="cuda")


def host(t) -> np.ndarray:
    import torch

    torch.cuda.synchronize()
    out = t.cpu().numpy()
    if out.dtype == np.int64:
        out = out.view(np.uint64)
    return out


def first_diff(a: np.ndarray, b: np.ndarray):
    if a.shape != b.shape:
        return f"shape {a.shape} vs {b.shape}"
    d = np.nonzero(a != b)[0]
    if d.size == 0:
        return None
    i = int(d[0])
    return f"{d.size} differing bytes, first at {i}: {a[i]} vs {b[i]}"
