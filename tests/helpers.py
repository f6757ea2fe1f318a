"""Small helpers shared by the GPU tests."""
import numpy as np


def relerr_per_body(a, ref):
    """Per-body relative force error |a_i - ref_i| / |ref_i|."""
    num = np.linalg.norm(np.asarray(a) - np.asarray(ref), axis=1)
    den = np.linalg.norm(np.asarray(ref), axis=1)
    return num / np.where(den > 0, den, 1.0)


def to_dev(arr, dev):
    import torch
    return torch.as_tensor(np.asarray(arr), dtype=torch.float64).to(dev).contiguous()


def host(t):
    return t.detach().cpu().numpy()
