"""Shared helpers of the GPU tests (metrics, device handling)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


def cuda_or_skip():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2401_08260_gb300 import build
    build.build()
    return torch.device("cuda", 0)


def rel_inf(a, b, wsum):
    """max |a - b| / sum|w|, the accuracy measure of the kernel sums."""
    a = a.detach().cpu().numpy() if hasattr(a, "detach") else np.asarray(a)
    return float(np.max(np.abs(a.astype(np.float64) - np.asarray(b, dtype=np.float64))) / wsum)


def to_dev(a, dev, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.to(dev)
