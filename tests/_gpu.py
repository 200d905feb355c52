"""Helpers shared by the GPU tests: library loading and tensor plumbing."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


def require_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2403_03571_gb300 import build, capi
    build.build()
    return capi.load()


def dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def instance_tensors(inst, w=None):
    x = dev(inst.x, torch.float64)
    A = dev(inst.A, torch.float64)
    ww = dev(inst.w if w is None else w, torch.float64)
    v = dev(inst.v, torch.float64)
    return x, A, ww, v
