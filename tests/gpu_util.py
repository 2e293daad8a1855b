"""Helpers shared by the GPU parity tests: device availability, the library context, and
numpy <-> torch transfers of complex128 fields."""
import numpy as np
import pytest


def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def context(dims):
    torch_cuda()
    from paper_1903_06986_gb300 import build, lqcd
    build.build()
    return lqcd.Context(dims)


def dev(a):
    torch = torch_cuda()
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.complex128)).cuda()


def host(t):
    return t.detach().cpu().numpy()


def rel_err(a, b):
    a, b = np.asarray(a), np.asarray(b)
    den = max(np.abs(b).max(), 1e-300)
    return float(np.abs(a - b).max() / den)
