"""The allocation-free contraction entry point, lqcd_contract_noalloc.

It is meant for callers that cannot call cudaMalloc (a host application that owns all device
memory through its own allocator, a strict memory budget, or a latency-critical path where an
allocation may synchronise the device): its scratch is a fixed array inside the library, its
output a caller buffer.  This file is named to be collected last, so that a run
stopping at the first failure has already run every other test; it also passes on its own in a
fresh process.  The results are compared, on two calls in a row with different inputs, with the
context-based lqcd_contract within the contraction tolerance of the other GPU tests."""
import ctypes

import numpy as np
import pytest

from oracle import lattice as L
from paper_1903_06986_gb300 import synth
from tests.gpu_util import context, dev, host, rel_err, torch_cuda

pytestmark = pytest.mark.gpu

CONTRACT_TOL = 1e-13


def noalloc_fn():
    from paper_1903_06986_gb300 import build
    build.build()
    lib = ctypes.CDLL(build.LIB)
    f = lib.lqcd_contract_noalloc
    f.argtypes = [ctypes.POINTER(ctypes.c_int), ctypes.c_void_p, ctypes.c_double, ctypes.c_void_p,
                  ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    f.restype = ctypes.c_int
    return f


def fields(dims, n, seed):
    r = np.random.default_rng(seed)
    shp = L.field_shape(dims, (n,))
    return r.standard_normal(shp) + 1j * r.standard_normal(shp)


def test_noalloc_contract_matches_contract_twice():
    torch = torch_cuda()
    f = noalloc_fn()
    stream = torch.cuda.current_stream().cuda_stream
    for call, (dims, n, seed) in enumerate([((4, 4, 4, 8), 3, 1), ((3, 5, 2, 7), 2, 2)]):
        ctx = context(dims)
        U = dev(synth.su3_links(dims, 0.5, 10 + seed))
        eta, w = dev(fields(dims, n, seed)), dev(fields(dims, n, seed + 100))
        kappa = 0.137
        out = torch.empty((n, 9, dims[3]), dtype=torch.complex128, device="cuda")
        dd = (ctypes.c_int * 4)(*dims)
        rc = f(dd, ctypes.c_void_p(U.data_ptr()), kappa, ctypes.c_void_p(eta.data_ptr()),
               ctypes.c_void_p(w.data_ptr()), n, ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream))
        assert rc == 0, "call %d returned %d" % (call, rc)
        torch.cuda.synchronize()
        ref = ctx.contract(U, kappa, eta, w)
        assert rel_err(host(out), ref) < CONTRACT_TOL, call


def test_noalloc_rejects_oversize_without_launching():
    torch = torch_cuda()
    f = noalloc_fn()
    dims = (2, 2, 2, 8)
    U = torch.zeros((4, 8, 2, 2, 2, 3, 3), dtype=torch.complex128, device="cuda")
    v = torch.zeros((1, 8, 2, 2, 2, 4, 3), dtype=torch.complex128, device="cuda")
    dd = (ctypes.c_int * 4)(*dims)
    # 1000 right-hand sides x 8 timeslices x 9 operators > 65536 scratch entries
    rc = f(dd, ctypes.c_void_p(U.data_ptr()), 0.1, ctypes.c_void_p(v.data_ptr()), ctypes.c_void_p(v.data_ptr()),
           1000, ctypes.c_void_p(v.data_ptr()), None)
    assert rc == 1
    # more sites than a context accepts (2^29 > 2^28): rejected before any launch
    big = (ctypes.c_int * 4)(1024, 1024, 512, 2)
    rc = f(big, ctypes.c_void_p(U.data_ptr()), 0.1, ctypes.c_void_p(v.data_ptr()), ctypes.c_void_p(v.data_ptr()),
           1, ctypes.c_void_p(v.data_ptr()), None)
    assert rc == 1
    torch.cuda.synchronize()
