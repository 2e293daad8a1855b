"""CPU checks of the C ABI: the library builds for sm_103a, loads, and exports every function that
include/lqcd.h declares.  No compute call is made (there is no GPU here)."""
import ctypes
import shutil

import pytest

from paper_1903_06986_gb300 import build, lqcd


@pytest.fixture(scope="module")
def lib():
    if shutil.which("nvcc") is None and not __import__("os").path.exists(build.LIB):
        pytest.skip("nvcc not available")
    build.build()
    return lqcd.load()


def test_header_declares_the_boundary():
    names = lqcd.header_functions()
    for required in ["lqcd_wilson_apply", "lqcd_gmresdr_solve", "lqcd_minresdr_solve", "lqcd_deflate_project",
                     "lqcd_loop_estimate", "lqcd_noise_z4", "lqcd_ctx_create", "lqcd_hop_traces",
                     "lqcd_poly_coeffs", "lqcd_proj_solve", "lqcd_contract", "lqcd_xi_inverse"]:
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    raw = ctypes.CDLL(build.LIB)
    missing = [n for n in lqcd.header_functions() if not hasattr(raw, n)]
    assert missing == []


def test_version_and_argument_checks(lib):
    assert b"sm_103a" in lib.lqcd_version()
    # argument validation happens before any CUDA call
    assert lib.lqcd_ctx_create(None, None, 18, None) == lqcd.ERR_INVALID_ARG
    h = ctypes.c_void_p()
    bad = (ctypes.c_int * 4)(4, 4, 1, 4)
    assert lib.lqcd_ctx_create(ctypes.byref(h), bad, 18, None) == lqcd.ERR_INVALID_ARG
    good = (ctypes.c_int * 4)(4, 4, 4, 4)
    assert lib.lqcd_ctx_create(ctypes.byref(h), good, 16, None) == lqcd.ERR_INVALID_ARG
    assert lib.lqcd_wilson_apply(None, None, 0.1, None, None, 1, 0, 0) == lqcd.ERR_INVALID_ARG


def test_new_entry_points_reject_bad_arguments_without_cuda(lib):
    # a NULL context is refused before any CUDA call (no GPU here)
    assert lib.lqcd_set_defl_engine(None, lqcd.DEFL_TENSOR) == lqcd.ERR_INVALID_ARG
    assert lib.lqcd_tc_vdag_x(None, None, 4, None, 1, None) == lqcd.ERR_INVALID_ARG
    assert lib.lqcd_tc_v_c(None, None, 4, None, 1, None) == lqcd.ERR_INVALID_ARG
    v = ctypes.c_double()
    assert lib.lqcd_timing_bytes(None, 0, ctypes.byref(v)) == lqcd.ERR_INVALID_ARG
    assert lqcd.KERNEL_CLASSES[9:] == ["tensor", "slice"]
    # the probe depth, the Lanczos window and the loop's inner restart and host-links entry points
    assert lib.lqcd_set_probe_depth(None, 2) == lqcd.ERR_INVALID_ARG
    assert lib.lqcd_set_inner_window(None, 2) == lqcd.ERR_INVALID_ARG
    assert lib.lqcd_loop_set_inner_restart(None, 80) == lqcd.ERR_INVALID_ARG
    assert lib.lqcd_loop_noises_host(None, None, 0, 1, None, None) == lqcd.ERR_INVALID_ARG


def test_tc_slice_bytes_host_query(lib):
    """Two slice copies of 7 bf16 (2 bytes) per real entry: at least 28 k L bytes, at most that
    with k padded to a row tile (128) for one copy and to a chunk (32) for the other, L padded to
    128, plus the exponent arrays."""
    for dims, k in (((24, 24, 24, 32), 200), ((4, 4, 4, 4), 5), ((3, 5, 2, 7), 130)):
        L = 24 * dims[0] * dims[1] * dims[2] * dims[3]
        b = lqcd.tc_slice_bytes(dims, k)
        pad = lambda x, m: -(-x // m) * m
        assert 28 * k * L <= b <= 14 * pad(L, 128) * (pad(k, 128) + pad(k, 32)) + 4 * L + 32 * (k + 2)
    assert lqcd.tc_slice_bytes((24, 24, 24, 32), 200) > 60e9     # the 24^3 x 32, 200-vector space
    out = ctypes.c_size_t()
    assert lib.lqcd_tc_slice_bytes((ctypes.c_int * 4)(4, 4, 1, 4), 5, ctypes.byref(out)) == lqcd.ERR_INVALID_ARG
    assert lib.lqcd_tc_slice_bytes((ctypes.c_int * 4)(4, 4, 4, 4), 0, ctypes.byref(out)) == lqcd.ERR_INVALID_ARG
    assert lib.lqcd_tc_slice_bytes((ctypes.c_int * 4)(4, 4, 4, 4), 5, None) == lqcd.ERR_INVALID_ARG
    # beyond the context limits (extent > 1024; more than 2^28 sites): rejected, no overflowed size
    assert lib.lqcd_tc_slice_bytes((ctypes.c_int * 4)(4, 4, 4, 2048), 5, ctypes.byref(out)) == lqcd.ERR_INVALID_ARG
    assert lib.lqcd_tc_slice_bytes((ctypes.c_int * 4)(1024, 1024, 1024, 1024), 200,
                                   ctypes.byref(out)) == lqcd.ERR_INVALID_ARG
    assert lib.lqcd_tc_slice_bytes((ctypes.c_int * 4)(256, 256, 64, 128), 1, ctypes.byref(out)) == lqcd.ERR_INVALID_ARG
