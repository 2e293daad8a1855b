"""Failure paths, made on the host (no GPU fault is ever caused):
  * NaN / Inf planted in the gauge links or in a deflation space -> LQCD_ERR_NONFINITE with a
    message, and the context keeps working (a valid call afterwards matches the oracle);
  * max_cycles = 1 -> LQCD_ERR_NOT_CONVERGED with the true residual reported;
  * a tensor-core pipeline wait made to run out (the loader stops filling stages, a flag that
    nothing then sets) under a short wait limit -> LQCD_ERR_TIMEOUT, device still answering."""
import numpy as np
import pytest

from oracle import lattice as L, subtract as S
from paper_1903_06986_gb300 import lqcd, synth
from tests.gpu_util import context, dev, host, rel_err, torch_cuda

pytestmark = pytest.mark.gpu

DIMS = (2, 2, 2, 4)
KW = dict(seed=3, nnoise=4, block=4, m=40, k=6, K=4, npoly=3, tol=1e-12, tol_special=1e-12)


@pytest.mark.parametrize("bad", [np.nan, np.inf], ids=["nan", "inf"])
def test_nonfinite_links_rejected_then_context_usable(bad):
    torch_cuda()
    ctx = context(DIMS)
    U = synth.su3_links(DIMS, 0.45, 5)
    Ubad = U.copy()
    Ubad[2, 1, 0, 1, 0, 1, 2] = bad
    with pytest.raises(lqcd.LqcdError) as e:
        ctx.loop_estimate(dev(Ubad), 0.14, **KW)
    assert e.value.status == lqcd.ERR_NONFINITE and "non-finite" in str(e.value)
    good = ctx.loop_estimate(dev(U), 0.14, **KW)
    fresh = context(DIMS).loop_estimate(dev(U), 0.14, **KW)
    assert good["converged"] and np.array_equal(good["per_noise"], fresh["per_noise"])


def test_max_cycles_one_reports_not_converged_with_true_residual():
    torch_cuda()
    ctx = context(DIMS)
    U = synth.su3_links(DIMS, 0.45, 6)
    b = ctx.noise_z4(9, 0, 1)
    x, info, _ = ctx.gmresdr_solve(dev(U), 0.14, b, 10, 3, 1e-12, max_cycles=1)
    assert info["converged"] == 0 and info["cycles"] == 1
    # the reported residual is the true one, recomputed here with the oracle's operator
    xh, bh = host(x)[0], host(b)[0]
    r = np.linalg.norm(bh - L.wilson(U, 0.14, xh)) / np.linalg.norm(bh)
    assert r > 1e-12 and abs(info["true_resid"] - r) <= 1e-10 * r
    res = ctx.loop_estimate(dev(U), 0.14, **dict(KW, max_cycles=1))
    assert res["status"] == lqcd.ERR_NOT_CONVERGED and not res["converged"]
    assert np.isfinite(res["max_true_resid"]) and res["max_true_resid"] > KW["tol"]


def _vectors(dims, k, seed):
    n = 12 * L.volume(dims)
    r = np.random.default_rng(seed)
    E, _ = np.linalg.qr(r.standard_normal((n, k)) + 1j * r.standard_normal((n, k)))
    return E


def test_tensor_core_wait_runs_out_then_recovers():
    torch = torch_cuda()
    ctx = context(DIMS)
    k = 6
    E = _vectors(DIMS, k, 7)
    Ed = dev(np.ascontiguousarray(E.T).reshape((k,) + L.field_shape(DIMS)))
    X = ctx.noise_z4(4, 0, 3)
    with pytest.raises(lqcd.LqcdError) as e:
        ctx.set_wait_limit(0.0)
    assert e.value.status == lqcd.ERR_INVALID_ARG
    ctx.set_wait_limit(0.05)
    ctx.inject_tc_stall(0)
    with pytest.raises(lqcd.LqcdError) as e:
        ctx.tc_vdag_x(Ed, X)
    assert e.value.status == lqcd.ERR_TIMEOUT and "timed out" in str(e.value)
    torch.cuda.synchronize()                         # the device still answers
    ref = S.defl_coeffs(E, host(X))
    G = ctx.tc_vdag_x(Ed, X)                         # the injection was one-shot
    assert rel_err(host(G), ref) < 1e-13
    # the same through the HFES projection with the tensor engine
    lam = np.linspace(0.1, 0.6, k).astype(np.complex128)
    defl = ctx.defl_import(Ed, lam)
    ctx.set_defl_engine(lqcd.DEFL_TENSOR)
    ctx.inject_tc_stall(0)
    with pytest.raises(lqcd.LqcdError) as e:
        ctx.deflate_project(defl, X, 1.0 / lam)
    assert e.value.status == lqcd.ERR_TIMEOUT
    y = ctx.deflate_project(defl, X, 1.0 / lam)
    assert rel_err(host(y), S.defl_vector(E, 1.0 / lam, host(X))) < 1e-13
    ctx.set_defl_engine(lqcd.DEFL_FP64)
    ctx.set_wait_limit(2.0)
    defl.close()


def test_nonfinite_deflation_vectors_rejected_by_tensor_engine():
    torch_cuda()
    ctx = context(DIMS)
    k = 5
    E = _vectors(DIMS, k, 8)
    Ebad = E.copy()
    Ebad[17, 3] = np.nan
    X = ctx.noise_z4(4, 0, 2)
    bad = dev(np.ascontiguousarray(Ebad.T).reshape((k,) + L.field_shape(DIMS)))
    with pytest.raises(lqcd.LqcdError) as e:
        ctx.tc_vdag_x(bad, X)
    assert e.value.status == lqcd.ERR_NONFINITE
    lam = np.linspace(0.1, 0.5, k).astype(np.complex128)
    defl = ctx.defl_import(bad, lam)
    ctx.set_defl_engine(lqcd.DEFL_TENSOR)
    with pytest.raises(lqcd.LqcdError) as e:
        ctx.deflate_project(defl, X, 1.0 / lam)
    assert e.value.status == lqcd.ERR_NONFINITE
    ctx.set_defl_engine(lqcd.DEFL_FP64)
    defl.close()
    good = dev(np.ascontiguousarray(E.T).reshape((k,) + L.field_shape(DIMS)))
    assert rel_err(host(ctx.tc_vdag_x(good, X)), S.defl_coeffs(E, host(X))) < 1e-13
