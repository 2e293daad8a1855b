"""GPU kernels compared with the oracle at the sizes the benchmark runs them (the launch shapes, grid
sizes and partial-reduction paths differ from the small parity cases):
  * one GMRES(30) cycle on 50 right-hand sides of the 8^3 x 16 workload (batched Arnoldi: multi-RHS
    Wilson, CGS2 multidot / multiaxpy / norms at N = 98304, 50 RHS), three sampled right-hand sides
    against the oracle's cycle at 1e-10 (Sec. 1, 7);
  * one GMRES-Proj cycle of the same 50 right-hand sides over a deflation space made by the oracle
    (imported with lqcd_defl_import_space), sampled against the oracle at 1e-10 (Sec. 5.3, 7);
  * the nine-operator contraction of 8 right-hand sides on 8^3 x 16 at 1e-13 (Sec. 6);
  * the packed FP32, FP16 and BF16 operators (recon 12, 8 right-hand sides) on 24^3 x 32 at
    sampled sites against Eq. xyz556 evaluated per site, within the rounding bound of the storage
    format (inputs are Z(4) noise, exact in every format; FP32 links and arithmetic)."""
import numpy as np
import pytest

from oracle import krylov as Kr, lattice as L, operators as O, rng
from paper_1903_06986_gb300 import lqcd, synth
from tests.gpu_util import context, dev, host, rel_err, torch_cuda

pytestmark = pytest.mark.gpu

DIMS8 = (8, 8, 8, 16)
KAPPA = 0.157
SAMPLE = (0, 23, 49)


@pytest.fixture(scope="module")
def workload8():
    U = synth.su3_links(DIMS8, 0.4323, 2024)
    ctx = context(DIMS8)
    etas = ctx.noise_z4(1, 0, 50)
    return U, ctx, etas


def test_gmres_cycle_50_rhs_sampled(workload8):
    U, ctx, etas = workload8
    x, info, _ = ctx.gmresdr_solve(dev(U), KAPPA, etas, 30, 0, 1e-30, max_cycles=1)
    assert info["cycles"] == 1
    A = lambda v: L.flat(L.wilson(U, KAPPA, L.unflat(v, DIMS8)))
    xh, eh = host(x), host(etas)
    for r in SAMPLE:
        xo, _, _ = Kr.gmres_dr(A, L.flat(eh[r]), 30, 0, 1e-30, 1)
        assert rel_err(L.flat(xh[r]), xo) < 1e-10, r


def test_gmres_proj_cycle_50_rhs_sampled(workload8):
    U, ctx, etas = workload8
    A = lambda v: L.flat(L.wilson(U, KAPPA, L.unflat(v, DIMS8)))
    b0 = L.flat(rng.z4_noise(1, rng.NOISE_SPECIAL, DIMS8))
    _, _, defl = Kr.gmres_dr(A, b0, 30, 10, 1e-30, 2)
    k = defl["Hbar"].shape[1]
    V = dev(np.ascontiguousarray(defl["V"].T).reshape((k + 1,) + L.field_shape(DIMS8)))
    space = ctx.defl_import_space(V, defl["Hbar"], hermitian=False)
    x, info = ctx.proj_solve(dev(U), KAPPA, space, etas, 20, 1e-30, max_cycles=1)
    assert info["cycles"] == 1
    xh, eh = host(x), host(etas)
    for r in SAMPLE:
        xo, _ = Kr.gmres_proj(A, L.flat(eh[r]), defl, 20, 1e-30, 1)
        assert rel_err(L.flat(xh[r]), xo) < 1e-10, r
    space.close()


def test_contract_8_rhs_8x8x8x16(workload8):
    U, ctx, _ = workload8
    r = np.random.default_rng(12)
    shp = L.field_shape(DIMS8, (8,))
    eta = r.standard_normal(shp) + 1j * r.standard_normal(shp)
    w = r.standard_normal(shp) + 1j * r.standard_normal(shp)
    got = ctx.contract(dev(U), KAPPA, dev(eta), dev(w))
    for n in range(8):
        ref = O.per_t(O.densities(U, KAPPA, eta[n], w[n]))
        assert rel_err(got[n], ref) < 1e-13, n


def test_packed_operators_24x24x24x32_sampled_sites():
    torch = torch_cuda()
    dims = (24, 24, 24, 32)
    U = synth.su3_links(dims, 0.4323, 7)
    ctx = lqcd.Context(dims, recon=12)
    Ud = dev(U)
    Up = ctx.pack_links_f32(Ud, 12)
    x = ctx.noise_z4(3, 0, 8)
    xh = host(x)
    r = np.random.default_rng(5)
    lt, lz, ly, lx = L.site_shape(dims)
    sites = [tuple(int(r.integers(n)) for n in (lt, lz, ly, lx)) for _ in range(48)]
    sites += [(0, 0, 0, 0), (lt - 1, lz - 1, ly - 1, lx - 1), (lt - 1, 0, ly - 1, 0), (0, lz - 1, 0, lx - 1)]
    ref = {n: L.wilson_at_sites(U, KAPPA, xh[n], sites) for n in (0, 3, 7)}
    # unit roundoff u of the output format, and a bound on the FP32 arithmetic: links rounded to
    # FP32 and row 2 rebuilt, each output component kappa times a sum of at most 48 terms of size
    # <= 1 for Z(4) input, about 30 rounded operations deep: 30 * 2^-24 * 48 * 2 kappa < 1e-5
    fp32_abs = 1e-5
    cases = [("f32", None, 2.0 ** -24), ("f16", lqcd.PREC_F16, 2.0 ** -11), ("bf16", lqcd.PREC_BF16, 2.0 ** -8)]
    cases = [(name + "/nr%d" % nr, prec, u, nr) for nr in (2, 3) for name, prec, u in cases]
    for name, prec, u, nr in cases:
        ctx.set_rhs_per_thread(nr)      # paired lanes, or paired lanes with staged neighbours
        if prec is None:
            y = ctx.unpack_f32(ctx.wilson_apply_packed(Up, 12, KAPPA, ctx.pack_f32(x)))
        else:
            xp = ctx.pack_half(x, prec)
            assert np.array_equal(host(ctx.unpack_half(xp, prec)), xh)      # Z(4) input is exact
            y = ctx.unpack_half(ctx.wilson_apply_half(Up, 12, KAPPA, xp, prec=prec), prec)
        yh = host(y)
        for n, want in ref.items():
            got = np.array([yh[n][s] for s in sites])
            bound = u * np.abs(want) + (1 + u) * fp32_abs
            assert np.all(np.abs(got - want) <= bound), (name, n, float((np.abs(got - want) - bound).max()))
    torch.cuda.synchronize()
    ctx.close()
