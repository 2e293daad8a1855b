"""GPU parity of the derivative stage (kappa and gauge links) with the oracle, and consistency of
the derivatives with central finite differences of the GPU estimates themselves."""
import numpy as np
import pytest

from oracle import derivs as Dv, lattice as L, pipeline as PL, rng
from paper_1903_06986_gb300 import lqcd, synth
from tests.gpu_util import context, dev, host, rel_err, torch_cuda

pytestmark = pytest.mark.gpu


def rand_fields(dims, n, seed):
    r = np.random.default_rng(seed)
    shp = L.field_shape(dims, (n,))
    return r.standard_normal(shp) + 1j * r.standard_normal(shp)


def test_link_grad_kernel_matches_oracle():
    dims = (3, 2, 4, 4)
    ctx = context(dims)
    U = synth.su3_links(dims, 0.5, 51)
    kappa = 0.137
    x, z = rand_fields(dims, 2, 1), rand_fields(dims, 2, 2)
    g, gl = lqcd.link_grad(ctx, dev(U), kappa, dev(z), dev(x), scale=0.5)
    ref = 0.5 * (Dv.link_gradient(U, kappa, x[0], z[0]) + Dv.link_gradient(U, kappa, x[1], z[1]))
    assert rel_err(host(g), ref) < 1e-12
    dU = dUc = 0
    for r in range(2):
        a, b = Dv.link_matrix_derivatives(U, kappa, x[r], z[r])
        dU, dUc = dU + a, dUc + b
    assert rel_err(host(gl), 0.5 * (dUc + dU.conj())) < 1e-12


@pytest.mark.parametrize("system", [lqcd.SYS_M, lqcd.SYS_MG5], ids=["M", "MG5"])
def test_loop_derivs_match_oracle(system):
    """Both solver paths (GMRES-DR/Proj on M, and MINRES-DR/Proj on M' = M gamma_5 with x = gamma_5 y)
    against the oracle's solves on M: the derivatives depend on the solutions only."""
    dims, kappa = (2, 2, 2, 4), 0.12
    ctx = context(dims)
    U = synth.su3_links(dims, 0.45, 2)
    N = 6
    # solves to 3e-14: x, y = M^{-1} P x and z agree within a few cond(M)^2 * 3e-14 (cond(M) = 12.5)
    g = lqcd.loop_derivs(ctx, dev(U), kappa, 5, N, 3, 40, 8, 7, 3e-14, 1e-14, system=system)
    assert g["converged"] and g["max_true_resid"] <= 3e-14
    ref = PL.loop_derivs(U, kappa, dims, 5, N, 40, 8, 7, 3e-14, 1e-14)
    for mode in range(2):
        want = ref["per_noise"][mode]
        scale = np.abs(want).max(axis=0)
        assert np.all(np.abs(g["per_noise"][mode] - want) <= 1e-11 * scale), mode
    assert rel_err(host(g["link_grad"]), ref["link_grad"]) < 1e-11


@pytest.mark.parametrize("prec", [1, 2], ids=["fp32", "fp16"])
def test_loop_derivs_mixed_precision_match_fp64(prec):
    """The derivative solves (x, y = M^{-1} P x, z = M^{-dag} eta) in mixed precision reach the same
    FP64 true residual as the plain path, so the derivatives agree within cond * tol."""
    dims, kappa = (2, 2, 2, 4), 0.14
    ctx = context(dims)
    U = dev(synth.su3_links(dims, 0.45, 2))
    args = (5, 6, 3, 40, 8, 7, 1e-12, 1e-13)
    ref = lqcd.loop_derivs(ctx, U, kappa, *args)
    got = lqcd.loop_derivs(ctx, U, kappa, *args, prec=prec)
    assert got["converged"] and got["max_true_resid"] <= 1e-12
    for mode in range(2):
        scale = np.abs(ref["per_noise"][mode]).max(axis=0)
        assert np.all(np.abs(got["per_noise"][mode] - ref["per_noise"][mode]) <= 1e-8 * scale + 1e-10), mode
    assert rel_err(host(got["link_grad"]), host(ref["link_grad"])) < 1e-8


def test_dkappa_matches_finite_difference_of_estimates():
    """The GPU d/dkappa of the NS and PS estimates equals a fourth-order central difference of the GPU
    loop estimate itself (same noises), for all nine operators."""
    dims = (4, 4, 4, 4)
    ctx = context(dims)
    U = dev(synth.su3_links(dims, 0.3, 1))
    kappa, h = 0.12, 1e-4
    kw = dict(m=20, k=5, K=4, npoly=3, tol=1e-13, tol_special=1e-13)
    d = lqcd.loop_derivs(ctx, U, kappa, 1, 4, 4, 20, 5, 4, 1e-13, 1e-13, want_grad=False)
    est = lambda k: ctx.loop_estimate(U, k, 1, 4, 4, modes=lqcd.SUB_NONE | lqcd.SUB_PERT, **kw)["mean"]
    f = {s: est(kappa + s * h) for s in (-2, -1, 1, 2)}
    fd = (-f[2] + 8 * f[1] - 8 * f[-1] + f[-2]) / (12 * h)
    for mode in range(2):
        assert np.allclose(d["dkappa"][mode], fd[[0, 1][mode]], rtol=2e-7, atol=1e-6), mode


def test_autograd_scalar_loop():
    torch = torch_cuda()
    from paper_1903_06986_gb300.autograd import scalar_loop
    dims = (2, 2, 2, 4)
    ctx = context(dims)
    U0 = synth.su3_links(dims, 0.45, 3)
    opts = dict(seed=9, nnoise=4, block=4, m=40, k=8, K=4, npoly=3, tol=1e-13, tol_special=1e-13)
    kappa = torch.tensor(0.13, dtype=torch.float64, requires_grad=True)
    links = dev(U0).requires_grad_(True)
    out = scalar_loop(kappa, links, ctx, **opts)
    out.backward()
    f = lambda k, UU: float(scalar_loop(torch.tensor(k, dtype=torch.float64), dev(UU), ctx, **opts))
    h = 1e-5
    fdk = (f(0.13 + h, U0) - f(0.13 - h, U0)) / (2 * h)
    assert abs(kappa.grad.item() - fdk) < 1e-6 * max(1.0, abs(fdk))
    # directional derivative along Lie-algebra perturbations of a few links: dL = Re <grad, dU>
    G = host(links.grad)
    r = np.random.default_rng(4)
    for _ in range(4):
        mu = int(r.integers(4))
        site = tuple(int(r.integers(n)) for n in L.site_shape(dims))
        a = int(r.integers(8))
        Up, Um = Dv.perturb_link(U0, mu, site, a, h), Dv.perturb_link(U0, mu, site, a, -h)
        fd = (f(0.13, Up) - f(0.13, Um)) / (2 * h)
        dU = (Up - Um) / (2 * h)
        pred = np.real(np.vdot(G, dU))
        assert abs(pred - fd) < 1e-6 * max(1.0, abs(fd)), (mu, site, a)
