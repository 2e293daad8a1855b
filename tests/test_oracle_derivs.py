"""Pins of the oracle's derivatives (kappa and gauge links) against central finite differences of
quantities computed from dense matrices, and against the chain rule."""
import numpy as np

from oracle import derivs as Dv, exact, lattice as L, operators as O, rng, subtract as S
from paper_1903_06986_gb300 import synth

DIMS = (2, 2, 2, 4)


def solve(U, kappa, f):
    M = L.dense(lambda v: L.wilson(U, kappa, v), DIMS)
    return L.unflat(np.linalg.solve(M, L.flat(f)), DIMS)


def test_exact_dkappa_matches_finite_difference():
    U = synth.su3_links(DIMS, 0.5, 41)
    kappa, h = 0.13, 1e-5
    d = Dv.exact_dkappa(U, kappa, DIMS)
    fd = (exact.exact_traces(U, kappa + h, DIMS) - exact.exact_traces(U, kappa - h, DIMS)) / (2 * h)
    assert np.allclose(d, fd, rtol=1e-6, atol=1e-6)


def fd4(f, x, h):
    """Fourth-order central difference."""
    return (-f(x + 2 * h) + 8 * f(x + h) - 8 * f(x - h) + f(x - 2 * h)) / (12 * h)


def test_per_noise_dkappa_matches_finite_difference():
    U = synth.su3_links(DIMS, 0.5, 42)
    kappa, h = 0.14, 1e-5
    eta = rng.z4_noise(3, 0, DIMS)
    x = solve(U, kappa, eta)
    y = solve(U, kappa, L.hop(U, x))
    d = Dv.dkappa_densities(U, kappa, eta, x, y).sum(axis=(-1, -2, -3, -4))
    T = lambda k: O.densities(U, k, eta, solve(U, k, eta)).sum(axis=(-1, -2, -3, -4))
    fd = fd4(T, kappa, h)
    assert np.allclose(d, fd, rtol=1e-8, atol=1e-8)


def test_pert_derivatives_match_finite_difference():
    U = synth.su3_links(DIMS, 0.5, 43)
    kappa, h, K = 0.12, 1e-5, 7
    eta = rng.z4_noise(4, 1, DIMS)
    fd = (S.hop_series(U, kappa + h, eta, K) - S.hop_series(U, kappa - h, eta, K)) / (2 * h)
    assert np.allclose(Dv.dpert_vector(U, kappa, eta, K), fd, atol=1e-8)
    A = lambda k: S.pert_addback(S.hop_traces(U, k, K, DIMS), k, K).sum(axis=(-1, -2, -3, -4))
    fda = (A(kappa + h) - A(kappa - h)) / (2 * h)
    got = Dv.dpert_addback(S.hop_traces(U, kappa, K, DIMS), kappa, K).sum(axis=(-1, -2, -3, -4))
    assert np.allclose(got, fda, rtol=1e-6, atol=1e-6)


def test_link_gradient_matches_finite_difference_on_16_links():
    U = synth.su3_links(DIMS, 0.5, 44)
    kappa, h = 0.14, 1e-5
    eta = rng.z4_noise(5, 2, DIMS)
    x = solve(U, kappa, eta)
    z = L.g5(solve(U, kappa, L.g5(eta)))            # M^{-dag} eta = g5 M^{-1} g5 eta
    g = Dv.link_gradient(U, kappa, x, z)
    T = lambda UU: np.vdot(eta, solve(UU, kappa, eta))
    r = np.random.default_rng(7)
    for _ in range(16):
        mu = int(r.integers(4))
        site = tuple(int(r.integers(n)) for n in L.site_shape(DIMS))
        a = int(r.integers(8))
        fd = (T(Dv.perturb_link(U, mu, site, a, h)) - T(Dv.perturb_link(U, mu, site, a, -h))) / (2 * h)
        assert abs(fd - g[(mu,) + site + (a,)]) < 1e-6 * max(1.0, abs(fd))


def test_matrix_derivatives_chain_rule():
    U = synth.su3_links(DIMS, 0.5, 45)
    kappa = 0.14
    eta = rng.z4_noise(6, 3, DIMS)
    x = solve(U, kappa, eta)
    z = L.g5(solve(U, kappa, L.g5(eta)))
    g = Dv.link_gradient(U, kappa, x, z)
    dU, dUc = Dv.link_matrix_derivatives(U, kappa, x, z)
    for a in range(8):
        dX = 0.5j * np.einsum('cd,...de->...ce', Dv.LAMBDA[a], U)      # d U / d w_a
        chain = np.einsum('...ab,...ab->...', dU, dX) + np.einsum('...ab,...ab->...', dUc, dX.conj())
        assert np.allclose(chain, g[..., a], atol=1e-12)
