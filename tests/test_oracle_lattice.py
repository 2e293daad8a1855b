"""Pins of the oracle's Wilson operator (Eq. xyz556) against facts the paper and the mathematics fix:
gamma algebra, gamma_5-hermiticity (Sec. 5.4, 6), the free-field plane-wave spectrum, gauge
covariance, and the flat index convention."""
import numpy as np
import pytest

from oracle import lattice as L
from paper_1903_06986_gb300 import synth

D2 = (2, 2, 2, 2)
D4 = (4, 4, 4, 4)


def rand_field(dims, batch=(), seed=0):
    r = np.random.default_rng(seed)
    shp = L.field_shape(dims, batch)
    return r.standard_normal(shp) + 1j * r.standard_normal(shp)


def test_gamma_algebra():
    for mu in range(4):
        assert np.allclose(L.G[mu], L.G[mu].conj().T)
        for nu in range(4):
            ac = L.G[mu] @ L.G[nu] + L.G[nu] @ L.G[mu]
            assert np.allclose(ac, 2.0 * (mu == nu) * np.eye(4))
        assert np.allclose(L.G5 @ L.G[mu] + L.G[mu] @ L.G5, 0)
    assert np.allclose(L.G5 @ L.G5, np.eye(4))
    assert np.allclose(L.G5, L.G5.conj().T)


@pytest.mark.parametrize("dims", [D2, (4, 2, 2, 6)])
def test_gamma5_hermiticity(dims):
    U = synth.su3_links(dims, 0.5, 3)
    kappa = 0.13
    a, b = rand_field(dims, seed=1), rand_field(dims, seed=2)
    lhs = np.vdot(a, L.wilson(U, kappa, b))
    # M^dag = gamma_5 M gamma_5  <=>  <a, M b> = <g5 M g5 a, b>
    rhs = np.vdot(L.g5(L.wilson(U, kappa, L.g5(a))), b)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)
    # the explicitly written adjoint stencil agrees
    assert np.allclose(L.wilson_dag(U, kappa, a), L.g5(L.wilson(U, kappa, L.g5(a))), atol=1e-13)
    # M' = M g5 is Hermitian
    Mp = L.dense(lambda v: L.wilson_g5(U, kappa, v), dims)
    assert np.abs(Mp - Mp.conj().T).max() < 1e-14


def test_free_field_plane_waves():
    """U = 1: psi(x) = exp(i p.x) u with (B.gamma) u = +-|B| u gives M psi = (A +- i|B|) psi,
    A = 1 - 2 kappa sum cos p_mu, B_mu = 2 kappa sin p_mu, p_mu = 2 pi n_mu / L_mu."""
    dims = (4, 4, 2, 6)
    U = synth.unit_links(dims)
    kappa = 0.11
    lx, ly, lz, lt = dims
    t, z, y, x = np.meshgrid(np.arange(lt), np.arange(lz), np.arange(ly), np.arange(lx), indexing='ij')
    coords = [x, y, z, t]
    for n in [(0, 0, 0, 0), (1, 0, 0, 0), (1, 1, 1, 1), (3, 2, 1, 5), (2, 0, 1, 3)]:
        p = [2 * np.pi * n[m] / dims[m] for m in range(4)]
        A = 1 - 2 * kappa * sum(np.cos(pm) for pm in p)
        B = [2 * kappa * np.sin(pm) for pm in p]
        Bg = sum(B[m] * L.G[m] for m in range(4))
        w, vecs = np.linalg.eigh(Bg)
        phase = np.exp(1j * sum(p[m] * coords[m] for m in range(4)))
        for j in range(4):
            u = vecs[:, j]
            psi = phase[..., None, None] * u[:, None] * np.array([1.0, 0.3j, -0.2])[None, :]
            lam = A + 1j * w[j]
            assert abs(abs(w[j]) - np.sqrt(sum(b * b for b in B))) < 1e-13
            assert np.allclose(L.wilson(U, kappa, psi), lam * psi, atol=1e-13)


def test_gauge_covariance():
    dims = (2, 4, 2, 4)
    U = synth.su3_links(dims, 0.6, 5)
    g = synth.su3_links(dims, 2.0, 6)[0]          # one random SU(3) matrix per site
    Ug = np.empty_like(U)
    for mu in range(4):
        gfwd = np.roll(g, -1, axis=L.SITE_AXIS[mu])
        Ug[mu] = g @ U[mu] @ np.conj(np.swapaxes(gfwd, -1, -2))
    psi = rand_field(dims, seed=7)
    gpsi = np.einsum('...ab,...sb->...sa', g, psi)
    lhs = L.wilson(Ug, 0.12, gpsi)
    rhs = np.einsum('...ab,...sb->...sa', g, L.wilson(U, 0.12, psi))
    assert np.allclose(lhs, rhs, atol=1e-13)


def test_flat_index_and_dense():
    dims = (2, 2, 2, 4)
    U = synth.su3_links(dims, 0.4, 9)
    psi = rand_field(dims, seed=3)
    f = L.flat(psi)
    # flat index 12 * s + 3 * spin + colour with s = x + Lx (y + Ly (z + Lz t))
    t, z, y, x, s, c = 3, 1, 0, 1, 2, 1
    assert f[12 * L.site_index(x, y, z, t, dims) + 3 * s + c] == psi[t, z, y, x, s, c]
    M = L.dense(lambda v: L.wilson(U, 0.1, v), dims)
    assert np.allclose(M @ f, L.flat(L.wilson(U, 0.1, psi)), atol=1e-13)


def test_link_generator():
    U = synth.su3_links(D4, 0.3, 1)
    UU = U @ np.conj(np.swapaxes(U, -1, -2))
    assert np.abs(UU - np.eye(3)).max() < 1e-14
    assert np.abs(np.linalg.det(U) - 1).max() < 1e-14
    # independent isotropic links: E[plaquette] = u0^4 with u0 = E[Re Tr U / 3]
    u0 = (np.trace(U, axis1=-2, axis2=-1).real / 3).mean()
    assert abs(synth.mean_plaquette(U) - u0 ** 4) < 0.01


def test_wilson_at_sites_equals_the_field_operator():
    """The per-site statement of Eq. xyz556 agrees with the whole-field one on a lattice with odd
    extents (every periodic wrap exercised)."""
    dims = (3, 5, 2, 7)
    U = synth.su3_links(dims, 0.5, 91)
    r = np.random.default_rng(92)
    psi = r.standard_normal(L.field_shape(dims)) + 1j * r.standard_normal(L.field_shape(dims))
    full = L.wilson(U, 0.13, psi)
    sites = [(t, z, y, x) for t in (0, 6) for z in (0, 1) for y in (0, 4) for x in (0, 2)] + [(3, 1, 2, 1)]
    got = L.wilson_at_sites(U, 0.13, psi, sites)
    for i, s in enumerate(sites):
        assert np.abs(got[i] - full[s]).max() < 1e-14
