"""Pins of the oracle's Krylov solvers against dense linear algebra: the minimum-residual property
of a GMRES cycle, convergence to the LU solution within cond * tol, harmonic Ritz values against
the dense spectrum (GMRES-DR on M, MINRES-DR form on M' = M gamma_5), the Arnoldi relation of
the deflation space, and the acceleration GMRES-Proj gets from it (Sec. 5.3, 7, 8)."""
import numpy as np
import pytest

from oracle import krylov as K, lattice as L, rng
from paper_1903_06986_gb300 import synth

DIMS = (2, 2, 2, 4)
KAPPA = 0.15


@pytest.fixture(scope="module")
def system():
    U = synth.su3_links(DIMS, 0.45, 21)
    M = L.dense(lambda v: L.wilson(U, KAPPA, v), DIMS)
    Mp = L.dense(lambda v: L.wilson_g5(U, KAPPA, v), DIMS)
    b = L.flat(rng.z4_noise(5, rng.NOISE_SPECIAL, DIMS))
    return U, M, Mp, b


def test_first_cycle_is_minimum_residual(system):
    U, M, Mp, b = system
    m = 8
    x, info, _ = K.gmres_dr(lambda v: M @ v, b, m, 0, 1e-30, 1)
    # dense least squares over K_m(M, b) = span(b, Mb, ..., M^{m-1} b)
    cols = [b]
    for _ in range(m - 1):
        cols.append(M @ cols[-1])
    Q, _ = np.linalg.qr(np.stack(cols, axis=1))
    y = np.linalg.lstsq(M @ Q, b, rcond=None)[0]
    assert np.linalg.norm(b - M @ x) <= np.linalg.norm(b - M @ (Q @ y)) * (1 + 1e-10)
    assert np.allclose(x, Q @ y, atol=1e-10)


def test_gmres_dr_converges_to_lu(system):
    U, M, Mp, b = system
    tol = 1e-12
    x, info, defl = K.gmres_dr(lambda v: M @ v, b, 30, 10, tol, 200)
    assert info["converged"] and info["true_resid"] < 10 * tol
    xe = np.linalg.solve(M, b)
    cond = np.linalg.cond(M)
    assert np.linalg.norm(x - xe) <= 10 * cond * tol * np.linalg.norm(xe)


def test_harmonic_ritz_match_dense_spectrum(system):
    U, M, Mp, b = system
    k = 10
    x, info, defl = K.gmres_dr(lambda v: M @ v, b, 40, k, 1e-13, 300)
    # the deflation space is an Arnoldi-like relation A V_k = V_{k+1} Hbar_k
    Vk1, Hk = defl["V"], defl["Hbar"]
    assert np.abs(M @ Vk1[:, :k] - Vk1 @ Hk).max() < 1e-11
    assert np.abs(Vk1.conj().T @ Vk1 - np.eye(k + 1)).max() < 1e-12
    lam, E, res = K.ritz_pairs(defl, hermitian=False)
    ev = np.linalg.eigvals(M)
    ev = ev[np.argsort(np.abs(ev))]
    for q in range(4):
        assert np.abs(ev - lam[q]).min() < 1e-7 * abs(lam[q])
    assert abs(abs(lam[0]) - abs(ev[0])) < 1e-7


def test_minres_dr_hermitian_eigenpairs(system):
    U, M, Mp, b = system
    k = 12
    y, info, defl = K.gmres_dr(lambda v: Mp @ v, b, 40, k, 1e-13, 300, hermitian=True)
    assert info["converged"]
    lam, E, res = K.ritz_pairs(defl, hermitian=True)
    assert np.abs(lam.imag).max() == 0.0
    w = np.linalg.eigvalsh(Mp)
    w = w[np.argsort(np.abs(w))]
    assert np.allclose(lam.real[:6], w[:6], rtol=1e-9, atol=1e-11)
    assert np.abs(E.conj().T @ E - np.eye(k)).max() < 1e-12
    for q in range(6):
        r = Mp @ E[:, q] - lam[q] * E[:, q]
        assert np.linalg.norm(r) < 1e-8
        assert abs(np.linalg.norm(r) - res[q]) < 1e-10
    # y solves M' y = b, so x = g5 y solves M x = b (Sec. 5.4)
    x = L.flat(L.g5(L.unflat(y, DIMS)))
    assert np.linalg.norm(M @ x - b) < 1e-11 * np.linalg.norm(b)


def test_gmres_proj_uses_deflation(system):
    U, M, Mp, b = system
    m, k = 30, 12
    _, _, defl = K.gmres_dr(lambda v: M @ v, b, m, k, 1e-13, 300)
    b2 = L.flat(rng.z4_noise(5, 3, DIMS))
    x, info = K.gmres_proj(lambda v: M @ v, b2, defl, m - k, 1e-11, 200)
    assert info["converged"]
    assert np.linalg.norm(M @ x - b2) <= 1e-11 * np.linalg.norm(b2) * 1.0001
    # plain restarted GMRES(m - k) needs more matrix-vector products
    xr, infor, _ = K.gmres_dr(lambda v: M @ v, b2, m - k, 0, 1e-11, 400)
    assert info["matvecs"] < infor["matvecs"]


def test_lanczos_window_on_hermitian_operator(system):
    """GMRES-Proj on M' = M gamma_5 with the inner cycles on the three-term Lanczos recurrence
    (window 2, Sec. 8's MINRES): the Hessenberg matrix of a cycle is tridiagonal and equals the full
    Arnoldi one to rounding (the dropped inner products vanish for a Hermitian operator), the Arnoldi
    relation holds, and the solve reaches the LU solution within cond * tol.  On the non-Hermitian
    M the same window changes the cycle: the window relies on hermiticity."""
    U, M, Mp, b = system
    n, m = b.shape[0], 16
    for A, herm in ((Mp, True), (M, False)):
        Hs, Vs = [], []
        for window in (0, 2):
            V = np.zeros((n, m + 1), dtype=np.complex128)
            H = np.zeros((m + 1, m), dtype=np.complex128)
            V[:, 0] = b / np.linalg.norm(b)
            K._arnoldi(lambda v: A @ v, V, H, 0, m, [0], window)
            assert np.abs(A @ V[:, :m] - V @ H).max() < 1e-12 * np.abs(A).max()
            Hs.append(H)
            Vs.append(V)
        assert np.abs(np.triu(Hs[1], 2)).max() == 0.0
        diff = np.abs(Hs[1] - Hs[0]).max() / np.abs(Hs[0]).max()
        if herm:
            assert diff < 1e-12
            assert np.abs(Vs[1].conj().T @ Vs[1] - np.eye(m + 1)).max() < 1e-10
        else:
            assert diff > 1e-3
    m_, k = 30, 12
    _, _, defl = K.gmres_dr(lambda v: Mp @ v, b, m_, k, 1e-13, 300, hermitian=True)
    b2 = L.flat(rng.z4_noise(5, 3, DIMS))
    tol = 1e-11
    x, info = K.gmres_proj(lambda v: Mp @ v, b2, defl, m_ - k, tol, 200, window=2)
    assert info["converged"]
    xe = np.linalg.solve(Mp, b2)
    assert np.linalg.norm(x - xe) <= 10 * np.linalg.cond(Mp) * tol * np.linalg.norm(xe)
