"""Pins of the oracle's even/odd preconditioning (Sec. 7) against dense linear algebra:
  * P couples only opposite parities on even extents (the block structure the method relies on);
  * the reduced matrix equals the Schur complement of the dense M's even/odd blocks;
  * reduced solve + reconstruction = dense LU solution of M x = b;
  * the full eigenpairs formed from the reduced ones satisfy M v = lambda v and give the whole
    spectrum of M; ES built from them has valid left vectors (Sec. 5.3, 7).
"""
import numpy as np
import pytest

from oracle import evenodd as EO, lattice as L, rng, subtract as S
from paper_1903_06986_gb300 import synth

DIMS = (2, 2, 2, 4)


def _perm(dims):
    """Flat unknown indices ordered (even sites, odd sites), 12 unknowns per site."""
    par = EO.parity(dims).reshape(-1)
    sites = np.concatenate([np.nonzero(par == 0)[0], np.nonzero(par == 1)[0]])
    return (12 * sites[:, None] + np.arange(12)[None, :]).reshape(-1)


def _reduced_dense(U, kappa, dims):
    nh = 12 * L.volume(dims) // 2
    cols = []
    for j in range(nh):
        e = np.zeros(nh, dtype=np.complex128)
        e[j] = 1.0
        cols.append(EO.reduced_apply(U, kappa, e.reshape(-1, 4, 3), dims).reshape(-1))
    return np.stack(cols, axis=1)


def test_hopping_couples_opposite_parities_only():
    U = synth.su3_links(DIMS, 0.5, 51)
    P = L.dense(lambda v: L.hop(U, v), DIMS)[np.ix_(_perm(DIMS), _perm(DIMS))]
    nh = P.shape[0] // 2
    assert np.abs(P[:nh, :nh]).max() == 0.0 and np.abs(P[nh:, nh:]).max() == 0.0
    assert np.abs(P[:nh, nh:]).max() > 0.1


def test_split_join_roundtrip_and_odd_extent_rejected():
    psi = rng.z4_noise(3, 0, DIMS)
    pe, po = EO.split(psi, DIMS)
    assert np.array_equal(EO.join(pe, po, DIMS), psi)
    with pytest.raises(ValueError):
        EO.split(np.zeros(L.field_shape((3, 2, 2, 2))), (3, 2, 2, 2))


def test_reduced_matrix_is_schur_complement():
    U = synth.su3_links(DIMS, 0.5, 52)
    kappa = 0.14
    M = L.dense(lambda v: L.wilson(U, kappa, v), DIMS)[np.ix_(_perm(DIMS), _perm(DIMS))]
    nh = M.shape[0] // 2
    schur = M[:nh, :nh] - M[:nh, nh:] @ np.linalg.solve(M[nh:, nh:], M[nh:, :nh])
    assert np.abs(_reduced_dense(U, kappa, DIMS) - schur).max() < 1e-13


def test_reduced_solve_reconstructs_full_solution():
    U = synth.su3_links(DIMS, 0.5, 53)
    kappa = 0.15
    b = rng.z4_noise(4, 0, DIMS)
    Mh = _reduced_dense(U, kappa, DIMS)
    xe = np.linalg.solve(Mh, EO.reduced_rhs(U, kappa, b, DIMS).reshape(-1)).reshape(-1, 4, 3)
    x = EO.reconstruct(U, kappa, xe, b, DIMS)
    M = L.dense(lambda v: L.wilson(U, kappa, v), DIMS)
    ref = L.unflat(np.linalg.solve(M, L.flat(b)), DIMS)
    assert np.abs(x - ref).max() < 1e-11 * np.abs(ref).max()


def test_full_eigenpairs_from_reduced_ones():
    U = synth.su3_links(DIMS, 0.45, 54)
    kappa = 0.15
    mu, Ve = np.linalg.eig(_reduced_dense(U, kappa, DIMS))
    lam, vecs = EO.full_eigenpairs(U, kappa, mu, Ve.T.reshape(len(mu), -1, 4, 3), DIMS)
    for q in range(len(lam)):
        r = L.wilson(U, kappa, vecs[q]) - lam[q] * vecs[q]
        assert np.linalg.norm(r) < 1e-10
    full = np.linalg.eigvals(L.dense(lambda v: L.wilson(U, kappa, v), DIMS))
    assert len(lam) == len(full)
    d = np.abs(lam[:, None] - full[None, :])
    assert d.min(axis=1).max() < 1e-8 and d.min(axis=0).max() < 1e-8
    # ES from the smallest full pairs (Sec. 7): left vectors from gamma_5-hermiticity are valid
    order = np.argsort(np.abs(lam))
    ER = L.flat(vecs[order]).T
    EL, found = S.es_left_vectors(ER, lam[order], DIMS)
    M = L.dense(lambda v: L.wilson(U, kappa, v), DIMS)
    sel = np.nonzero(found)[0][:20]
    assert len(sel) == 20
    res = EL[:, sel].conj().T @ M - lam[order][sel, None] * EL[:, sel].conj().T
    assert np.abs(res).max() < 1e-9 * np.abs(M).max()


def test_full_eigenpairs_reject_reduced_eigenvalue_one():
    """mu = 1 means 1 - lambda = 0: the odd part kappa P_oe v_e / (1 - lambda) does not exist, so the
    oracle refuses instead of returning non-finite vectors (and accepts mu just away from 1)."""
    U = synth.su3_links(DIMS, 0.45, 55)
    ve = np.zeros((1, 12 * L.volume(DIMS) // 2 // 12, 4, 3), dtype=np.complex128)
    ve[0, 0, 0, 0] = 1.0
    with pytest.raises(ValueError):
        EO.full_eigenpairs(U, 0.15, np.array([1.0 + 0j]), ve, DIMS)
    with pytest.raises(ValueError):
        EO.full_eigenpairs(U, 0.15, np.array([1.0 + 1e-18j]), ve, DIMS)
    lam, vecs = EO.full_eigenpairs(U, 0.15, np.array([1.0 - 1e-6 + 0j]), ve, DIMS)
    assert np.all(np.isfinite(vecs)) and np.all(np.isfinite(lam))
