"""CPU checks of the library's host dense routines (the per-cycle least squares, Schur, eigen and
generalised Hermitian eigen problems of GMRES-DR / MINRES-DR / GMRES-Proj) against numpy and
scipy on random and structured matrices.  The routines are compiled from the library's source
together with a small C harness (tests/native/dense_shim.cpp) by the host C++ compiler."""
import ctypes
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest
import scipy.linalg as sla

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1903_06986_gb300", "csrc")


@pytest.fixture(scope="module")
def lib():
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    out = os.path.join(tempfile.mkdtemp(prefix="dense_shim_"), "libdense_shim.so")
    # the library's host flags (complex products without the NaN-recovery path)
    subprocess.run([cxx, "-O2", "-std=c++17", "-fcx-fortran-rules", "-shared", "-fPIC", "-I", CSRC,
                    os.path.join(ROOT, "tests", "native", "dense_shim.cpp"), os.path.join(CSRC, "dense.cpp"),
                    "-o", out], check=True)
    return ctypes.CDLL(out)


def cbuf(a):
    return np.asfortranarray(a, dtype=np.complex128)


def ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def rand(r, c, seed):
    g = np.random.default_rng(seed)
    return g.standard_normal((r, c)) + 1j * g.standard_normal((r, c))


def test_lstsq_matches_numpy_on_hessenberg(lib):
    for m, seed in ((5, 1), (30, 2), (60, 3)):
        H = np.triu(rand(m + 1, m, seed), -1)              # (m+1) x m upper Hessenberg
        c = rand(m + 1, 1, seed + 10)[:, 0]
        A, x = cbuf(H), np.zeros(m, dtype=np.complex128)
        lib.shim_lstsq(ptr(A), m + 1, m, ptr(np.ascontiguousarray(c)), ptr(x))
        ref = np.linalg.lstsq(H, c, rcond=None)[0]
        # the minimal residual agrees to rounding; the minimiser within cond(H) times rounding
        assert abs(np.linalg.norm(c - H @ x) - np.linalg.norm(c - H @ ref)) <= 1e-12 * np.linalg.norm(c)
        # backward-stable: the normal equations hold to rounding of the size ||H||^2 ||x|| eps
        nH = np.linalg.norm(H, 2)
        assert np.linalg.norm(H.conj().T @ (c - H @ x)) <= 100 * m * 2.2e-16 * nH * (nH * np.linalg.norm(x)
                                                                                   + np.linalg.norm(c))
        assert np.linalg.norm(x - ref) <= 1e-14 * np.linalg.cond(H) * np.linalg.norm(ref) * m


def test_solve_matches_numpy_and_flags_singular(lib):
    A0 = rand(12, 12, 4)
    b = np.ascontiguousarray(rand(12, 1, 5)[:, 0])
    x = np.zeros(12, dtype=np.complex128)
    assert lib.shim_solve(ptr(cbuf(A0)), 12, ptr(b), ptr(x)) == 0
    ref = np.linalg.solve(A0, b)
    assert np.linalg.norm(x - ref) <= 1e-14 * np.linalg.cond(A0) * np.linalg.norm(ref) * 12
    S = A0.copy()
    S[:, 3] = 0.0                                          # a zero pivot
    assert lib.shim_solve(ptr(cbuf(S)), 12, ptr(b), ptr(x)) == 1


def test_schur_is_unitary_triangular_and_similar(lib):
    for n, seed in ((8, 6), (40, 7)):
        A = rand(n, n, seed)
        T, Z = np.zeros((n, n), dtype=np.complex128, order="F"), np.zeros((n, n), dtype=np.complex128, order="F")
        assert lib.shim_schur(ptr(cbuf(A)), n, ptr(T), ptr(Z)) == 0
        assert np.allclose(Z.conj().T @ Z, np.eye(n), atol=1e-12)
        assert np.abs(np.tril(T, -1)).max() < 1e-12 * np.abs(A).max()
        assert np.allclose(Z @ T @ Z.conj().T, A, atol=1e-11 * np.abs(A).max())


def test_eig_matches_scipy_eigenvalues_and_residuals(lib):
    n = 30
    A = rand(n, n, 8)
    w, X = np.zeros(n, dtype=np.complex128), np.zeros((n, n), dtype=np.complex128, order="F")
    assert lib.shim_eig(ptr(cbuf(A)), n, ptr(w), ptr(X)) == 0
    ref = sla.eigvals(A)
    for v in ref:                                          # same multiset of eigenvalues
        assert np.abs(w - v).min() < 1e-10 * np.abs(ref).max()
    assert np.allclose(np.linalg.norm(X, axis=0), 1.0, atol=1e-12)
    assert np.abs(A @ X - X * w).max() < 1e-10 * np.abs(A).max()


def test_eigh_and_generalised_eigh_match_scipy(lib):
    n = 25
    R = rand(n, n, 9)
    A = (R + R.conj().T) / 2
    w, X = np.zeros(n), np.zeros((n, n), dtype=np.complex128, order="F")
    assert lib.shim_eigh(ptr(cbuf(A)), n, ptr(w), ptr(X)) == 0
    assert np.allclose(w, sla.eigh(A, eigvals_only=True), atol=1e-11 * np.abs(w).max())
    assert np.allclose(X.conj().T @ X, np.eye(n), atol=1e-12)
    # Hermitian-definite pair, as in the harmonic Ritz problem H g = mu Hbar^H Hbar g
    Hb = np.triu(rand(n + 1, n, 10), -1)
    B = Hb.conj().T @ Hb
    mu, G = np.zeros(n), np.zeros((n, n), dtype=np.complex128, order="F")
    assert lib.shim_eigh_gen(ptr(cbuf(A)), ptr(cbuf(B)), n, ptr(mu), ptr(G)) == 0
    ref = sla.eigh(A, B, eigvals_only=True)
    assert np.allclose(mu, ref, rtol=1e-9, atol=1e-9 * np.abs(ref).max())
    assert np.allclose(G.conj().T @ B @ G, np.eye(n), atol=1e-9)
    assert np.abs(A @ G - B @ G * mu).max() < 1e-9 * np.abs(A).max() * np.abs(G).max()


def test_orthonormalize_spans_the_same_columns_in_order(lib):
    A = rand(50, 9, 11)
    Q = np.zeros((50, 9), dtype=np.complex128, order="F")
    lib.shim_orthonormalize(ptr(cbuf(A)), 50, 9, ptr(Q))
    assert np.allclose(Q.conj().T @ Q, np.eye(9), atol=1e-13)
    # Gram-Schmidt in column order: Q^H A is upper triangular (column j of A lies in span q_0..q_j)
    R = Q.conj().T @ A
    assert np.abs(np.tril(R, -1)).max() < 1e-12 * np.abs(A).max()
