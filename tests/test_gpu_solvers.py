"""GPU parity of GMRES-DR, MINRES-DR and GMRES-Proj with the oracle (Sec. 5.3, 7, 8).

The GPU and the oracle run the same algorithm in different rounding orders, so iterates agree to
rounding after a fixed number of cycles, and converged solutions agree within cond(M) * tol.
Ritz values are checked against the dense spectrum; eigenvectors only where they are converged."""
import numpy as np
import pytest

from oracle import krylov as Kr, lattice as L, rng
from paper_1903_06986_gb300 import lqcd, synth
from tests.gpu_util import context, dev, host, rel_err

pytestmark = pytest.mark.gpu

DIMS = (4, 4, 4, 4)
KAPPA = 0.150


@pytest.fixture(scope="module")
def setup():
    U = synth.su3_links(DIMS, 0.3, 1)
    A = lambda v: L.flat(L.wilson(U, KAPPA, L.unflat(v, DIMS)))
    Ap = lambda v: L.flat(L.wilson_g5(U, KAPPA, L.unflat(v, DIMS)))
    b = L.flat(rng.z4_noise(1, rng.NOISE_SPECIAL, DIMS))
    M = L.dense(lambda f: L.wilson(U, KAPPA, f), DIMS)
    return dict(U=U, A=A, Ap=Ap, b=b, M=M, cond=np.linalg.cond(M), ctx=context(DIMS), Ud=dev(U))


@pytest.mark.parametrize("cycles", [1, 3])
def test_gmresdr_iterates_match_oracle(setup, cycles):
    s = setup
    x_ref, _, _ = Kr.gmres_dr(s["A"], s["b"], 20, 5, 1e-30, cycles)
    x, info, _ = s["ctx"].gmresdr_solve(s["Ud"], KAPPA, dev(L.unflat(s["b"], DIMS)), 20, 5, 1e-30, cycles)
    assert info["cycles"] == cycles
    assert rel_err(L.flat(host(x)), x_ref) < 1e-10


def test_gmresdr_converges_and_deflates(setup):
    s = setup
    tol = 1e-12
    x, info, defl = s["ctx"].gmresdr_solve(s["Ud"], KAPPA, dev(L.unflat(s["b"], DIMS)), 20, 5, tol, 500,
                                           want_defl=True)
    assert info["converged"] and info["true_resid"] <= tol
    xe = np.linalg.solve(s["M"], s["b"])
    assert np.linalg.norm(L.flat(host(x)) - xe) <= 10 * s["cond"] * tol * np.linalg.norm(xe)
    # the exported deflation space satisfies M V_k = V_{k+1} Hbar_k with orthonormal V_{k+1}
    ex = defl.export()
    V = host(ex["V"]).T
    H = ex["Hbar"]
    assert np.abs(V.conj().T @ V - np.eye(6)).max() < 1e-12
    assert np.abs(s["M"] @ V[:, :5] - V @ H).max() < 1e-10


def test_minresdr_ritz_values_and_solution(setup):
    s = setup
    tol = 1e-13
    y, info, defl = s["ctx"].minresdr_solve(s["Ud"], KAPPA, dev(L.unflat(s["b"], DIMS)), 40, 12, tol, 500,
                                            want_defl=True)
    assert info["converged"]
    x = L.flat(L.g5(host(y)))
    assert np.linalg.norm(s["M"] @ x - s["b"]) <= 1.01 * tol * np.linalg.norm(s["b"]) * 10
    ex = defl.export()
    lam, E, res = ex["lam"], host(ex["E"]).T, ex["eig_resid"]
    assert np.abs(lam.imag).max() == 0.0
    Mp = L.dense(lambda f: L.wilson_g5(s["U"], KAPPA, f), DIMS)
    w = np.linalg.eigvalsh(Mp)
    assert np.abs(E.conj().T @ E - np.eye(12)).max() < 1e-12
    for q in range(12):
        r = Mp @ E[:, q] - lam[q] * E[:, q]
        assert abs(np.linalg.norm(r) - res[q]) < 1e-9 + 1e-6 * res[q]
        # Hermitian: a Ritz value lies within its residual norm of an eigenvalue
        assert np.abs(w - lam[q].real).min() <= res[q] * (1 + 1e-8) + 1e-12
    # iterates after 2 cycles match the oracle's Hermitian form
    y_ref, _, _ = Kr.gmres_dr(s["Ap"], s["b"], 40, 12, 1e-30, 2, hermitian=True)
    y2, _, _ = s["ctx"].minresdr_solve(s["Ud"], KAPPA, dev(L.unflat(s["b"], DIMS)), 40, 12, 1e-30, 2)
    assert rel_err(L.flat(host(y2)), y_ref) < 1e-10


def test_gmres_proj_multi_rhs(setup):
    s = setup
    ctx = s["ctx"]
    _, _, defl = ctx.gmresdr_solve(s["Ud"], KAPPA, dev(L.unflat(s["b"], DIMS)), 20, 5, 1e-13, 500, want_defl=True)
    ex = defl.export()
    dref = dict(V=host(ex["V"]).T, Hbar=ex["Hbar"])
    etas = rng.z4_block(1, 0, 3, DIMS)
    # one cycle: identical algorithm on identical deflation data
    x1, _ = ctx.proj_solve(s["Ud"], KAPPA, defl, dev(etas), 15, 1e-30, 1)
    for r in range(3):
        xr, _ = Kr.gmres_proj(s["A"], L.flat(etas[r]), dref, 15, 1e-30, 1)
        assert rel_err(L.flat(host(x1)[r]), xr) < 1e-10
    # to convergence; every right-hand side meets the tolerance with its true residual
    tol = 1e-12
    x, info = ctx.proj_solve(s["Ud"], KAPPA, defl, dev(etas), 15, tol, 500)
    assert info["converged"] and info["true_resid"] <= tol
    for r in range(3):
        xe = np.linalg.solve(s["M"], L.flat(etas[r]))
        assert np.linalg.norm(L.flat(host(x)[r]) - xe) <= 10 * s["cond"] * tol * np.linalg.norm(xe)
    # solving one right-hand side alone gives the same answer
    xa, _ = ctx.proj_solve(s["Ud"], KAPPA, defl, dev(etas[1:2]), 15, tol, 500)
    assert rel_err(host(xa)[0], host(x)[1]) < 10 * s["cond"] * tol


@pytest.mark.parametrize("prec", [1, 2, 3], ids=["fp32", "fp16", "bf16"])
def test_mixed_precision_proj_reaches_fp64_tolerance(setup, prec):
    """FP64 defect correction around the FP32 / FP16 / BF16 GMRES-Proj: the FP64 true residual
    (recomputed here with the dense oracle matrix) meets 1e-10 and the solution agrees with the
    dense FP64 solve within cond * tol, like the plain FP64 path."""
    s = setup
    ctx = s["ctx"]
    _, _, defl = ctx.gmresdr_solve(s["Ud"], KAPPA, dev(L.unflat(s["b"], DIMS)), 20, 5, 1e-12, 500, want_defl=True)
    etas = rng.z4_block(2, 0, 4, DIMS)
    tol = 1e-10
    x, info = ctx.proj_solve(s["Ud"], KAPPA, defl, dev(etas), 15, tol, 500, prec=prec)
    assert info["converged"] and info["true_resid"] <= tol
    x64, _ = ctx.proj_solve(s["Ud"], KAPPA, defl, dev(etas), 15, tol, 500)
    for r in range(4):
        b = L.flat(etas[r])
        xm = L.flat(host(x)[r])
        assert np.linalg.norm(s["M"] @ xm - b) <= tol * np.linalg.norm(b) * 1.0001
        xe = np.linalg.solve(s["M"], b)
        assert np.linalg.norm(xm - xe) <= 10 * s["cond"] * tol * np.linalg.norm(xe)
        assert np.linalg.norm(xm - L.flat(host(x64)[r])) <= 20 * s["cond"] * tol * np.linalg.norm(xe)


@pytest.mark.parametrize("prec", [lqcd.PREC_F16, lqcd.PREC_BF16, lqcd.PREC_F32], ids=["f16", "bf16", "f32"])
def test_lanczos_window_inner_cycles_on_hermitian_operator(setup, prec):
    """Mixed-precision GMRES-Proj on M' = M gamma_5 (the Hermitian path) with the inner cycles
    orthogonalising each vector against the last two only (the Lanczos recurrence of MINRES-DR,
    Sec. 8): the FP64 true residual (dense oracle matrix) meets 1e-10, and the solution agrees with
    the dense solve and with full Gram-Schmidt within cond * tol."""
    s = setup
    ctx = s["ctx"]
    _, _, defl = ctx.minresdr_solve(s["Ud"], KAPPA, dev(L.unflat(s["b"], DIMS)), 40, 12, 1e-12, 500, want_defl=True)
    Mp = L.dense(lambda f: L.wilson_g5(s["U"], KAPPA, f), DIMS)
    cond = np.linalg.cond(Mp)
    etas = rng.z4_block(3, 0, 4, DIMS)
    tol = 1e-10
    ctx.set_inner_window(0)
    x_full, info_full = ctx.proj_solve(s["Ud"], KAPPA, defl, dev(etas), 30, tol, 500, prec=prec)
    ctx.set_inner_window(2)
    try:
        x, info = ctx.proj_solve(s["Ud"], KAPPA, defl, dev(etas), 30, tol, 500, prec=prec)
    finally:
        ctx.set_inner_window(0)
    assert info["converged"] and info["true_resid"] <= tol
    assert info_full["converged"]
    for r in range(4):
        b = L.flat(etas[r])
        xm = L.flat(host(x)[r])
        assert np.linalg.norm(Mp @ xm - b) <= tol * np.linalg.norm(b) * 1.0001
        xe = np.linalg.solve(Mp, b)
        assert np.linalg.norm(xm - xe) <= 10 * cond * tol * np.linalg.norm(xe)
        assert np.linalg.norm(xm - L.flat(host(x_full)[r])) <= 20 * cond * tol * np.linalg.norm(xe)


def test_lanczos_window_rejects_bad_values(setup):
    ctx = setup["ctx"]
    with pytest.raises(Exception):
        ctx.set_inner_window(1)
    with pytest.raises(Exception):
        ctx.set_inner_window(-3)
    ctx.set_inner_window(0)


@pytest.mark.parametrize("hermitian", [False, True], ids=["gmresdr", "minresdr"])
def test_polynomial_preconditioned_solve_matches_lu(hermitian):
    """A solve with a polynomial right preconditioner (Krylov on A p(A), x = p(A) y) returns the
    LU solution of A x = b within cond * tol, and its deflation space satisfies the Arnoldi relation
    of the dense A p(A)."""
    dims, kappa = (2, 2, 2, 4), 0.12
    U = synth.su3_links(dims, 0.45, 2)
    ctx = context(dims)
    b = ctx.noise_z4(9, 0, 1)
    A = L.dense(lambda v: (L.wilson_g5 if hermitian else L.wilson)(U, kappa, v), dims)
    a = np.array([1.9, -0.8, 0.25, -0.03], dtype=np.complex128)
    solve = ctx.minresdr_solve if hermitian else ctx.gmresdr_solve
    x, info, defl = solve(dev(U), kappa, b, 30, 6, 1e-13, max_cycles=300, want_defl=True, poly=a)
    assert info["converged"] and info["true_resid"] <= 1e-13
    bh = host(b)[0].reshape(-1)
    xe = np.linalg.solve(A, bh)
    assert np.linalg.norm(host(x)[0].reshape(-1) - xe) <= 10 * np.linalg.cond(A) * 1e-13 * np.linalg.norm(xe)
    B = A @ sum(a[j] * np.linalg.matrix_power(A, j) for j in range(len(a)))
    ex = defl.export()
    V = host(ex["V"]).reshape(7, -1).T
    assert np.abs(B @ V[:, :6] - V @ ex["Hbar"]).max() < 1e-12 * np.abs(B).max()
    defl.close()
