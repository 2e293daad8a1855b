"""Pins of the oracle's whole-path composition (oracle/pipeline.py) against dense linear algebra.

Every function of the pipeline is checked against matrices built here from the definitions,
independently of the pipeline's own code paths:
  * setup: the GMRES-DR space satisfies the Arnoldi relation of the dense M, the MINRES-DR pairs
    are eigenpairs of the dense M' = M gamma_5 (Sec. 5.4), the Min-Res coefficients satisfy the
    normal equations for the noise NOISE_POLY (Sec. 5.2), t_k equals Tr(Theta P^k) of dense
    powers for every k the add-backs need (Sec. 5.1), and 1/xi'_q for PS and POLY equals
    e'^dag gamma_5 tilde M^{-1} e' with dense tilde M^{-1} (Sec. 5.5);
  * subtraction_vector applies, and addbacks traces, the dense tilde M^{-1} of each mode;
  * solve_noises solves M x = eta for the right noise indices;
  * loop_estimate: every per-noise value equals eta^dag Theta (M^{-1} - tilde M^{-1}) eta +
    Tr(Theta tilde M^{-1}) from dense matrices, the estimators are unbiased for the dense-LU trace
    and their sample variance follows Eq. xyz255 (Sec. 3-5);
  * loop_derivs: per-noise d/dkappa values equal the dense-matrix derivative of the same per-noise
    estimate (central differences in kappa), the mean is unbiased for d Tr(Theta M^{-1})/dkappa, and
    the link gradient matches finite differences of the mean scalar estimate.
"""
import numpy as np
import pytest

from oracle import derivs as Dv, estimate as E, exact, lattice as L, operators as O, pipeline as PL, rng
from paper_1903_06986_gb300 import synth

DIMS = (2, 2, 2, 4)
KAPPA = 0.12
SEED = 5
M_DR, K_DR, K_PS, NPOLY = 40, 8, 7, 7   # NPOLY + 1 > K_PS: the add-backs need t_k for k <= NPOLY


def dense(apply):
    return L.dense(apply, DIMS)


@pytest.fixture(scope="module")
def dense_ops():
    U = synth.su3_links(DIMS, 0.45, 61)
    M = exact.dense_M(U, KAPPA, DIMS)
    P = dense(lambda v: L.hop(U, v))
    G5 = dense(L.g5)
    Minv = np.linalg.inv(M)
    thetas = [exact.dense_theta(U, KAPPA, op, DIMS) for op in range(O.NOPS)]
    return dict(U=U, M=M, P=P, G5=G5, Minv=Minv, thetas=thetas)


@pytest.fixture(scope="module")
def state(dense_ops):
    # super-converged (Ritz residuals <= 1e-12) so that the Ritz values of M come in conjugate pairs
    # to the pairing tolerance of the ES left vectors
    return PL.setup(dense_ops["U"], KAPPA, DIMS, SEED, M_DR, K_DR, K_PS, NPOLY, 1e-14, eig_tol=1e-12)


def tilde_dense(d, st):
    """The six tilde M^{-1} of Sec. 5 from dense matrices and the setup's coefficients."""
    n = d["M"].shape[0]
    pert = sum(np.linalg.matrix_power(KAPPA * d["P"], k) for k in range(K_PS))
    poly = sum(st["a"][j] * np.linalg.matrix_power(d["M"], j) for j in range(NPOLY + 1))
    Ev, lam = st["Ev"], st["lam"]
    D = lambda w: d["G5"] @ Ev @ np.diag(w) @ Ev.conj().T
    out = dict(none=np.zeros((n, n), dtype=np.complex128), pert=pert, poly=poly, defl=D(1 / lam))
    out["defl_pert"] = pert + D(1 / lam - st["xi_pert"])
    out["defl_poly"] = poly + D(1 / lam - st["xi_poly"])
    if st["es"] is not None:
        Er, El, lm = st["es"]
        out["es"] = Er @ np.diag(1 / lm) @ El.conj().T
    else:
        out["es"] = np.zeros((n, n), dtype=np.complex128)
    return out


def test_setup_spaces_are_those_of_the_dense_operator(dense_ops, state):
    d, st = dense_ops, state
    assert st["info_m"]["converged"] and st["info_m"]["true_resid"] <= 1e-13
    # GMRES-DR space on M: A V_k = V_{k+1} Hbar_k with orthonormal V_{k+1}
    V, H = st["defl_m"]["V"], st["defl_m"]["Hbar"]
    assert V.shape == (d["M"].shape[0], K_DR + 1) and H.shape == (K_DR + 1, K_DR)
    assert np.abs(V.conj().T @ V - np.eye(K_DR + 1)).max() < 1e-12
    assert np.abs(d["M"] @ V[:, :K_DR] - V @ H).max() < 1e-12
    # MINRES-DR pairs are eigenpairs of the dense M' within the residuals reported
    Mp = d["M"] @ d["G5"]
    Ev, lam = st["Ev"], st["lam"]
    res = np.linalg.norm(Mp @ Ev - Ev * lam[None, :], axis=0)
    assert np.all(res <= st["eig_resid"] + 1e-12)
    assert np.abs(Ev.conj().T @ Ev - np.eye(K_DR)).max() < 1e-12
    assert np.all(np.abs(lam.imag) == 0.0)
    # Ritz values lie within their residual of an eigenvalue of the dense M'
    w = np.linalg.eigvalsh(Mp)
    for q in range(K_DR):
        assert np.abs(w - lam[q].real).min() <= st["eig_resid"][q] + 1e-12


def test_setup_polynomial_uses_the_poly_noise(dense_ops, state):
    """The Min-Res normal equations hold for the noise NOISE_POLY of the seed (Sec. 5.2, reading 8)
    and fail for another noise; b is the same polynomial in powers of kappa P."""
    d, st = dense_ops, state
    a = st["a"]

    def normal_residual(b):
        r = b - d["M"] @ sum(a[j] * np.linalg.matrix_power(d["M"], j) @ b for j in range(NPOLY + 1))
        cols = [np.linalg.matrix_power(d["M"], j + 1) @ b for j in range(NPOLY + 1)]
        return max(abs(np.vdot(c, r)) / (np.linalg.norm(c) * np.linalg.norm(b)) for c in cols)

    assert normal_residual(L.flat(rng.z4_noise(SEED, rng.NOISE_POLY, DIMS))) < 1e-10
    assert normal_residual(L.flat(rng.z4_noise(SEED, rng.NOISE_SPECIAL, DIMS))) > 1e-4
    pa = sum(a[j] * np.linalg.matrix_power(d["M"], j) for j in range(NPOLY + 1))
    pb = sum(st["b"][k] * np.linalg.matrix_power(KAPPA * d["P"], k) for k in range(NPOLY + 1))
    assert np.abs(pa - pb).max() < 1e-10 * np.abs(pa).max()


def test_setup_hopping_traces_and_xi(dense_ops, state):
    d, st = dense_ops, state
    Kt = max(K_PS, NPOLY + 1)
    assert st["t"].shape[0] == Kt
    for k in range(Kt):
        Pk = np.linalg.matrix_power(d["P"], k)
        for op in range(O.NOPS):
            ref = np.trace(d["thetas"][op] @ Pk)
            assert abs(st["t"][k][op].sum() - ref) < 1e-9 * max(1.0, abs(ref)), (k, op)
    td = tilde_dense(d, st)
    for q in range(K_DR):
        e = st["Ev"][:, q]
        assert abs(st["xi_pert"][q] - np.vdot(e, d["G5"] @ td["pert"] @ e)) < 1e-12
        assert abs(st["xi_poly"][q] - np.vdot(e, d["G5"] @ td["poly"] @ e)) < 1e-11
    assert np.abs(st["xi_pert"] - st["xi_poly"]).max() > 1e-6     # the two are distinct


def test_subtraction_vectors_and_addbacks_are_the_dense_matrices(dense_ops, state):
    d, st = dense_ops, state
    td = tilde_dense(d, st)
    add = PL.addbacks(d["U"], KAPPA, DIMS, st, K_PS)
    eta = rng.z4_noise(SEED, 3, DIMS)
    for mode in E.MODES:
        got = L.flat(PL.subtraction_vector(mode, st, eta))
        ref = td[mode] @ L.flat(eta)
        assert np.abs(got - ref).max() < 1e-11 * max(1.0, np.abs(ref).max()), mode
        for op in range(O.NOPS):
            ref = np.trace(d["thetas"][op] @ td[mode])
            assert abs(add[mode][op].sum() - ref) < 1e-10 * max(1.0, abs(ref)), (mode, op)


def test_es_space_gives_left_and_right_eigenvectors_of_the_dense_matrix(dense_ops, state):
    """ES data of the setup (Sec. 5.3): Ritz pairs of M on the GMRES-DR space with left vectors from
    gamma_5-hermiticity, every kept pair an eigen-triple of the dense M within its Ritz residual,
    closed under conjugation, and e_L^dag e_R = 1."""
    d, st = dense_ops, state
    Er, El, lm = st["es"]
    assert len(lm) >= 4
    for q in range(len(lm)):
        rr = np.linalg.norm(d["M"] @ Er[:, q] - lm[q] * Er[:, q])
        rl = np.linalg.norm(El[:, q].conj() @ d["M"] - lm[q] * El[:, q].conj())
        assert rr < 1e-10 and rl < 1e-8 * np.linalg.norm(El[:, q])
        assert abs(np.vdot(El[:, q], Er[:, q]) - 1) < 1e-12
        assert np.abs(lm - np.conj(lm[q])).min() <= 1e-8 * abs(lm[q])


def test_solve_noises_solves_the_right_systems(dense_ops, state):
    d, st = dense_ops, state
    xs, infos = PL.solve_noises(st, DIMS, SEED, 7, 3, M_DR - K_DR, 1e-13)
    cond = np.linalg.cond(d["M"])
    for i in range(3):
        assert infos[i]["converged"]
        x = d["Minv"] @ L.flat(rng.z4_noise(SEED, 7 + i, DIMS))
        assert np.linalg.norm(L.flat(xs[i]) - x) <= 10 * cond * 1e-13 * np.linalg.norm(x)


@pytest.fixture(scope="module")
def estimate(dense_ops):
    out, st, _ = PL.loop_estimate(dense_ops["U"], KAPPA, DIMS, SEED, 200, M_DR, K_DR, K_PS, NPOLY, 1e-13, 1e-14)
    return out, st


def test_loop_estimate_per_noise_values_are_the_dense_formula(dense_ops, estimate):
    """Per noise n and mode: eta_n^dag Theta (M^{-1} - tilde M^{-1}) eta_n + Tr(Theta tilde M^{-1})."""
    d = dense_ops
    out, st = estimate
    td = tilde_dense(d, st)
    for n in (0, 1, 57, 199):
        eta = L.flat(rng.z4_noise(SEED, n, DIMS))
        for mode in E.MODES:
            Q = d["Minv"] - td[mode]
            for op in range(O.NOPS):
                ref = np.vdot(eta, d["thetas"][op] @ Q @ eta) + np.trace(d["thetas"][op] @ td[mode])
                got = out[mode]["per_noise"][n, op]
                assert abs(got - ref) < 1e-9 * max(1.0, abs(ref)), (n, mode, op)


def test_loop_estimate_unbiased_with_exact_variance(dense_ops, estimate):
    d = dense_ops
    out, st = estimate
    td = tilde_dense(d, st)
    N = out["none"]["per_noise"].shape[0]
    exact_tr = exact.exact_traces(d["U"], KAPPA, DIMS, d["Minv"])
    for mode in E.MODES:
        for op in range(O.NOPS):
            _, vre, vim = exact.z4_variance(d["thetas"][op] @ (d["Minv"] - td[mode]))
            var = vre if O.OP_PART[op] == 0 else vim
            sig = exact_tr[op].real if O.OP_PART[op] == 0 else exact_tr[op].imag
            assert abs(out[mode]["signal"][op] - sig) <= 5 * np.sqrt(var / N) + 1e-10, (mode, op)
            svar = (out[mode]["stderr"][op] ** 2) * N
            if var > 1e-20:
                assert 0.6 < svar / var < 1.6, (mode, op, svar, var)
            assert abs(out[mode]["addback_t"][op].sum() - np.trace(d["thetas"][op] @ td[mode])) < 1e-10 * max(
                1.0, abs(np.trace(d["thetas"][op] @ td[mode]))), (mode, op)


@pytest.fixture(scope="module")
def derivs(dense_ops):
    return PL.loop_derivs(dense_ops["U"], KAPPA, DIMS, SEED, 40, M_DR, K_DR, K_PS, 1e-13, 1e-14)


def _per_noise_dense(U, kappa, eta):
    """NS and PS per-noise estimates of the nine operators from dense matrices at this kappa."""
    M = exact.dense_M(U, kappa, DIMS)
    P = dense(lambda v: L.hop(U, v))
    Minv = np.linalg.inv(M)
    pert = sum(np.linalg.matrix_power(kappa * P, k) for k in range(K_PS))
    ns, ps = [], []
    for op in range(O.NOPS):
        Th = exact.dense_theta(U, kappa, op, DIMS)
        ns.append(np.vdot(eta, Th @ Minv @ eta))
        ps.append(np.vdot(eta, Th @ (Minv - pert) @ eta) + np.trace(Th @ pert))
    return np.array(ns), np.array(ps)


def test_loop_derivs_per_noise_match_dense_central_differences(dense_ops, derivs):
    U, h = dense_ops["U"], 1e-5
    for n in (0, 13, 39):
        eta = L.flat(rng.z4_noise(SEED, n, DIMS))
        ns_p, ps_p = _per_noise_dense(U, KAPPA + h, eta)
        ns_m, ps_m = _per_noise_dense(U, KAPPA - h, eta)
        fd_ns, fd_ps = (ns_p - ns_m) / (2 * h), (ps_p - ps_m) / (2 * h)
        assert np.abs(derivs["per_noise"][0, n] - fd_ns).max() < 1e-6 * max(1.0, np.abs(fd_ns).max()), n
        assert np.abs(derivs["per_noise"][1, n] - fd_ps).max() < 1e-6 * max(1.0, np.abs(fd_ps).max()), n


def test_loop_derivs_unbiased_and_link_gradient(dense_ops, derivs):
    d = dense_ops
    U = d["U"]
    ex = Dv.exact_dkappa(U, KAPPA, DIMS)
    per = derivs["per_noise"]
    N = per.shape[1]
    for mode in range(2):
        for op in range(O.NOPS):
            part = per[mode, :, op].real if O.OP_PART[op] == 0 else per[mode, :, op].imag
            want = ex[op].real if O.OP_PART[op] == 0 else ex[op].imag
            err = part.std(ddof=1) / np.sqrt(N)
            assert abs(part.mean() - want) <= 5 * err + 1e-9, (mode, op)
    # link gradient of the mean NS scalar estimate (1/N) sum_n eta_n^dag M^{-1} eta_n
    etas = [L.flat(rng.z4_noise(SEED, n, DIMS)) for n in range(N)]
    Eta = np.stack(etas, axis=1)
    T = lambda UU: np.mean(np.sum(Eta.conj() * np.linalg.solve(exact.dense_M(UU, KAPPA, DIMS), Eta), axis=0))
    r = np.random.default_rng(11)
    h = 1e-5
    for _ in range(4):
        mu = int(r.integers(4))
        site = tuple(int(r.integers(n)) for n in L.site_shape(DIMS))
        a = int(r.integers(8))
        fd = (T(Dv.perturb_link(U, mu, site, a, h)) - T(Dv.perturb_link(U, mu, site, a, -h))) / (2 * h)
        got = derivs["link_grad"][(mu,) + site + (a,)]
        assert abs(got - fd) < 1e-6 * max(1.0, abs(fd)), (mu, site, a)


def test_hermitian_path_solves_and_estimates(dense_ops):
    """system="MG5": one MINRES-DR space serves the eigenpairs and the noise solves (M' y = eta,
    x = gamma_5 y); the solutions are those of M x = eta and the per-noise values follow the same
    dense formula."""
    d = dense_ops
    st = PL.setup(d["U"], KAPPA, DIMS, SEED, M_DR, K_DR, K_PS, NPOLY, 1e-14, system="MG5")
    assert st["defl_m"] is not None and st["info_m"] is st["info_h"]
    xs, infos = PL.solve_noises(st, DIMS, SEED, 2, 3, M_DR - K_DR, 1e-13)
    cond = np.linalg.cond(d["M"])
    for i in range(3):
        assert infos[i]["converged"]
        x = d["Minv"] @ L.flat(rng.z4_noise(SEED, 2 + i, DIMS))
        assert np.linalg.norm(L.flat(xs[i]) - x) <= 10 * cond * 1e-13 * np.linalg.norm(x)
    out, st2, _ = PL.loop_estimate(d["U"], KAPPA, DIMS, SEED, 3, M_DR, K_DR, K_PS, NPOLY, 1e-13, 1e-14,
                                   system="MG5")
    td = tilde_dense(d, st2)
    for n in range(3):
        eta = L.flat(rng.z4_noise(SEED, n, DIMS))
        for mode in E.MODES:
            for op in (0, 4, 8):
                Th = d["thetas"][op]
                ref = np.vdot(eta, Th @ (d["Minv"] - td[mode]) @ eta) + np.trace(Th @ td[mode])
                assert abs(out[mode]["per_noise"][n, op] - ref) < 1e-9 * max(1.0, abs(ref)), (n, mode, op)


@pytest.mark.parametrize("system", ["M", "MG5"])
def test_polynomial_preconditioned_solves(dense_ops, system):
    """prec_degree = 4: the noise solves work on B = A p(A) (A = M, or M' on the Hermitian path) with
    p the Min-Res polynomial of A on the polynomial noise; the GMRES-DR space is one of the dense B,
    the HFES eigenpairs are eigenpairs of the dense M', the solutions are the LU ones, the per-noise
    values follow the dense formula, and the preconditioned solves need fewer Krylov steps."""
    d = dense_ops
    A = d["M"] @ d["G5"] if system == "MG5" else d["M"]
    st = PL.setup(d["U"], KAPPA, DIMS, SEED, M_DR, K_DR, K_PS, NPOLY, 1e-14, system=system, prec_degree=4)
    a = st["prec_a"]
    if system == "MG5":
        assert np.all(a.imag == 0.0)
    pA = sum(a[j] * np.linalg.matrix_power(A, j) for j in range(len(a)))
    B = A @ pA
    b = L.flat(rng.z4_noise(SEED, rng.NOISE_POLY, DIMS))
    cols = [np.linalg.matrix_power(A, j + 1) @ b for j in range(len(a))]
    r = b - B @ b
    assert max(abs(np.vdot(c, r)) / (np.linalg.norm(c) * np.linalg.norm(b)) for c in cols) < 1e-6
    V, H = st["defl_m"]["V"], st["defl_m"]["Hbar"]
    assert np.abs(B @ V[:, :K_DR] - V @ H).max() < 1e-11
    Mp = d["M"] @ d["G5"]
    res = np.linalg.norm(Mp @ st["Ev"] - st["Ev"] * st["lam"][None, :], axis=0)
    assert np.all(res <= st["eig_resid"] + 1e-12)
    xs, infos = PL.solve_noises(st, DIMS, SEED, 0, 2, M_DR - K_DR, 1e-12)
    cond = np.linalg.cond(d["M"])
    for i in range(2):
        x = d["Minv"] @ L.flat(rng.z4_noise(SEED, i, DIMS))
        assert np.linalg.norm(L.flat(xs[i]) - x) <= 10 * cond * 1e-12 * np.linalg.norm(x)
    st_plain = PL.setup(d["U"], KAPPA, DIMS, SEED, M_DR, K_DR, K_PS, NPOLY, 1e-14, system=system)
    _, infos_plain = PL.solve_noises(st_plain, DIMS, SEED, 0, 2, M_DR - K_DR, 1e-12)
    steps = lambda inf: sum(len(i["resid"]) for i in inf)
    assert steps(infos) < steps(infos_plain)
    out, st2, _ = PL.loop_estimate(d["U"], KAPPA, DIMS, SEED, 2, M_DR, K_DR, K_PS, NPOLY, 1e-12, 1e-14,
                                   system=system, prec_degree=4)
    td = tilde_dense(d, st2)
    for n in range(2):
        eta = L.flat(rng.z4_noise(SEED, n, DIMS))
        for mode in E.MODES:
            for op in (0, 4, 8):
                Th = d["thetas"][op]
                ref = np.vdot(eta, Th @ (d["Minv"] - td[mode]) @ eta) + np.trace(Th @ td[mode])
                assert abs(out[mode]["per_noise"][n, op] - ref) < 1e-8 * max(1.0, abs(ref)), (n, mode, op)
