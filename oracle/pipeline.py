"""The whole loop-estimate path on one gauge configuration, step by step (Sec. 5, 7).

Test infrastructure (see ``oracle/__init__.py``).

  1. special right-hand side b0 = Z(4) noise NOISE_SPECIAL:
       GMRES-DR(m, k) on M   -> deflation space (V_{k+1}, Hbar_k) for GMRES-Proj,
       MINRES-DR(m, k) on M' -> Q = k eigenpairs (lambda'_q, e'_q) of M' for HFES;
     with system="MG5" (the Hermitian path) only the MINRES-DR solve runs, and its space also
     serves the noise solves, done on M' y = eta with x = gamma_5 y (reading: the paper moves to
     the Hermitian system and MINRES-DR at kappa_crit, Sec. 8; a field whose spectrum of M
     surrounds the origin needs that for the noise solves too);
     ES (Sec. 5.3) uses the Rayleigh-Ritz pairs of M on the GMRES-DR space with left vectors from
     gamma_5-hermiticity (subtract.es_left_vectors); on the Hermitian path there is no space of M
     and ES subtracts nothing;
  2. Min-Res polynomial coefficients a from the noise NOISE_POLY (Sec. 5.2);
  3. hopping traces t_k by probing (Sec. 5.1); 1/xi'_q for HFPS and HFPOLY (Sec. 5.5);
  4. for every noise n: eta = Z(4) noise n, x = M^{-1} eta by GMRES-Proj, and for every mode the
     subtraction vector tilde x; the noise terms eta^dag Theta (x - tilde x) per timeslice;
  5. add-backs and the summary (mean, error bar) per mode and operator.
"""
import time

import numpy as np

from . import estimate as E
from . import krylov as Kr
from . import lattice as L
from . import operators as O
from . import rng
from . import subtract as S


def prec_coeffs(Asolve, b, degree, hermitian):
    """Coefficients of the polynomial preconditioner p of the noise solves (Sec. 5.2's Min-Res
    polynomial, of the solver's operator A, on the noise b): p(A) ~ A^{-1}.  For Hermitian A the
    Min-Res coefficients are real (b^dag A^j b is real), and their real parts are taken so that
    A p(A) is exactly Hermitian."""
    a = S.poly_coeffs(Asolve, b, degree)
    return a.real.astype(np.complex128) if hermitian else a


def setup(U, kappa, dims, seed, m, k, K, npoly, tol_special, max_cycles=2000, eig_tol=None, system="M",
          prec_degree=0):
    A = lambda v: L.flat(L.wilson(U, kappa, L.unflat(v, dims)))
    Ap = lambda v: L.flat(L.wilson_g5(U, kappa, L.unflat(v, dims)))
    b0 = L.flat(rng.z4_noise(seed, rng.NOISE_SPECIAL, dims))
    if system not in ("M", "MG5"):
        raise ValueError(system)
    # polynomial preconditioning (reading: the outlook of Sec. 5.2 / 10, POLY combined with deflation
    # inside the solver): the Krylov solves of the noise system work on B = A p(A), x = p(A) y
    Asolve = Ap if system == "MG5" else A
    ap = None
    Bsolve = Asolve
    if prec_degree > 0:
        ap = prec_coeffs(Asolve, L.flat(rng.z4_noise(seed, rng.NOISE_POLY, dims)), prec_degree, system == "MG5")
        Bsolve = lambda v: Asolve(S.poly_apply(Asolve, ap, v))
    if system == "M":
        _, info_m, defl_m = Kr.gmres_dr(Bsolve, b0, m, k, tol_special, max_cycles, eig_tol=eig_tol)
        _, info_h, defl_h = Kr.gmres_dr(Ap, b0, m, k, tol_special, max_cycles, hermitian=True, eig_tol=eig_tol)
    else:
        _, info_h, defl_h = Kr.gmres_dr(Bsolve, b0, m, k, tol_special, max_cycles, hermitian=True, eig_tol=eig_tol)
        info_m, defl_m = info_h, defl_h
    lam, Ev, eres = Kr.ritz_pairs(defl_h, hermitian=True)
    if system == "MG5" and ap is not None:
        # Ritz vectors of B' = M' p(M') are those of M' (B' is a function of M'): the eigenvalues of M'
        # are their Rayleigh quotients, ordered by |lambda'|, with residuals ||M' e - lambda' e||
        ME = np.stack([Ap(Ev[:, q]) for q in range(Ev.shape[1])], axis=1)
        lam = np.einsum('iq,iq->q', Ev.conj(), ME).real.astype(np.complex128)
        order = np.argsort(np.abs(lam), kind='stable')
        lam, Ev, ME = lam[order], Ev[:, order], ME[:, order]
        eres = np.linalg.norm(ME - Ev * lam[None, :], axis=0)
    Af = lambda f: L.wilson(U, kappa, f)
    a = S.poly_coeffs(Af, rng.z4_noise(seed, rng.NOISE_POLY, dims), npoly)
    t = S.hop_traces(U, kappa, max(K, npoly + 1), dims)
    pert = lambda f: S.hop_series(U, kappa, f, K)
    poly = lambda f: S.poly_apply(Af, a, f)
    xi_p = S.xi_inverse(Ev, pert, dims)
    xi_q = S.xi_inverse(Ev, poly, dims)
    es = None
    if system == "M" and ap is None:
        lam_m, Er, _ = Kr.ritz_pairs(defl_m, hermitian=False)
        El, found = S.es_left_vectors(Er, lam_m, dims)
        es = (Er[:, found], El[:, found], lam_m[found])
    return dict(A=A, Ap=Ap, system=system, defl_m=defl_m, info_m=info_m, info_h=info_h, lam=lam, Ev=Ev, eig_resid=eres,
                es=es, Asolve=Asolve, Bsolve=Bsolve, prec_a=ap,
                a=a, b=S.a_to_b(a), t=t, xi_pert=xi_p, xi_poly=xi_q, pert=pert, poly=poly)


def addbacks(U, kappa, dims, st, K):
    lam, Ev = st["lam"], st["Ev"]
    add = dict(none=np.zeros((O.NOPS,) + L.site_shape(dims), dtype=np.complex128),
               pert=S.pert_addback(st["t"], kappa, K),
               poly=S.poly_addback(st["t"], kappa, st["b"]),
               defl=S.defl_addback(U, kappa, Ev, 1 / lam, dims))
    add["defl_pert"] = add["pert"] + S.defl_addback(U, kappa, Ev, 1 / lam - st["xi_pert"], dims)
    add["defl_poly"] = add["poly"] + S.defl_addback(U, kappa, Ev, 1 / lam - st["xi_poly"], dims)
    add["es"] = S.es_addback(U, kappa, *st["es"], dims) if st["es"] is not None else add["none"].copy()
    return add


def subtraction_vector(mode, st, eta):
    lam, Ev = st["lam"], st["Ev"]
    if mode == "none":
        return np.zeros_like(eta)
    if mode == "pert":
        return st["pert"](eta)
    if mode == "poly":
        return st["poly"](eta)
    if mode == "defl":
        return S.defl_vector(Ev, 1 / lam, eta)
    if mode == "defl_pert":
        return st["pert"](eta) + S.defl_vector(Ev, 1 / lam - st["xi_pert"], eta)
    if mode == "defl_poly":
        return st["poly"](eta) + S.defl_vector(Ev, 1 / lam - st["xi_poly"], eta)
    if mode == "es":
        return S.es_vector(*st["es"], eta) if st["es"] is not None else np.zeros_like(eta)
    raise ValueError(mode)


def solve_noises(st, dims, seed, first, count, m_inner, tol, max_cycles=2000):
    xs, infos = [], []
    for n in range(first, first + count):
        eta = L.flat(rng.z4_noise(seed, n, dims))
        # solve B y = eta over the space of B (B = A, or A p(A) with polynomial preconditioning; its
        # relative residual is that of x = p(A) y for A x = eta), then x = gamma_5 x' on the Hermitian path
        y, info = Kr.gmres_proj(st["Bsolve"], eta, st["defl_m"], m_inner, tol, max_cycles)
        if st["prec_a"] is not None:
            y = S.poly_apply(st["Asolve"], st["prec_a"], y)
        xs.append(L.g5(L.unflat(y, dims)) if st["system"] == "MG5" else L.unflat(y, dims))
        infos.append(info)
    return np.stack(xs), infos


def loop_estimate(U, kappa, dims, seed, nnoise, m, k, K, npoly, tol, tol_special, modes=E.MODES, eig_tol=None,
                  system="M", prec_degree=0):
    """Run steps 1-5; returns (results per mode, setup state, timing).  eig_tol: see krylov.gmres_dr;
    system: "M" or "MG5" (step 1); prec_degree: polynomial preconditioning of the noise solves."""
    t0 = time.perf_counter()
    st = setup(U, kappa, dims, seed, m, k, K, npoly, tol_special, eig_tol=eig_tol, system=system,
               prec_degree=prec_degree)
    add = addbacks(U, kappa, dims, st, K)
    t1 = time.perf_counter()
    xs, infos = solve_noises(st, dims, seed, 0, nnoise, m - k, tol)
    etas = rng.z4_block(seed, 0, nnoise, dims)
    out = {}
    for mode in modes:
        ws = xs - np.stack([subtraction_vector(mode, st, e) for e in etas])
        out[mode] = E.summarize(E.noise_terms(U, kappa, etas, ws), O.per_t(add[mode]))
        out[mode]["addback_t"] = O.per_t(add[mode])
    t2 = time.perf_counter()
    return out, st, dict(setup_s=t1 - t0, noise_s=t2 - t1, solve_infos=infos)


def loop_derivs(U, kappa, dims, seed, nnoise, m, k, K, tol, tol_special, max_cycles=2000, eig_tol=None):
    """Derivatives of the loop estimates (see oracle/derivs.py), step by step: GMRES-DR on M for the
    special right-hand side; per noise x = M^{-1} eta, y = M^{-1} P x and z = M^{-dag} eta by
    GMRES-Proj; per-noise d/dkappa of the NS and PS estimates of the nine operators (PS add-back
    derivative included) and the mean link gradient of the NS scalar estimate.
    Returns dict(per_noise=[2, n, op], link_grad=(4, T, Z, Y, X, 8))."""
    from . import derivs as Dv
    A = lambda v: L.flat(L.wilson(U, kappa, L.unflat(v, dims)))
    b0 = L.flat(rng.z4_noise(seed, rng.NOISE_SPECIAL, dims))
    _, _, defl = Kr.gmres_dr(A, b0, m, k, tol_special, max_cycles, eig_tol=eig_tol)
    solve = lambda f: L.unflat(Kr.gmres_proj(A, L.flat(f), defl, m - k, tol, max_cycles)[0], dims)
    t = S.hop_traces(U, kappa, K, dims)
    dadd = O.per_t(Dv.dpert_addback(t, kappa, K)).sum(axis=-1)
    per = np.zeros((2, nnoise, O.NOPS), dtype=np.complex128)
    grad = np.zeros(U.shape[:-2] + (8,), dtype=np.complex128)
    for n in range(nnoise):
        eta = rng.z4_noise(seed, n, dims)
        x = solve(eta)
        y = solve(L.hop(U, x))
        z = L.g5(solve(L.g5(eta)))
        d_none = Dv.dkappa_densities(U, kappa, eta, x, y).sum(axis=(-1, -2, -3, -4))
        xt = S.hop_series(U, kappa, eta, K)
        dxt = Dv.dpert_vector(U, kappa, eta, K)
        d_pert = Dv.dkappa_densities(U, kappa, eta, x - xt, y - dxt).sum(axis=(-1, -2, -3, -4))
        per[0, n] = d_none
        per[1, n] = d_pert + dadd
        grad += Dv.link_gradient(U, kappa, x, z) / nnoise
    return dict(per_noise=per, link_grad=grad)
