"""Deflated restarted Krylov solvers: GMRES-DR, its Hermitian form (MINRES-DR) and GMRES-Proj.

Test infrastructure (see ``oracle/__init__.py``).

The paper uses these solvers without restating them (Sec. 1, 5.3, 7, 8): GMRES-DR(m, k) for the
first ("super-convergence") right-hand side, whose last cycle yields k harmonic Ritz vectors;
GMRES-Proj for every later right-hand side (a minimum-residual projection over that deflation
space alternating with GMRES cycles); MINRES-DR for the Hermitian M' = M gamma_5 (Sec. 8).  The
steps below are Morgan's published GMRES-DR cycle, in the paper's notation where it has one:

  1. r = b - A x;  c = ||r|| e_1;  v_1 = r / ||r||.
  2. Arnoldi from column j0 (0 on the first cycle, k after a restart) to m, with classical
     Gram-Schmidt applied twice:  A V_m = V_{m+1} Hbar_m.
  3. d = argmin || c - Hbar_m d ||;  x += V_m d;  s = c - Hbar_m d (the residual in V_{m+1}).
  4. Harmonic Ritz pairs of H_m:  (H_m + |h_{m+1,m}|^2 H_m^{-H} e_m e_m^T) g = theta g;  keep the k
     with smallest |theta|.
  5. P_{k+1} = orthonormal basis of [g_1 .. g_k (padded with a zero row), w], w spanning the
     orthogonal complement of range(Hbar_m) (reading: s is orthogonal to range(Hbar_m), so in exact
     arithmetic it is parallel to w = [-conj(h_{m+1,m}) H_m^{-H} e_m; 1]; every harmonic Ritz
     residual Hbar_m g - theta [g; 0] is parallel to w too, which is what makes step 6 exact.  Once
     the system has converged, s is rounding noise and its direction is not w's, so w is used).
  6. V_{k+1} <- V_{m+1} P_{k+1};  Hbar_k <- P_{k+1}^H Hbar_m P_k;  c <- P_{k+1}^H s;  go to 2 with j0 = k.
  The cycles stop when the residual is below tol and, if eig_tol is given, every Rayleigh-Ritz
  residual of the deflation space (below) is below eig_tol as well: the "super-convergence" of the
  first right-hand side, solved far below its tolerance so that the eigenvectors converge (Sec. 5.4, 7).

Hermitian form (reading; the paper cites MINRES-DR without restating it): the same cycle on a
Hermitian A, minimum residual over the same spaces; the harmonic Ritz values theta of step 4 are
real for Hermitian A and are taken as such (their rounding-level imaginary parts dropped), and the
final Rayleigh-Ritz problem is solved as a Hermitian one.  Step 4 is solved in its general form,
not as the equivalent Hermitian-definite problem H_m g = (1/theta) Hbar_m^H Hbar_m g with H_m
symmetrised: with the symmetrised H_m the vectors g satisfy step 6's relation only to the rounding
asymmetry of H_m, and over long runs that error grew by a factor of ~1.23 per cycle (4^4 lattice,
GMRES-DR(20,5) on M gamma_5: ||A V_k - V_{k+1} Hbar_k|| from 1e-16 to 1e-2 in 200 cycles), while
the general form keeps it at rounding level.

Eigenpairs for deflation (reading of "smallest" eigenvalues, Sec. 5.4): after the final cycle the
deflation space V_k is Rayleigh-Ritz'd, T = V_k^H A V_k = (Hbar_k)_{1:k,1:k}, eigenvalues ordered by
increasing |lambda|.
"""
import numpy as np
import scipy.linalg as sla


def _cgs2(V, w):
    """Classical Gram-Schmidt twice of w against the columns of V; returns (h, w_orth)."""
    h = V.conj().T @ w
    w = w - V @ h
    h2 = V.conj().T @ w
    w = w - V @ h2
    return h + h2, w


def _arnoldi(A, V, H, j0, m, counter, window=0):
    """Extend A V[:, :m] = V[:, :m+1] H[:m+1, :m] from column j0 (columns < j0 already valid).
    window > 0 (Hermitian A only): orthogonalise against the last `window` columns; with window 2 this
    is the three-term Lanczos recurrence of MINRES (Sec. 8), whose other Hessenberg entries vanish
    in exact arithmetic for Hermitian A, and H is tridiagonal."""
    for j in range(j0, m):
        w = A(V[:, j])
        counter[0] += 1
        lo = max(0, j + 1 - window) if window > 0 else 0
        h, w = _cgs2(V[:, lo:j + 1], w)
        H[lo:j + 1, j] = h
        nrm = np.linalg.norm(w)
        H[j + 1, j] = nrm
        V[:, j + 1] = w / nrm if nrm > 0 else 0.0


def harmonic_ritz(Hbar, k, hermitian=False):
    """Step 4: k harmonic Ritz pairs (theta, g) of the (m+1) x m Hessenberg Hbar, smallest |theta| first."""
    m = Hbar.shape[1]
    Hm = Hbar[:m, :m]
    em = np.zeros(m, dtype=np.complex128)
    em[-1] = 1.0
    f = np.linalg.solve(Hm.conj().T, em)
    F = Hm + (abs(Hbar[m, m - 1]) ** 2) * np.outer(f, em)
    theta, G = np.linalg.eig(F)
    if hermitian:
        theta = theta.real.astype(np.complex128)
    order = np.argsort(np.abs(theta), kind='stable')[:k]
    return theta[order], G[:, order]


def lsq_complement(Hbar):
    """Unit vector w spanning the orthogonal complement of range(Hbar) for an (m+1) x m Hbar with
    nonsingular H_m: Hbar^H w = 0 gives w = [-conj(h_{m+1,m}) H_m^{-H} e_m; 1], normalised."""
    m = Hbar.shape[1]
    em = np.zeros(m, dtype=np.complex128)
    em[-1] = 1.0
    f = np.linalg.solve(Hbar[:m, :m].conj().T, em)
    w = np.concatenate([-np.conj(Hbar[m, m - 1]) * f, [1.0 + 0j]])
    return w / np.linalg.norm(w)


def _restart_basis(G, w):
    """Step 5: orthonormal P_{k+1} from the k harmonic Ritz coordinate vectors and the vector w."""
    m1 = w.shape[0]
    k = G.shape[1]
    Gp = np.zeros((m1, k), dtype=np.complex128)
    Gp[:m1 - 1, :] = G
    Q, _ = np.linalg.qr(Gp)
    t = w - Q @ (Q.conj().T @ w)
    t = t - Q @ (Q.conj().T @ t)
    t = t / np.linalg.norm(t)
    return np.concatenate([Q, t[:, None]], axis=1)


def gmres_dr(A, b, m, k, tol, max_cycles, x0=None, hermitian=False, eig_tol=None):
    """GMRES-DR(m, k) (MINRES-DR form when hermitian=True) for A x = b.

    Returns (x, info, defl) where defl = dict(V=V_{k+1}, Hbar=Hbar_k, theta=harmonic Ritz values)
    is the deflation space of the final cycle (A V_k = V_{k+1} Hbar_k), used by GMRES-Proj and
    by `ritz_pairs`.  info: cycles, matvecs, resid (per-cycle recursive relative residual norms),
    eig_resid (largest Rayleigh-Ritz residual of the final space), true_resid (relative),
    converged (residual below tol, and the eigen residuals below eig_tol when it is given).
    """
    n = b.shape[0]
    x = np.zeros(n, dtype=np.complex128) if x0 is None else x0.astype(np.complex128).copy()
    bnorm = np.linalg.norm(b)
    counter = [0]
    r = b - A(x) if x0 is not None else b.astype(np.complex128).copy()
    if x0 is not None:
        counter[0] += 1
    V = np.zeros((n, m + 1), dtype=np.complex128)
    H = np.zeros((m + 1, m), dtype=np.complex128)
    beta = np.linalg.norm(r)
    V[:, 0] = r / beta
    c = np.zeros(m + 1, dtype=np.complex128)
    c[0] = beta
    j0 = 0
    hist = []
    converged = False
    defl = None
    cycles = 0
    for cyc in range(max_cycles):
        cycles = cyc + 1
        _arnoldi(A, V, H, j0, m, counter)
        d = np.linalg.lstsq(H, c, rcond=None)[0]
        x = x + V[:, :m] @ d
        s = c - H @ d
        rel = np.linalg.norm(s) / bnorm
        hist.append(rel)
        theta, G = harmonic_ritz(H, k, hermitian)
        P = _restart_basis(G, lsq_complement(H))
        Vn = V @ P
        Hn = P.conj().T @ H @ P[:m, :k]
        defl = dict(V=Vn.copy(), Hbar=Hn.copy(), theta=theta.copy())
        eres = ritz_pairs(defl, hermitian)[2].max() if k > 0 else 0.0
        if rel <= tol and (eig_tol is None or eres <= eig_tol):
            converged = True
            break
        V[:, :k + 1] = Vn
        V[:, k + 1:] = 0.0
        H[:, :] = 0.0
        H[:k + 1, :k] = Hn
        c = np.zeros(m + 1, dtype=np.complex128)
        c[:k + 1] = P.conj().T @ s
        j0 = k
    true = np.linalg.norm(b - A(x)) / bnorm
    counter[0] += 1
    info = dict(cycles=cycles, matvecs=counter[0], resid=hist, eig_resid=eres, true_resid=true,
                converged=converged)
    return x, info, defl


def ritz_pairs(defl, hermitian=True):
    """Rayleigh-Ritz eigenpairs on span(V_k) of a deflation space: returns (lam, E, resid) with
    E = V_k Y (orthonormal columns when hermitian), ordered by increasing |lam|, and the eigen
    residual norms ||A e - lam e|| = ||Hbar_k y - lam [y; 0]||."""
    Vk1, Hk = defl["V"], defl["Hbar"]
    k = Hk.shape[1]
    T = Hk[:k, :k]
    if hermitian:
        lam, Y = np.linalg.eigh(0.5 * (T + T.conj().T))
        lam = lam.astype(np.complex128)
    else:
        lam, Y = np.linalg.eig(T)
    order = np.argsort(np.abs(lam), kind='stable')
    lam, Y = lam[order], Y[:, order]
    E = Vk1[:, :k] @ Y
    Ypad = np.vstack([Y, np.zeros((1, k))])
    res = np.linalg.norm(Hk @ Y - Ypad * lam[None, :], axis=0)
    return lam, E, res


def gmres_proj(A, b, defl, m_inner, tol, max_cycles, window=0):
    """GMRES-Proj for a later right-hand side (Sec. 5.3, 7): alternately (i) minimum-residual
    projection over the deflation space, d = argmin || V_{k+1}^H r - Hbar_k d ||, x += V_k d,
    r -= V_{k+1} Hbar_k d; and (ii) one GMRES(m_inner) cycle from r (on the Lanczos recurrence when
    window = 2 and A is Hermitian, see ``_arnoldi``).  Stops when the recursive residual is below
    tol * ||b||, then re-checks with the true residual (continuing from it if the recursion drifted)."""
    n = b.shape[0]
    Vk1, Hk = defl["V"], defl["Hbar"]
    k = Hk.shape[1]
    bnorm = np.linalg.norm(b)
    x = np.zeros(n, dtype=np.complex128)
    r = b.astype(np.complex128).copy()
    counter = [0]
    hist = []
    converged = False
    cycles = 0
    for cyc in range(max_cycles):
        cycles = cyc + 1
        cp = Vk1.conj().T @ r
        dp = np.linalg.lstsq(Hk, cp, rcond=None)[0]
        x = x + Vk1[:, :k] @ dp
        r = r - Vk1 @ (Hk @ dp)
        beta = np.linalg.norm(r)
        if beta <= tol * bnorm:
            hist.append(beta / bnorm)
            rt = b - A(x)
            counter[0] += 1
            if np.linalg.norm(rt) / bnorm <= tol:
                converged = True
                break
            r = rt
            beta = np.linalg.norm(r)
        V = np.zeros((n, m_inner + 1), dtype=np.complex128)
        H = np.zeros((m_inner + 1, m_inner), dtype=np.complex128)
        V[:, 0] = r / beta
        _arnoldi(A, V, H, 0, m_inner, counter, window)
        c = np.zeros(m_inner + 1, dtype=np.complex128)
        c[0] = beta
        d = np.linalg.lstsq(H, c, rcond=None)[0]
        x = x + V[:, :m_inner] @ d
        r = V @ (c - H @ d)
        rel = np.linalg.norm(r) / bnorm
        hist.append(rel)
        if rel <= tol:
            rt = b - A(x)
            counter[0] += 1
            if np.linalg.norm(rt) / bnorm <= tol:
                converged = True
                break
            r = rt
    true = np.linalg.norm(b - A(x)) / bnorm
    counter[0] += 1
    info = dict(cycles=cycles, matvecs=counter[0], resid=hist, true_resid=true, converged=converged)
    return x, info
