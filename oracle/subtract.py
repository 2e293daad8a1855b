"""Subtraction matrices tilde M^{-1} of Sec. 5 and their trace add-backs.

Test infrastructure (see ``oracle/__init__.py``).

  PS      tilde x = sum_{k=0}^{K-1} (kappa P)^k eta            (Sec. 5.1; "seventh order" = K = 7 terms)
  POLY    tilde x = sum_{j=0}^{n} a_j M^j eta, a from the Min-Res projection (Sec. 5.2)
  ES      tilde x = V_R Lambda^{-1} V_L^dag eta                  (Sec. 5.3; left vectors from gamma_5-hermiticity)
  HFES    tilde x = gamma_5 V' Lambda'^{-1} V'^dag eta          (Sec. 5.4)
  HFPS /  tilde x = tilde x_{pert|poly} + gamma_5 V' (Lambda'^{-1} - Xi^{-1}) V'^dag eta,
  HFPOLY  1/xi'_q = e'_q^dag gamma_5 tilde M^{-1}_{pert|poly} e'_q (Sec. 5.5, reading of tilde M'^{-1} = gamma_5 tilde M^{-1})

Add-backs Tr(Theta tilde M^{-1}) (Sec. 5.1-5.5) are returned as per-site densities over the base
site of each operator (see ``operators.densities``).  The hopping traces t_k(Theta) = Tr(Theta P^k)
are taken from the exact diagonal by probing: with probe vectors z_c = sum over a colour class
of unit vectors e_i, every off-diagonal term e_i^dag Theta P^k e_j (i != j in one class) vanishes
when distinct members of a class are further apart (taxicab, on the torus) than k + 1 hops, so
sum_c densities(z_c, P^k z_c) is the exact diagonal density.  With every site its own class this
is the paper's sum_i e_i^dag Theta tilde M^{-1} e_i (Sec. 5.1) term by term.
"""
import math

import numpy as np

from . import lattice as L
from . import operators as O


def hop_series(U, kappa, eta, K):
    """PS: sum_{k=0}^{K-1} (kappa P)^k eta."""
    term = eta.copy()
    acc = eta.copy()
    for _ in range(1, K):
        term = kappa * L.hop(U, term)
        acc = acc + term
    return acc


def poly_coeffs(A, b, n):
    """Min-Res polynomial P_n(M) = sum_{j=0}^n a_j M^j (Eq. xyz646): a minimises ||b - M P_n(M) b||.
    The paper writes the normal equations (v^dag v) a = v^dag b with v = (Mb, M^2 b, .., M^{n+1} b);
    reading: their solution is computed by a Householder QR of v (same minimiser, stable)."""
    cols = []
    w = b.copy()
    for _ in range(n + 1):
        w = A(w)
        cols.append(w.ravel())
    v = np.stack(cols, axis=1)
    Q, R = np.linalg.qr(v)
    a = np.linalg.solve(R, Q.conj().T @ b.ravel())
    return a


def poly_apply(A, a, eta):
    """POLY: sum_j a_j M^j eta, powers applied one after another."""
    term = eta.copy()
    acc = a[0] * eta
    for j in range(1, len(a)):
        term = A(term)
        acc = acc + a[j] * term
    return acc


def a_to_b(a):
    """Coefficients of the same polynomial in powers of kappa P (Sec. 5.2): with M = 1 - kappa P,
    M^j = sum_k C(j, k) (-kappa P)^k, so b_k = (-1)^k sum_{j >= k} C(j, k) a_j.  (The text's
    'M = I + kappa P' at this point contradicts Eq. xyz556; reading: Eq. xyz556 holds.)"""
    n = len(a) - 1
    b = np.zeros(n + 1, dtype=np.complex128)
    for k in range(n + 1):
        for j in range(k, n + 1):
            b[k] += ((-1) ** k) * math.comb(j, k) * a[j]
    return b


def probe_classes(dims, spacing):
    """Colour class of each site for probing with periods spacing = (px, py, pz, pt), each dividing
    the extent: class = (x mod px, y mod py, z mod pz, t mod pt).  Returns (class_of_site (T,Z,Y,X), n_classes)."""
    lx, ly, lz, lt = dims
    px, py, pz, pt = spacing
    t, z, y, x = np.meshgrid(np.arange(lt), np.arange(lz), np.arange(ly), np.arange(lx), indexing='ij')
    cls = (x % px) + px * ((y % py) + py * ((z % pz) + pz * (t % pt)))
    return cls, px * py * pz * pt


def default_spacing(dims, K):
    """Smallest period >= K + 1 dividing each extent (paths of up to K-1 hops plus the one hop of
    a point-split operator then never join two members of a class), else the full extent."""
    out = []
    for l in dims:
        p = l
        for cand in range(K + 1, l):
            if l % cand == 0:
                p = cand
                break
        out.append(p)
    return tuple(out)


def hop_traces(U, kappa, K, dims, spacing=None, batch=256):
    """Per-site densities of t_k(Theta) = Tr(Theta P^k) for k = 0..K-1 and all nine operators.
    Returns t[k, op, T, Z, Y, X] (complex).  kappa only enters the point-split operators' own
    kappa prefactor (Table Table903)."""
    if spacing is None:
        spacing = default_spacing(dims, K)
    cls, ncls = probe_classes(dims, spacing)
    out = np.zeros((K, O.NOPS) + L.site_shape(dims), dtype=np.complex128)
    probes = [(c, a) for c in range(ncls) for a in range(12)]
    for i0 in range(0, len(probes), batch):
        chunk = probes[i0:i0 + batch]
        z = np.zeros(L.field_shape(dims, (len(chunk),)), dtype=np.complex128)
        for b_, (c, a) in enumerate(chunk):
            z[b_][cls == c, a // 3, a % 3] = 1.0
        w = z.copy()
        for k in range(K):
            if k > 0:
                w = L.hop(U, w)
            out[k] += O.densities(U, kappa, z, w).sum(axis=1)
    return out


def _member_distance(dims, spacing, c):
    """Torus taxicab distance of every site to the nearest member of Cartesian class c (members:
    x_mu = c_mu mod p_mu); per axis the nearest residue, summed (the members form a product lattice)."""
    px, py, pz, pt = spacing
    cx, cy, cz, ct = c % px, (c // px) % py, (c // (px * py)) % pz, c // (px * py * pz)
    t, z, y, x = np.meshgrid(*[np.arange(l) for l in reversed(dims)], indexing='ij')
    d = 0
    for coord, r, p in ((x, cx, px), (y, cy, py), (z, cz, pz), (t, ct, pt)):
        a = (coord - r) % p
        d = d + np.minimum(a, p - a)
    return d


def _member_owner(dims, spacing, c):
    """Site index (T, Z, Y, X tuple of arrays) of the member of class c nearest to every site."""
    px, py, pz, pt = spacing
    cs = (c % px, (c // px) % py, (c // (px * py)) % pz, c // (px * py * pz))
    t, z, y, x = np.meshgrid(*[np.arange(l) for l in reversed(dims)], indexing='ij')
    own = []
    for coord, r, p, l in zip((x, y, z, t), cs, (px, py, pz, pt), dims):
        a = (coord - r) % p
        own.append((coord - np.where(a <= p // 2, a, a - p)) % l)
    return own[3], own[2], own[1], own[0]


def hop_traces_meet(U, kappa, K, dims, spacing=None, completion_radius=None):
    """Meet-in-the-middle form of ``hop_traces`` (Sec. 5.1 add-back), the same densities t[k, op, site].

    With h = ceil((K - 1) / 2) and probe fields W_j = P^j z_c (j <= h) of each colour class c:
      * local operators (scalar, gamma_mu), every order k = j1 + j2 with j2 = min(k, h):
        by gamma_5-hermiticity of P, (P^j1)_{x,y} = g5 [(P^j1)_{y,x}]^dag g5, so
        tr[Gamma (P^k)_{xx}] = sum_y tr[Gamma g5 B_j1(y)^dag g5 B_j2(y)], where B_j(y) is the 12 x 12
        block (P^j)_{y,x} read off the 12 probes of the class at site y, and x is the class member
        nearest y (members are more than 2h hops apart, so every nonzero block has one member);
      * point-split operators, orders k > h: the contraction reads P^k z only at the members and
        their neighbours, so P^k z is needed only within R_k = max(1, K - k) hops of a member and
        is formed as P applied to P^(k-1) z, then cut to that neighbourhood (``completion_radius``
        overrides R_k, to show that a smaller one changes the result).
    The probing classes are Cartesian with the periods of ``default_spacing``."""
    if spacing is None:
        spacing = default_spacing(dims, K)
    h = (K - 1 + 1) // 2
    cls, ncls = probe_classes(dims, spacing)
    out = np.zeros((K, O.NOPS) + L.site_shape(dims), dtype=np.complex128)
    I3 = np.eye(3, dtype=np.complex128)
    g5 = np.kron(L.G5, I3)
    gam = [np.eye(12, dtype=np.complex128)] + [np.kron(L.G[mu], I3) for mu in range(4)]
    nsite = L.volume(dims)
    for c in range(ncls):
        z = np.zeros(L.field_shape(dims, (12,)), dtype=np.complex128)
        for a in range(12):
            z[a][cls == c, a // 3, a % 3] = 1.0
        W = [z]
        for j in range(1, h + 1):
            W.append(L.hop(U, W[-1]))
        # blocks B_j[site, comp, probe]
        B = [w.reshape(12, nsite, 12).transpose(1, 2, 0) for w in W]
        owner = _member_owner(dims, spacing, c)
        for k in range(K):
            j2 = min(k, h)
            j1 = k - j2
            M1 = np.einsum('ab,scb,cd->sad', g5, B[j1].conj(), g5)      # (P^j1)_{x,y}: [site y, a, comp]
            for op in range(5):
                q = np.einsum('ba,sac,scb->s', gam[op], M1, B[j2]).reshape(L.site_shape(dims))
                np.add.at(out[k, op], owner, q)
        dist = _member_distance(dims, spacing, c)
        w = z
        for k in range(K):
            if k > 0:
                w = L.hop(U, w)
                if k > h:
                    r = max(1, K - k) if completion_radius is None else completion_radius(K, k)
                    w = np.where((dist <= r)[None, ..., None, None], w, 0.0)
            d = O.densities(U, kappa, z, w).sum(axis=1)
            out[k, 5:] += d[5:]
    return out


def pert_addback(t, kappa, K):
    """PS add-back densities: sum_{k<K} kappa^k t_k."""
    return sum((kappa ** k) * t[k] for k in range(K))


def poly_addback(t, kappa, b):
    """POLY add-back densities: sum_k b_k kappa^k t_k."""
    return sum(b[k] * (kappa ** k) * t[k] for k in range(len(b)))


def defl_coeffs(E, X):
    """C = V'^dag eta (Sec. 5.4) for the Q columns of E (N_dim, Q) and the fields X (n, ...):
    C[q, r] = sum_i conj(E[i, q]) X_r[i].  Returns (Q, n)."""
    xf = X.reshape(X.shape[0], -1)
    return E.conj().T @ xf.T


def defl_expand(E, Cm):
    """Y_r = sum_q E[:, q] C[q, r] (the V' C of Sec. 5.4) as (n, N_dim) rows."""
    return (E @ Cm).T


def defl_vector(E, dvals, eta):
    """gamma_5 V' diag(dvals) V'^dag eta for fields eta (..., T, Z, Y, X, 4, 3); E is (N_dim, Q)."""
    dims_shape = eta.shape[-6:]
    ef = eta.reshape(eta.shape[:-6] + (-1,))
    c = ef @ E.conj()                     # (..., Q) = V'^dag eta
    y = (c * dvals) @ E.T                 # (..., N_dim)
    return L.g5(y.reshape(eta.shape[:-6] + dims_shape))


def defl_addback(U, kappa, E, dvals, dims):
    """Densities of Tr(Theta gamma_5 V' diag(dvals) V'^dag) = sum_q dvals_q e'_q^dag Theta gamma_5 e'_q."""
    out = np.zeros((O.NOPS,) + L.site_shape(dims), dtype=np.complex128)
    for q in range(E.shape[1]):
        e = L.unflat(E[:, q], dims)
        out += dvals[q] * O.densities(U, kappa, e, L.g5(e))
    return out


def es_left_vectors(ER, lam, dims, rel_tol=1e-8):
    """Left eigenvectors for ES (Sec. 5.3) from right eigenvectors of the gamma_5-hermitian M.

    M^dag = gamma_5 M gamma_5 turns a right eigenvector of lambda* into a left eigenvector of
    lambda: e_L(lambda_q) = gamma_5 e_R(lambda_p) / conj(e_R(lambda_p)^dag gamma_5 e_R(lambda_q)) with
    lambda_p = conj(lambda_q), normalised so that e_L^dag e_R = 1.  ER: (N_dim, Q) right
    eigenvectors, lam: (Q,) their eigenvalues.  Returns (EL, found): found[q] is False when no
    computed eigenvalue lies within rel_tol |lambda_q| of conj(lambda_q) (such a mode has no left
    vector among the Q and cannot be subtracted)."""
    Q = ER.shape[1]
    EL = np.zeros_like(ER)
    found = np.zeros(Q, dtype=bool)
    g5R = L.flat(L.g5(L.unflat(ER.T, dims))).T        # gamma_5 applied to every column
    for q in range(Q):
        dist = np.abs(lam - np.conj(lam[q]))
        p = int(np.argmin(dist))
        if dist[p] > rel_tol * max(abs(lam[q]), 1e-300):
            continue
        norm = np.vdot(g5R[:, p], ER[:, q])               # e_R(lambda_p)^dag gamma_5 e_R(lambda_q)
        EL[:, q] = g5R[:, p] / np.conj(norm)
        found[q] = True
    return EL, found


def es_vector(ER, EL, lam, eta):
    """ES subtraction vector tilde x_eig = sum_q e_R^(q) (1/lambda_q) (e_L^(q)dag eta) (Sec. 5.3)."""
    dims_shape = eta.shape[-6:]
    ef = eta.reshape(eta.shape[:-6] + (-1,))
    c = ef @ EL.conj()                      # (..., Q) = e_L^dag eta
    y = (c / lam) @ ER.T
    return y.reshape(eta.shape[:-6] + dims_shape)


def es_addback(U, kappa, ER, EL, lam, dims):
    """Densities of Tr(Theta tilde M^{-1}_eig) = sum_q (1/lambda_q) e_L^(q)dag Theta e_R^(q) (Sec. 5.3;
    for Theta = 1 this is sum_q 1/lambda_q)."""
    out = np.zeros((O.NOPS,) + L.site_shape(dims), dtype=np.complex128)
    for q in range(ER.shape[1]):
        out += O.densities(U, kappa, L.unflat(EL[:, q], dims), L.unflat(ER[:, q], dims)) / lam[q]
    return out


def xi_inverse(E, apply_tilde, dims):
    """1/xi'_q = e'_q^dag gamma_5 tilde M^{-1} e'_q for each eigenvector (Sec. 5.5)."""
    out = np.zeros(E.shape[1], dtype=np.complex128)
    for q in range(E.shape[1]):
        e = L.unflat(E[:, q], dims)
        out[q] = np.vdot(e, L.g5(apply_tilde(e)))
    return out
