"""Derivatives of the loop estimates with respect to kappa and to the gauge links.

Test infrastructure (see ``oracle/__init__.py``).  The paper has no derivatives; this is the
differentiation stage of the hot path, written from the definitions of Sec. 5-6:

* With M = 1 - kappa P (Eq. xyz556), dM/dkappa = -P, so d M^{-1}/dkappa = M^{-1} P M^{-1} and
      d Tr(Theta M^{-1}) / dkappa = Tr(dTheta/dkappa M^{-1}) + Tr(Theta M^{-1} P M^{-1}).
  The point-split operators carry kappa as a prefactor (Table Table903), dTheta/dkappa = Theta/kappa;
  the local ones do not depend on kappa.  Per noise: with x = M^{-1} eta and y = M^{-1} P x,
      d(eta^dag Theta x)/dkappa = eta^dag (dTheta/dkappa) x + eta^dag Theta y.
* PS subtraction (Sec. 5.1) differentiated term by term: d tilde x/dkappa = sum_{k>=1} k kappa^{k-1} P^k eta,
  d/dkappa sum_k kappa^k Tr(Theta P^k) = sum_k k kappa^{k-1} Tr(Theta P^k) + sum_k kappa^k Tr(dTheta/dkappa P^k).
* Link gradient of the scalar estimate eta^dag M^{-1} eta: with z = M^{-dag} eta and x = M^{-1} eta,
      d(eta^dag M^{-1} eta) = -z^dag dM x = kappa z^dag dP x.
  For the Lie-algebra perturbation U_mu(x) -> exp(i w lambda_a / 2) U_mu(x) (Gell-Mann lambda_a):
      dT/dw_a = (i kappa / 2) tr(lambda_a B_mu(x)),
      B = sum_{s,s'} (1 - g_mu)_{s s'} u_{s'} z(x)_s^dag - sum_{s,s'} (1 + g_mu)_{s s'} x(x)_{s'} (U_mu(x) z(x+mu)_s)^dag,
      u_{s'} = U_mu(x) x(x+mu)_{s'}.
  The complex-matrix derivatives are dT/dU_ab = kappa sum_{s s'} z(x)*_{s a} (1-g)_{s s'} x(x+mu)_{s' b} and
  dT/d(U*)_ab = kappa sum_{s s'} z(x+mu)*_{s b} (1+g)_{s s'} x(x)_{s' a}.
"""
import numpy as np

from . import lattice as L
from . import operators as O


def gell_mann():
    g = np.zeros((8, 3, 3), dtype=np.complex128)
    g[0][0, 1] = g[0][1, 0] = 1
    g[1][0, 1], g[1][1, 0] = -1j, 1j
    g[2][0, 0], g[2][1, 1] = 1, -1
    g[3][0, 2] = g[3][2, 0] = 1
    g[4][0, 2], g[4][2, 0] = -1j, 1j
    g[5][1, 2] = g[5][2, 1] = 1
    g[6][1, 2], g[6][2, 1] = -1j, 1j
    g[7][0, 0] = g[7][1, 1] = 1 / np.sqrt(3)
    g[7][2, 2] = -2 / np.sqrt(3)
    return g


LAMBDA = gell_mann()


def dkappa_densities(U, kappa, eta, x, y):
    """Per-site densities of d(eta^dag Theta x)/dkappa for the nine operators, [op, ...sites]."""
    d = O.densities(U, kappa, eta, y)
    dx = O.densities(U, kappa, eta, x)
    d[5:9] = d[5:9] + dx[5:9] / kappa
    return d


def dpert_vector(U, kappa, eta, K):
    """d tilde x_pert / dkappa = sum_{k=1}^{K-1} k kappa^{k-1} P^k eta."""
    term = eta.copy()
    acc = np.zeros_like(eta)
    for k in range(1, K):
        term = L.hop(U, term)
        acc = acc + k * kappa ** (k - 1) * term
    return acc


def dpert_addback(t, kappa, K):
    """d/dkappa of the PS add-back densities sum_k kappa^k t_k(Theta) (t from subtract.hop_traces,
    computed with the same kappa: the point-split t_k carry one power of kappa)."""
    out = sum(k * kappa ** (k - 1) * t[k] for k in range(1, K))
    out = out + 0 * t[0]
    ps = sum((kappa ** k) * t[k][5:9] for k in range(K)) / kappa
    out[5:9] = out[5:9] + ps
    return out


def exact_dkappa(U, kappa, dims):
    """d Tr(Theta M^{-1}) / dkappa for the nine operators from dense matrices."""
    from . import exact
    Minv = exact.inverse(U, kappa, dims)
    P = L.dense(lambda v: L.hop(U, v), dims)
    W = Minv @ P @ Minv
    out = []
    for op in range(O.NOPS):
        Th = exact.dense_theta(U, kappa, op, dims)
        v = np.sum(Th * W.T)
        if op >= 5:
            v = v + np.sum(Th * Minv.T) / kappa
        out.append(v)
    return np.array(out)


def link_gradient(U, kappa, x, z):
    """dT/dw_a for every link (shape (4, T, Z, Y, X, 8), complex) of T = eta^dag M^{-1} eta, given
    x = M^{-1} eta and z = M^{-dag} eta (single fields)."""
    out = np.zeros(U.shape[:-2] + (8,), dtype=np.complex128)
    for mu in range(4):
        xf = L.shift(x, mu, +1)                       # x(x + mu)
        u = L.color_apply(U[mu], xf)                  # U x(x+mu), per spin
        a1 = np.einsum('st,...tc,...sd->...cd', L.ONE4 - L.G[mu], u, z.conj())
        q = L.color_apply(U[mu], L.shift(z, mu, +1))  # U z(x+mu)
        a2 = np.einsum('st,...tc,...sd->...cd', L.ONE4 + L.G[mu], x, q.conj())
        B = a1 - a2
        out[mu] = 0.5j * kappa * np.einsum('acd,...dc->...a', LAMBDA, B)
    return out


def link_matrix_derivatives(U, kappa, x, z):
    """(dT/dU, dT/dU*) per link, shape (4, T, Z, Y, X, 3, 3) each, entries [a, b] as in the module text."""
    dU = np.zeros(U.shape, dtype=np.complex128)
    dUc = np.zeros(U.shape, dtype=np.complex128)
    for mu in range(4):
        xf = L.shift(x, mu, +1)
        zf = L.shift(z, mu, +1)
        dU[mu] = kappa * np.einsum('...sa,st,...tb->...ab', z.conj(), L.ONE4 - L.G[mu], xf)
        dUc[mu] = kappa * np.einsum('...sb,st,...ta->...ab', zf.conj(), L.ONE4 + L.G[mu], x)
    return dU, dUc


def perturb_link(U, mu, site, a, h):
    """Copy of U with U_mu(site) -> exp(i h lambda_a / 2) U_mu(site); site = (t, z, y, x)."""
    w, Vh = np.linalg.eigh(LAMBDA[a])
    E = (Vh * np.exp(0.5j * h * w)) @ Vh.conj().T
    U2 = U.copy()
    U2[(mu,) + tuple(site)] = E @ U[(mu,) + tuple(site)]
    return U2
