"""The nine loop operators of Table Table903 (Sec. 6) and their per-site contractions.

Test infrastructure (see ``oracle/__init__.py``).

Operator numbering (reading): 0 scalar; 1..4 local vector gamma_mu for mu = x, y, z, t;
5..8 point-split vector for mu = x, y, z, t.  The paper's "J_4" is mu = t (operators 4 and 8).

For a matrix Theta the noise term of every estimator is eta^dag Theta w (Sec. 5).  We split it
into a density over base sites x:
  scalar       d(x) = eta(x)^dag w(x)
  local        d(x) = eta(x)^dag gamma_mu w(x)
  point-split  d(x) = kappa [ eta(x+mu)^dag (1 + g_mu) U_mu(x)^dag w(x)
                              - eta(x)^dag (1 - g_mu) U_mu(x) w(x + mu) ]
The point-split form is Table Table903's field representation with psi-bar -> eta^dag and
psi -> w; as a matrix, Theta_{(x+mu),(x)} = kappa (1+g_mu) U_mu(x)^dag and
Theta_{(x),(x+mu)} = -kappa (1-g_mu) U_mu(x).  sum_x d(x) = eta^dag Theta w.
Scalar estimates carry their signal in the real part, vector ones in the imaginary part (Sec. 6).
"""
import numpy as np

from . import lattice as L

NOPS = 9
OP_NAMES = ["scalar", "local_x", "local_y", "local_z", "local_t",
            "psplit_x", "psplit_y", "psplit_z", "psplit_t"]
# which part carries the signal: 0 = real, 1 = imaginary
OP_PART = [0, 1, 1, 1, 1, 1, 1, 1, 1]


def _inner(a, b):
    """Per-site a(x)^dag b(x) summed over spin and colour."""
    return np.einsum('...sc,...sc->...', a.conj(), b)


def densities(U, kappa, eta, w):
    """d[op, ..., T, Z, Y, X] for all nine operators (see module docstring)."""
    out = []
    out.append(_inner(eta, w))
    for mu in range(4):
        out.append(_inner(eta, L.spin_apply(L.G[mu], w)))
    for mu in range(4):
        a = L.spin_apply(L.ONE4 + L.G[mu], L.color_apply_dag(U[mu], w))
        t1 = _inner(L.shift(eta, mu, +1), a)
        b = L.spin_apply(L.ONE4 - L.G[mu], L.color_apply(U[mu], L.shift(w, mu, +1)))
        t2 = _inner(eta, b)
        out.append(kappa * (t1 - t2))
    return np.stack(out)


def per_t(d):
    """Sum densities d[..., T, Z, Y, X] over space: returns d[..., T]."""
    return d.sum(axis=(-1, -2, -3))


def theta_apply(U, kappa, op, w):
    """(Theta w)(y) for one operator, as a field: with it, eta^dag (Theta w) = sum_x d(x)."""
    if op == 0:
        return w.copy()
    if op <= 4:
        return L.spin_apply(L.G[op - 1], w)
    mu = op - 5
    a = L.shift(L.spin_apply(L.ONE4 + L.G[mu], L.color_apply_dag(U[mu], w)), mu, -1)
    b = L.spin_apply(L.ONE4 - L.G[mu], L.color_apply(U[mu], L.shift(w, mu, +1)))
    return kappa * (a - b)
