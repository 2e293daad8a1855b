"""Exact (dense) quantities the estimators are unbiased for, and the exact Z(4) noise variance.

Test infrastructure (see ``oracle/__init__.py``).  Small lattices only (dense N x N, N = 12 V).

  * Tr(Theta M^{-1}) by a dense LU solve (Sec. 5: the quantity every estimator targets);
  * the exact variance of one Z(N >= 3) noise estimate of Tr(Q) (Eq. xyz255):
        Var = sum_{i != j} |q_ij|^2,
    split into its real and imaginary parts (derived from the Z(4) moments of Sec. 3,
    <|X_ji|^2> = 1/N, <X_ji^2> = 0):
        Var(Re) = 1/2 sum_{i != j} (|q_ij|^2 + Re q_ij q_ji),  Var(Im) = 1/2 sum_{i != j} (|q_ij|^2 - Re q_ij q_ji).
"""
import numpy as np
import scipy.linalg as sla

from . import lattice as L
from . import operators as O


def dense_M(U, kappa, dims):
    return L.dense(lambda v: L.wilson(U, kappa, v), dims)


def dense_theta(U, kappa, op, dims):
    return L.dense(lambda v: O.theta_apply(U, kappa, op, v), dims)


def inverse(U, kappa, dims):
    M = dense_M(U, kappa, dims)
    lu = sla.lu_factor(M)
    return sla.lu_solve(lu, np.eye(M.shape[0], dtype=np.complex128))


def exact_traces(U, kappa, dims, Minv=None):
    """Tr(Theta M^{-1}) for the nine operators."""
    if Minv is None:
        Minv = inverse(U, kappa, dims)
    return np.array([np.sum(dense_theta(U, kappa, op, dims) * Minv.T) for op in range(O.NOPS)])


def z4_variance(Q):
    """(Var, Var_Re, Var_Im) of eta^dag Q eta for a single Z(4) noise vector (Eq. xyz255)."""
    off = Q - np.diag(np.diag(Q))
    a = np.sum(np.abs(off) ** 2)
    b = np.sum((off * off.T).real)
    return a, 0.5 * (a + b), 0.5 * (a - b)
