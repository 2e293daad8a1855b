"""Seeded synthetic inputs: near-identity SU(3) gauge fields.

This module only shapes inputs; it holds none of the loop-estimation arithmetic, so both the
CUDA path and the CPU oracle may be fed from it.  The paper's workloads are quenched beta = 6.0
and MILC HISQ ensembles, which are not available; these fields stand in for them with the
paper's lattice shapes (Sec. 7-9).

Recipe: for every link draw A with independent standard complex Gaussian entries, form the
traceless Hermitian H = (A + A^dag)/2 - Tr(.)/3, set U = exp(i eps H) through the eigen-
decomposition of H, then re-unitarise (Gram-Schmidt on rows 1 and 2, row 3 = (row1 x row2)^*),
which makes det U = 1 to rounding.  Links are stored as complex128 with shape
(4, T, Z, Y, X, 3, 3), direction mu = x, y, z, t, row-major colour matrices.
"""
import numpy as np


def su3_links(dims, eps, seed):
    lx, ly, lz, lt = dims
    rng = np.random.default_rng(seed)
    n = 4 * lt * lz * ly * lx
    A = (rng.standard_normal((n, 3, 3)) + 1j * rng.standard_normal((n, 3, 3))) / np.sqrt(2.0)
    H = 0.5 * (A + np.conj(np.swapaxes(A, -1, -2)))
    tr = np.trace(H, axis1=-2, axis2=-1).real / 3.0
    H = H - tr[:, None, None] * np.eye(3)[None]
    w, W = np.linalg.eigh(H)
    U = (W * np.exp(1j * eps * w)[:, None, :]) @ np.conj(np.swapaxes(W, -1, -2))
    return reunitarize(U).reshape(4, lt, lz, ly, lx, 3, 3)


def reunitarize(U):
    r1 = U[..., 0, :]
    r1 = r1 / np.linalg.norm(r1, axis=-1, keepdims=True)
    r2 = U[..., 1, :]
    r2 = r2 - np.sum(np.conj(r1) * r2, axis=-1, keepdims=True) * r1
    r2 = r2 / np.linalg.norm(r2, axis=-1, keepdims=True)
    r3 = np.conj(np.cross(r1, r2))
    return np.stack([r1, r2, r3], axis=-2)


def unit_links(dims):
    lx, ly, lz, lt = dims
    U = np.zeros((4, lt, lz, ly, lx, 3, 3), dtype=np.complex128)
    U[..., 0, 0] = U[..., 1, 1] = U[..., 2, 2] = 1.0
    return U


def mean_plaquette(U):
    """(1/3) Re Tr of the elementary plaquettes, averaged over sites and the six planes."""
    axis = {0: 3, 1: 2, 2: 1, 3: 0}
    acc = 0.0
    for mu in range(4):
        for nu in range(mu + 1, 4):
            b = np.roll(U[nu], -1, axis=axis[mu])
            c = np.conj(np.swapaxes(np.roll(U[mu], -1, axis=axis[nu]), -1, -2))
            d = np.conj(np.swapaxes(U[nu], -1, -2))
            p = U[mu] @ b @ c @ d
            acc += np.trace(p, axis1=-2, axis2=-1).real.mean() / 3.0
    return acc / 6.0


def eps_for_plaquette(dims, target, seed, lo=0.0, hi=1.5, iters=40):
    """Bisection on eps (fixed seed) so that the mean plaquette matches the target."""
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        if mean_plaquette(su3_links(dims, mid, seed)) > target:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)
