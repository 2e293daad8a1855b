"""Lattice data and the Wilson matrix M = 1 - kappa P  (Eq. xyz556, Sec. 5.1).

Test infrastructure (see ``oracle/__init__.py``): slow, plain FP64 numpy.

Conventions (readings of the paper, which fixes neither):
  * A field psi has shape (..., T, Z, Y, X, 4, 3): site axes t-slowest, then Dirac spin, then
    colour.  The flat (lexicographic) site index is s = x + Lx*(y + Ly*(z + Lz*t)) and the
    flat unknown index is 12*s + 3*spin + colour (Sec. 2: "space-time-color-Dirac space").
  * Gauge links U have shape (4, T, Z, Y, X, 3, 3); direction mu = 0, 1, 2, 3 is x, y, z, t.
  * Euclidean Hermitian gamma matrices in the Dirac representation:
        gamma_k = [[0, -i sigma_k], [i sigma_k, 0]]  (k = 1, 2, 3 -> mu = 0, 1, 2)
        gamma_4 = diag(1, 1, -1, -1)                 (mu = 3)
        gamma_5 = gamma_1 gamma_2 gamma_3 gamma_4.
  * Periodic boundary conditions in all four directions (Sec. 7).
  * The garbled deltas of the P_ij definition (Eq. after xyz556) are read as: the forward term
    (1 - gamma_mu) U_mu(x) couples psi(x + mu), the backward term (1 + gamma_mu) U_mu(x - mu)^dag
    couples psi(x - mu).
"""
import numpy as np

# site-array axis (within T, Z, Y, X) of direction mu
SITE_AXIS = {0: 3, 1: 2, 2: 1, 3: 0}


def pauli():
    s1 = np.array([[0, 1], [1, 0]], dtype=np.complex128)
    s2 = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
    s3 = np.array([[1, 0], [0, -1]], dtype=np.complex128)
    return s1, s2, s3


def gammas():
    """Return (g, g5): g[mu] for mu = 0..3 (x, y, z, t) and gamma_5, all 4x4 complex."""
    z2 = np.zeros((2, 2), dtype=np.complex128)
    i2 = np.eye(2, dtype=np.complex128)
    g = []
    for s in pauli():
        g.append(np.block([[z2, -1j * s], [1j * s, z2]]))
    g.append(np.block([[i2, z2], [z2, -i2]]))
    g = np.array(g)
    g5 = g[0] @ g[1] @ g[2] @ g[3]
    return g, g5


G, G5 = gammas()
ONE4 = np.eye(4, dtype=np.complex128)


def volume(dims):
    """dims = (Lx, Ly, Lz, Lt); number of sites V."""
    return int(np.prod(dims))


def site_shape(dims):
    lx, ly, lz, lt = dims
    return (lt, lz, ly, lx)


def site_index(x, y, z, t, dims):
    """Lexicographic site index s = x + Lx (y + Ly (z + Lz t))."""
    lx, ly, lz, _ = dims
    return x + lx * (y + ly * (z + lz * t))


def field_shape(dims, batch=()):
    return tuple(batch) + site_shape(dims) + (4, 3)


def _site_ax(psi, mu):
    return psi.ndim - 6 + SITE_AXIS[mu]


def spin_apply(S, psi):
    """(S psi) on the spin index for a 4x4 matrix S."""
    return np.matmul(S, psi)


def color_apply(Umu, psi):
    """U_mu(x) psi(x) for every site (colour matrix times colour vector, spin untouched):
    out[s, a] = sum_b U[a, b] psi[s, b], i.e. psi times U transposed."""
    return np.matmul(psi, np.swapaxes(Umu, -1, -2))


def color_apply_dag(Umu, psi):
    """U_mu(x)^dagger psi(x) for every site: out[s, a] = sum_b conj(U[b, a]) psi[s, b]."""
    return np.matmul(psi, Umu.conj())


def shift(psi, mu, sign):
    """shift(psi, mu, +1)(x) = psi(x + mu);  shift(psi, mu, -1)(x) = psi(x - mu)  (periodic)."""
    return np.roll(psi, -sign, axis=_site_ax(psi, mu))


def hop(U, psi):
    """P psi with  P = sum_mu [(1 - g_mu) U_mu(x) delta_{y, x+mu} + (1 + g_mu) U_mu(x-mu)^dag delta_{y, x-mu}]
    (the matrix below Eq. xyz556)."""
    out = np.zeros_like(psi)
    for mu in range(4):
        fwd = color_apply(U[mu], shift(psi, mu, +1))
        out += spin_apply(ONE4 - G[mu], fwd)
        bwd = shift(color_apply_dag(U[mu], psi), mu, -1)
        out += spin_apply(ONE4 + G[mu], bwd)
    return out


def wilson(U, kappa, psi):
    """M psi = psi - kappa P psi  (Eq. xyz556)."""
    return psi - kappa * hop(U, psi)


def wilson_at_sites(U, kappa, psi, sites):
    """(M psi)(x) at the listed sites only, x = (t, z, y, x) tuples, from the definition of
    Eq. xyz556 term by term (for checking operators on lattices too large for `wilson`):
    psi(x) - kappa sum_mu [(1 - g_mu) U_mu(x) psi(x + mu) + (1 + g_mu) U_mu(x - mu)^dag psi(x - mu)].
    psi: one field (T, Z, Y, X, 4, 3).  Returns (len(sites), 4, 3)."""
    ext = psi.shape[:4]
    out = []
    for site in sites:
        acc = np.zeros((4, 3), dtype=np.complex128)
        for mu in range(4):
            ax = SITE_AXIS[mu]
            up = list(site)
            up[ax] = (up[ax] + 1) % ext[ax]
            dn = list(site)
            dn[ax] = (dn[ax] - 1) % ext[ax]
            fwd = psi[tuple(up)] @ U[(mu,) + tuple(site)].T          # U_mu(x) psi(x + mu), per spin
            bwd = psi[tuple(dn)] @ U[(mu,) + tuple(dn)].conj()        # U_mu(x - mu)^dag psi(x - mu)
            acc += (ONE4 - G[mu]) @ fwd + (ONE4 + G[mu]) @ bwd
        out.append(psi[tuple(site)] - kappa * acc)
    return np.array(out)


def g5(psi):
    return spin_apply(G5, psi)


def wilson_g5(U, kappa, psi):
    """M' psi = M gamma_5 psi  (Sec. 5.4: gamma_5 multiplied on the right)."""
    return wilson(U, kappa, g5(psi))


def wilson_dag(U, kappa, psi):
    """M^dag psi, computed as the plain adjoint of the stencil (not through gamma_5-hermiticity):
    P^dag = sum_mu [(1 - g_mu) U_mu(x-mu)^dag delta_{y,x-mu} + (1 + g_mu) U_mu(x) delta_{y,x+mu}]
    because the gamma matrices are Hermitian."""
    out = np.zeros_like(psi)
    for mu in range(4):
        bwd = shift(color_apply_dag(U[mu], spin_apply(ONE4 - G[mu], psi)), mu, -1)
        fwd = color_apply(U[mu], shift(spin_apply(ONE4 + G[mu], psi), mu, +1))
        out += bwd + fwd
    return psi - np.conj(kappa) * out


def dense(apply, dims, dtype=np.complex128):
    """Dense N x N matrix of a linear map on fields (N = 12 V): column j = apply(e_j)."""
    n = 12 * volume(dims)
    eye = np.eye(n, dtype=dtype).reshape((n,) + field_shape(dims))
    cols = apply(eye).reshape(n, n)
    return cols.T.copy()


def flat(psi):
    """Field (..., T, Z, Y, X, 4, 3) -> (..., N) with the flat unknown index of the module docstring."""
    lead = psi.shape[:-6]
    return psi.reshape(lead + (-1,))


def unflat(v, dims):
    lead = v.shape[:-1]
    return v.reshape(lead + site_shape(dims) + (4, 3))

