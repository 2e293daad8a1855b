"""Even/odd preconditioning of the Wilson matrix (Sec. 7) and the full eigenpairs it yields for ES.

Test infrastructure (see ``oracle/__init__.py``): slow, plain FP64 numpy.

The paper solves the reduced (even/odd preconditioned) Wilson system with GMRES-DR / GMRES-Proj
and forms the eigenpairs of the full matrix from those of the reduced one for eigenvalue
subtraction (Sec. 7).  With a site's parity (x + y + z + t) mod 2 and every lattice extent even,
the hopping matrix P of Eq. xyz556 couples only sites of opposite parity, so with the unknowns
ordered (even, odd)

    M = 1 - kappa P = [[1, -kappa P_eo], [-kappa P_oe, 1]].

Eliminating the odd sites gives the reduced (Schur complement) matrix on the even sites

    hat M = 1 - kappa^2 P_eo P_oe,    hat M x_e = b_e + kappa P_eo b_o,    x_o = b_o + kappa P_oe x_e.

Eigenpairs (reading of "easily related", Sec. 7): if M v = lambda v then
kappa^2 P_eo P_oe v_e = (1 - lambda)^2 v_e, so v_e is an eigenvector of hat M with eigenvalue
mu = 1 - (1 - lambda)^2.  Conversely each reduced pair (mu, v_e) gives the two full pairs
1 - lambda = +-sqrt(1 - mu), v = (v_e, kappa P_oe v_e / (1 - lambda)) (normalised to unit length).
P_oe and P_eo are applied here through the full hopping matrix on fields zero on the other
parity, so that they are exactly the blocks of P.
"""
import numpy as np

from . import lattice as L


def parity(dims):
    """Site parity (x + y + z + t) mod 2 as an array over (T, Z, Y, X)."""
    lx, ly, lz, lt = dims
    t, z, y, x = np.meshgrid(np.arange(lt), np.arange(lz), np.arange(ly), np.arange(lx), indexing="ij")
    return (x + y + z + t) % 2


def _check(dims):
    if any(d % 2 for d in dims):
        raise ValueError("even/odd decomposition needs even extents: %s" % (dims,))


def split(psi, dims):
    """Field (..., T, Z, Y, X, 4, 3) -> (even, odd) arrays (..., V/2, 4, 3), sites in lexicographic order."""
    _check(dims)
    par = parity(dims).reshape(-1)
    f = psi.reshape(psi.shape[:-6] + (-1, 4, 3))
    return f[..., par == 0, :, :], f[..., par == 1, :, :]


def join(pe, po, dims):
    """Inverse of split."""
    _check(dims)
    par = parity(dims).reshape(-1)
    lead = pe.shape[:-3]
    f = np.zeros(lead + (par.size, 4, 3), dtype=np.result_type(pe, po))
    f[..., par == 0, :, :] = pe
    f[..., par == 1, :, :] = po
    return f.reshape(lead + L.site_shape(dims) + (4, 3))


def hop_oe(U, ve, dims):
    """P_oe v_e: the odd-site part of P applied to a field that is v_e on even sites, 0 on odd."""
    return split(L.hop(U, join(ve, np.zeros_like(ve), dims)), dims)[1]


def hop_eo(U, vo, dims):
    """P_eo v_o: the even-site part of P applied to a field that is v_o on odd sites, 0 on even."""
    return split(L.hop(U, join(np.zeros_like(vo), vo, dims)), dims)[0]


def reduced_apply(U, kappa, ve, dims):
    """hat M v_e = v_e - kappa^2 P_eo P_oe v_e."""
    return ve - kappa ** 2 * hop_eo(U, hop_oe(U, ve, dims), dims)


def reduced_rhs(U, kappa, b, dims):
    """b_e + kappa P_eo b_o for a full field b."""
    be, bo = split(b, dims)
    return be + kappa * hop_eo(U, bo, dims)


def reconstruct(U, kappa, xe, b, dims):
    """Full solution from the even part: x_o = b_o + kappa P_oe x_e."""
    _, bo = split(b, dims)
    return join(xe, bo + kappa * hop_oe(U, xe, dims), dims)


def full_eigenpairs(U, kappa, mu, Ve, dims, tol=1e-8):
    """Both full eigenpairs of M from each reduced pair (mu_q, v_e^(q)) of hat M (module docstring).
    mu: (Q,); Ve: (Q, V/2, 4, 3).  Returns lam (2Q,) and unit right eigenvectors (2Q, T, Z, Y, X, 4, 3).
    Raises ValueError for a mu with |sqrt(1 - mu)| <= tol (lambda = 1, where 1 - lambda vanishes)."""
    lams, vecs = [], []
    for q in range(len(mu)):
        r = np.sqrt(complex(1.0 - mu[q]))
        if abs(r) <= tol:
            # 1 - lambda = 0: the odd part kappa P_oe v_e / (1 - lambda) is undefined, so the full
            # pair cannot be rebuilt from v_e alone
            raise ValueError("reduced eigenvalue mu = %r is 1 to within %g: no full eigenpair" % (mu[q], tol))
        po = kappa * hop_oe(U, Ve[q], dims)
        for one_minus_lam in (r, -r):
            v = join(Ve[q], po / one_minus_lam, dims)
            lams.append(1.0 - one_minus_lam)
            vecs.append(v / np.linalg.norm(v))
    return np.array(lams), np.stack(vecs)
