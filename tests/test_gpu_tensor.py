"""GPU parity of the split-precision tensor-core deflation contractions (Sec. 5.4) with the oracle.

G = E^dag X and Y = E C run on the tcgen05 tensor cores with bf16 slices of the FP64 operands.  The
splitting truncates every operand entry below 2^-54 of the largest entry of its row (left operand)
or column (right operand), so an entry sum_i a_i b_i of the result is off by less than about
2^-52 (max|a| sum|b| + sum|a| max|b|) plus FP64 rounding; each entry is compared with the oracle's
definition within 2^-50 of that sum (complex moduli, a factor 2 above the real-component form).  Cases cover one and several 128-row tiles
with ragged tails, 1 to 40 right-hand sides (NP = 16 .. 64 columns and two sub-blocks), Gaussian
operands (seven slices each) and Z(4) noise (one exact slice), then the HFES projection and a whole
loop estimate with the tensor-core engine against the FP64 engine, and sampled entries at the
24^3 x 32 size with 200 vectors."""
import math

import numpy as np
import pytest

from oracle import lattice as L, rng, subtract as S
from paper_1903_06986_gb300 import lqcd, synth
from tests.gpu_util import context, dev, host, rel_err, torch_cuda

pytestmark = pytest.mark.gpu

TC_TOL = 2.0 ** -50


def _two_prod(a, b):
    """Dekker's exact product a * b = p + e of float64 arrays (Veltkamp splitting, no FMA)."""
    def split(x):
        c = 134217729.0 * x        # 2^27 + 1
        hi = c - (c - x)
        return hi, x - hi
    p = a * b
    ah, al = split(a)
    bh, bl = split(b)
    e = ((ah * bh - p) + ah * bl + al * bh) + al * bl
    return p, e


def exact_matmul(A, B):
    """A @ B for complex128 A (m, K), B (K, n), every entry correctly rounded: the exact products
    of the real components summed by math.fsum (reference far below the tolerances tested)."""
    out = np.empty((A.shape[0], B.shape[1]), dtype=np.complex128)
    for j in range(B.shape[1]):
        b = B[:, j]
        terms_re = [_two_prod(A.real, b.real[None, :]), _two_prod(-A.imag, b.imag[None, :])]
        terms_im = [_two_prod(A.real, b.imag[None, :]), _two_prod(A.imag, b.real[None, :])]
        re = np.concatenate([x for t in terms_re for x in t], axis=1)
        im = np.concatenate([x for t in terms_im for x in t], axis=1)
        out[:, j] = [complex(math.fsum(r), math.fsum(i)) for r, i in zip(re, im)]
    return out


def split_bound(A, B):
    """max|a| sum|b| + sum|a| max|b| for every entry of A @ B (rows of A, columns of B)."""
    a, b = np.abs(A), np.abs(B)
    return a.max(axis=1)[:, None] * b.sum(axis=0)[None, :] + a.sum(axis=1)[:, None] * b.max(axis=0)[None, :]


def gauss(r, shape):
    return r.standard_normal(shape) + 1j * r.standard_normal(shape)


@pytest.mark.parametrize("dims,k,nrhs,z4", [((4, 4, 4, 4), 5, 1, True), ((4, 4, 4, 4), 37, 3, False),
                                            ((3, 5, 2, 7), 130, 16, True), ((3, 5, 2, 7), 130, 16, False),
                                            ((4, 4, 4, 4), 64, 40, False), ((2, 2, 2, 2), 200, 24, True)])
def test_vdag_x_matches_definition(dims, k, nrhs, z4):
    ctx = context(dims)
    r = np.random.default_rng(100 + k + nrhs)
    n = 12 * L.volume(dims)
    E = gauss(r, (k, n)) * np.exp(r.uniform(-3, 3, size=(k, 1)))     # rows of different scales
    X = rng.z4_block(5, 0, nrhs, dims).reshape(nrhs, n) if z4 else gauss(r, (nrhs, n))
    got = host(ctx.tc_vdag_x(dev(E), dev(X)))
    ref = S.defl_coeffs(E.T, X)
    ratio = np.abs(got - ref) / split_bound(E, X.T)
    assert ratio.max() <= TC_TOL, "max error / bound = 2^%.2f" % np.log2(ratio.max())
    # same call twice gives the same bits (deterministic reductions)
    again = host(ctx.tc_vdag_x(dev(E), dev(X)))
    assert np.array_equal(got, again)


@pytest.mark.parametrize("dims,k,nrhs", [((4, 4, 4, 4), 5, 1), ((3, 5, 2, 7), 37, 16), ((2, 2, 2, 2), 200, 40),
                                         ((4, 4, 4, 4), 33, 8)])
def test_v_c_matches_definition(dims, k, nrhs):
    ctx = context(dims)
    r = np.random.default_rng(200 + k + nrhs)
    n = 12 * L.volume(dims)
    E = gauss(r, (k, n)) * np.exp(r.uniform(-3, 3, size=(k, 1)))
    Cm = gauss(r, (k, nrhs)) * np.exp(r.uniform(-4, 4, size=(k, 1)))
    got = host(ctx.tc_v_c(dev(E), dev(Cm))).reshape(nrhs, n)
    ref = exact_matmul(E.T, Cm).T
    # the oracle's FP64 definition agrees with the correctly rounded reference to FP64 rounding
    assert rel_err(S.defl_expand(E.T, Cm), ref) < 1e-13
    ratio = np.abs(got - ref) / split_bound(E.T, Cm).T
    assert ratio.max() <= TC_TOL, "max error / bound = 2^%.2f" % np.log2(ratio.max())


def _orthonormal(n, k, seed):
    r = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(gauss(r, (n, k)))
    return Q


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (3, 5, 2, 7)])
def test_deflate_project_tensor_engine(dims):
    ctx = context(dims)
    n = 12 * L.volume(dims)
    E = _orthonormal(n, 6, 10)
    lam = np.array([0.11, -0.12, 0.2, -0.25, 0.3, 0.31], dtype=np.complex128)
    defl = ctx.defl_import(dev(E.T), lam)
    eta = rng.z4_block(4, 0, 3, dims)
    d = 1.0 / lam - 0.3j
    ref = S.defl_vector(E, d, eta)
    ctx.set_defl_engine(lqcd.DEFL_TENSOR)
    got = host(ctx.deflate_project(defl, dev(eta), d))
    got2 = host(ctx.deflate_project(defl, dev(eta), d))      # cached slices
    ctx.set_defl_engine(lqcd.DEFL_FP64)
    fp64 = host(ctx.deflate_project(defl, dev(eta), d))
    assert rel_err(got, ref) < 1e-13
    assert np.array_equal(got, got2)
    assert rel_err(got, fp64) < 1e-13


def test_loop_estimate_tensor_engine_matches_fp64():
    """Whole HFES / HFPS / HFPOLY estimate on 4^4 with the tensor-core projections against the FP64
    engine on the same deflation space: the per-noise estimates agree to 1e-11 relative."""
    dims = (4, 4, 4, 4)
    U = dev(synth.su3_links(dims, 0.3, 1))
    kw = dict(seed=1, nnoise=10, block=10, m=20, k=5, K=4, npoly=6, tol=1e-12, tol_special=1e-14)
    ctx = context(dims)
    a = ctx.loop_estimate(U, 0.150, **kw)
    ctx.set_defl_engine(lqcd.DEFL_TENSOR)
    b = ctx.loop_estimate(U, 0.150, **kw)
    ctx.set_defl_engine(lqcd.DEFL_FP64)
    assert b["converged"]
    for key in ("per_noise", "mean"):
        assert rel_err(b[key], a[key]) < 1e-11


def test_vdag_x_and_v_c_sampled_at_full_size():
    """24^3 x 32 (5.3M complex unknowns), 200 vectors, 16 Z(4) noises: G entries and Y sites sampled
    and recomputed by the oracle's definition from copies of the vectors involved."""
    torch = torch_cuda()
    dims = (24, 24, 24, 32)
    ctx = context(dims)
    n = 12 * L.volume(dims)
    k, nrhs = 200, 16
    gen = torch.Generator(device="cuda").manual_seed(7)
    E = torch.randn((k, n), dtype=torch.complex128, device="cuda", generator=gen)
    X = ctx.noise_z4(11, 0, nrhs).reshape(nrhs, n)
    G = host(ctx.tc_vdag_x(E, X))
    r = np.random.default_rng(3)
    for q, j in zip(r.integers(0, k, 6), r.integers(0, nrhs, 6)):
        e = host(E[q])
        x = host(X[j])
        ref = np.vdot(e, x)
        assert abs(G[q, j] - ref) <= TC_TOL * split_bound(e[None, :], x[:, None])[0, 0]
    Cm = torch.from_numpy(gauss(r, (k, nrhs))).cuda()
    Y = ctx.tc_v_c(E, Cm)
    Ch = host(Cm)
    for i, j in zip(r.integers(0, n, 8), r.integers(0, nrhs, 8)):
        col = host(E[:, i])
        ref = np.sum(col * Ch[:, j])
        assert abs(host(Y[j, i]) - ref) <= TC_TOL * split_bound(col[None, :], Ch[:, j:j + 1])[0, 0]
    del E, X, Y
    torch.cuda.empty_cache()


@pytest.mark.parametrize("hermitian", [True, False], ids=["minresdr", "gmresdr"])
def test_restart_rotation_on_tensor_engine(hermitian):
    """GMRES-DR / MINRES-DR with one right-hand side rotate their basis at every restart,
    V_{k+1} = V_{m+1} P_{k+1}, and form the Ritz vectors E = V_k Y: with the tensor-core engine both
    products run as the split-precision FP64 emulation.  Against the FP64 engine: the same solution
    within cond(M) tol, the same Ritz values, and the final space keeps the Arnoldi relation
    A V_k = V_{k+1} Hbar_k to 1e-12 (A = M gamma_5 or M; Sec. 5.3, 5.4)."""
    dims, kappa = (4, 4, 4, 4), 0.12
    U = dev(synth.su3_links(dims, 0.3, 4))
    ctx = context(dims)
    b = ctx.noise_z4(3, 0, 1)
    solve = ctx.minresdr_solve if hermitian else ctx.gmresdr_solve
    runs = {}
    for eng in (lqcd.DEFL_FP64, lqcd.DEFL_TENSOR):
        ctx.set_defl_engine(eng)
        x, info, defl = solve(U, kappa, b, 30, 10, 1e-13, want_defl=True, eig_tol=1e-12)
        assert info["converged"] and info["true_resid"] <= 1e-13
        runs[eng] = (host(x), defl.export(), info)
    ctx.set_defl_engine(lqcd.DEFL_FP64)
    (x64, e64, _), (xtc, etc, itc) = runs[lqcd.DEFL_FP64], runs[lqcd.DEFL_TENSOR]
    assert rel_err(xtc, x64) < 10 * 12.5 * 1e-13
    assert np.allclose(np.sort_complex(etc["lam"]), np.sort_complex(e64["lam"]), rtol=1e-9, atol=1e-12)
    V, H = etc["V"], etc["Hbar"]
    k = H.shape[1]
    flags = lqcd.APPLY_G5R if hermitian else lqcd.APPLY_M
    AV = host(ctx.wilson_apply(U, kappa, V[:k].reshape((k,) + tuple(ctx.field(1).shape[1:])).contiguous(),
                               flags=flags)).reshape(k, -1)
    VH = (host(V).reshape(k + 1, -1).T @ H).T
    assert np.abs(AV - VH).max() <= 1e-12 * np.abs(AV).max()
