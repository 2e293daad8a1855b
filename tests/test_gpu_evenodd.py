"""GPU parity of the even/odd (Schur complement) system with the oracle (Sec. 7): the split of
fields by parity (bit-exact), the hopping blocks P_eo / P_oe and the reduced operator hat M in its
three forms (1e-14), the reduced right-hand side and reconstruction, reduced GMRES-DR / MINRES-DR /
GMRES-Proj solves against the dense LU solution of the full M, and the full eigenpairs of M built
from reduced ones."""
import numpy as np
import pytest

from oracle import evenodd as EO, exact as X, lattice as L
from paper_1903_06986_gb300 import lqcd, synth
from tests.gpu_util import dev, host, rel_err, torch_cuda

pytestmark = pytest.mark.gpu

DIMS = (4, 2, 6, 4)   # non-cubic, every extent even


def eo_context(dims):
    torch_cuda()
    from paper_1903_06986_gb300 import build
    build.build()
    return lqcd.EvenOddContext(dims)


def rand_full(dims, n, seed):
    r = np.random.default_rng(seed)
    shp = L.field_shape(dims, (n,))
    return r.standard_normal(shp) + 1j * r.standard_normal(shp)


def test_split_join_bit_exact():
    ctx = eo_context(DIMS)
    b = rand_full(DIMS, 3, 1)
    e, o = ctx.split(dev(b))
    we, wo = EO.split(b, DIMS)
    assert np.array_equal(host(e), we) and np.array_equal(host(o), wo)
    assert np.array_equal(host(ctx.join(e, o)), b)


def test_hop_blocks_and_reduced_operator():
    ctx = eo_context(DIMS)
    U = synth.su3_links(DIMS, 0.5, 11)
    kappa = 0.137
    b = rand_full(DIMS, 2, 2)
    ve, vo = EO.split(b, DIMS)
    Ud = dev(U)
    got_eo = host(ctx.hop(Ud, dev(vo), 0))
    got_oe = host(ctx.hop(Ud, dev(ve), 1))
    for r in range(2):
        assert rel_err(got_eo[r], EO.hop_eo(U, vo[r], DIMS)) < 1e-14
        assert rel_err(got_oe[r], EO.hop_oe(U, ve[r], DIMS)) < 1e-14
    g5s = lambda v: np.einsum("ab,...bc->...ac", np.kron(np.array([[0, -1], [-1, 0]]), np.eye(2)), v)
    for flags, ref in ((lqcd.APPLY_M, lambda v: EO.reduced_apply(U, kappa, v, DIMS)),
                       (lqcd.APPLY_G5R, lambda v: EO.reduced_apply(U, kappa, g5s(v), DIMS)),
                       (lqcd.APPLY_DAG, lambda v: g5s(EO.reduced_apply(U, kappa, g5s(v), DIMS)))):
        got = host(ctx.wilson_apply(Ud, kappa, dev(ve), flags=flags))
        for r in range(2):
            assert rel_err(got[r], ref(ve[r])) < 1e-14, flags
    # hat M gamma_5 is Hermitian: <a, B c> = <B a, c>
    a, c = dev(ve[0:1]), dev(ve[1:2])
    Ba = host(ctx.wilson_apply(Ud, kappa, a, flags=lqcd.APPLY_G5R))
    Bc = host(ctx.wilson_apply(Ud, kappa, c, flags=lqcd.APPLY_G5R))
    lhs, rhs = np.vdot(host(a), Bc), np.vdot(Ba, host(c))
    assert abs(lhs - rhs) <= 1e-13 * abs(lhs)


def test_rhs_and_reconstruct():
    ctx = eo_context(DIMS)
    U = synth.su3_links(DIMS, 0.5, 12)
    kappa = 0.13
    b = rand_full(DIMS, 2, 3)
    xe = EO.split(rand_full(DIMS, 2, 4), DIMS)[0]
    Ud = dev(U)
    be = host(ctx.rhs(Ud, kappa, dev(b)))
    x = host(ctx.reconstruct(Ud, kappa, dev(xe), dev(b)))
    for r in range(2):
        assert rel_err(be[r], EO.reduced_rhs(U, kappa, b[r], DIMS)) < 1e-14
        assert rel_err(x[r], EO.reconstruct(U, kappa, xe[r], b[r], DIMS)) < 1e-14


@pytest.mark.parametrize("hermitian", [False, True], ids=["gmresdr", "minresdr"])
def test_reduced_solve_matches_lu(hermitian):
    """Reduced solve + reconstruction = the dense LU solution of the full M (cond(M) = 12.5 at
    kappa 0.12: solutions to 1e-13 agree within cond * tol), and GMRES-Proj over the reduced space."""
    dims = (2, 2, 2, 4)
    ctx = eo_context(dims)
    U = synth.su3_links(dims, 0.45, 2)
    kappa = 0.12
    Ud = dev(U)
    b = rand_full(dims, 3, 5)
    be = ctx.rhs(Ud, kappa, dev(b))
    tol = 1e-13
    if hermitian:
        ye, info, defl = ctx.minresdr_solve(Ud, kappa, be[:1].contiguous(), 30, 8, tol, want_defl=True)
        xe0 = torch_cuda().from_numpy(np.ascontiguousarray(np.einsum(
            "ab,...bc->...ac", np.kron(np.array([[0, -1], [-1, 0]]), np.eye(2)), host(ye)))).cuda()
    else:
        xe0, info, defl = ctx.gmresdr_solve(Ud, kappa, be[:1].contiguous(), 30, 8, tol, want_defl=True)
    assert info["converged"] and info["true_resid"] <= tol
    Minv = X.inverse(U, kappa, dims)
    xs = [L.unflat(Minv @ L.flat(b[r]), dims) for r in range(3)]
    x0 = host(ctx.reconstruct(Ud, kappa, xe0, dev(b[:1])))
    assert rel_err(x0[0], xs[0]) < 10 * 12.5 * tol
    # the remaining right-hand sides by GMRES-Proj over the reduced deflation space
    sysm = lqcd.SYS_MG5 if hermitian else lqcd.SYS_M
    y, pinfo = ctx.proj_solve(Ud, kappa, defl, be[1:].contiguous(), 12, tol, system=sysm)
    assert pinfo["converged"] and pinfo["true_resid"] <= tol
    ye = host(y)
    if hermitian:
        ye = np.einsum("ab,...bc->...ac", np.kron(np.array([[0, -1], [-1, 0]]), np.eye(2)), ye)
    x = host(ctx.reconstruct(Ud, kappa, dev(ye), dev(b[1:])))
    for r in range(2):
        assert rel_err(x[r], xs[r + 1]) < 10 * 12.5 * tol


def test_full_eigenpairs_from_reduced():
    """Reduced pairs (mu, v_e) from the GMRES-DR space of hat M -> full pairs of M: the same vectors as
    the oracle's map on the same input (1e-13), and M v = lambda v to the reduced residual level."""
    dims = (2, 2, 2, 4)
    ctx = eo_context(dims)
    U = synth.su3_links(dims, 0.45, 2)
    kappa = 0.12
    Ud = dev(U)
    be = ctx.rhs(Ud, kappa, dev(rand_full(dims, 1, 6)))
    _, _, defl = ctx.gmresdr_solve(Ud, kappa, be, 40, 10, 1e-14, want_defl=True, eig_tol=1e-13)
    ex = defl.export()
    mu, Ve = ex["lam"], ex["E"]
    lam, E = ctx.full_eigenpairs(Ud, kappa, mu, Ve)
    lam_o, E_o = EO.full_eigenpairs(U, kappa, mu, host(Ve).reshape(len(mu), -1, 4, 3), dims)
    assert np.allclose(lam, lam_o, rtol=0, atol=1e-14)
    assert rel_err(host(E), E_o) < 1e-13
    Eh = host(E)
    for q in range(len(lam)):
        res = np.linalg.norm(L.wilson(U, kappa, Eh[q]) - lam[q] * Eh[q])
        assert res < 1e-9, (q, res)


def test_full_lattice_entry_points_refused():
    ctx = eo_context(DIMS)
    with pytest.raises(lqcd.LqcdError):
        ctx.noise_z4(1, 0, 1, out=ctx.full_field(1))
    with pytest.raises(lqcd.LqcdError):
        ctx.loop_estimate(dev(synth.su3_links(DIMS, 0.5, 1)), 0.12, 1, 2, 2, 10, 3, 4, 3, 1e-10, 1e-10)


@pytest.mark.parametrize("system", [lqcd.SYS_M, lqcd.SYS_MG5], ids=["M", "MG5"])
def test_loop_estimate_evenodd_equals_full_system(system):
    """The loop estimate with the noise solves on the reduced system equals the one on the full system
    (same noises, same subtraction spaces; solves to 3e-14 at cond(M) = 12.5) and the oracle's, for
    the NS, PS, POLY, HFES, HFPS and HFPOLY modes (1e-11 relative per noise and operator)."""
    from oracle import pipeline as PL
    dims, kappa = (2, 2, 2, 4), 0.12
    ctx = lqcd.Context(dims)
    U = synth.su3_links(dims, 0.45, 2)
    Ud = dev(U)
    modes = lqcd.SUB_ALL & ~lqcd.SUB_ES
    kw = dict(m=40, k=8, K=7, npoly=4, tol=3e-14, tol_special=1e-14, eig_tol=1e-13, modes=modes, system=system)
    full = ctx.loop_estimate(Ud, kappa, 3, 6, 3, **kw)
    eo = ctx.loop_estimate(Ud, kappa, 3, 6, 3, evenodd=1, **kw)
    assert eo["converged"] and eo["max_true_resid"] <= 3e-14
    for mode in range(6):
        want = full["per_noise"][mode]
        scale = np.abs(want).max(axis=0)
        assert np.all(np.abs(eo["per_noise"][mode] - want) <= 1e-11 * scale), mode
    ref, _, _ = PL.loop_estimate(U, kappa, dims, 3, 6, 40, 8, 7, 4, 3e-14, 1e-14, eig_tol=1e-13,
                                 system="MG5" if system == lqcd.SYS_MG5 else "M",
                                 modes=["none", "pert", "poly", "defl", "defl_pert", "defl_poly"])
    for mode, name in enumerate(("none", "pert", "poly", "defl", "defl_pert", "defl_poly")):
        want = ref[name]["per_noise"]
        scale = np.abs(want).max(axis=0)
        assert np.all(np.abs(eo["per_noise"][mode] - want) <= 1e-11 * scale), name


def test_loop_estimate_evenodd_es_from_reduced_pairs():
    """ES on the even/odd path takes the full eigenpairs of M built from the reduced Ritz pairs: each
    per-noise ES estimate equals the oracle's ES estimate with the oracle's map of the same reduced
    pairs (e_L from gamma_5-hermiticity, Sec. 5.3) applied to the exact solution."""
    from oracle import operators as OP, subtract as SB, rng
    dims, kappa = (2, 2, 2, 4), 0.12
    ctx = lqcd.Context(dims)
    ectx = eo_context(dims)
    U = synth.su3_links(dims, 0.45, 2)
    Ud = dev(U)
    kw = dict(m=40, k=8, K=7, npoly=4, tol=3e-14, tol_special=1e-14, eig_tol=1e-13, modes=lqcd.SUB_ES)
    got = ctx.loop_estimate(Ud, kappa, 3, 4, 4, evenodd=1, **kw)
    assert got["converged"]
    # the same reduced space: GMRES-DR on hat M for the reduced special right-hand side
    bs = ctx.noise_z4(3, 0xFFFFFFFE, 1)
    be = ectx.rhs(Ud, kappa, bs)
    _, _, defl = ectx.gmresdr_solve(Ud, kappa, be, 40, 8, 1e-14, eig_tol=1e-13, want_defl=True)
    ex = defl.export()
    lam, E = EO.full_eigenpairs(U, kappa, ex["lam"], host(ex["E"]).reshape(8, -1, 4, 3), dims)
    ER = E.reshape(len(lam), -1).T
    EL, found = SB.es_left_vectors(ER, lam, dims)
    assert found.any()
    ER, EL, lam = ER[:, found], EL[:, found], lam[found]
    add = SB.es_addback(U, kappa, ER, EL, lam, dims).reshape(9, -1).sum(axis=-1)
    Minv = X.inverse(U, kappa, dims)
    for n in range(4):
        eta = rng.z4_noise(3, n, dims)
        x = L.unflat(Minv @ L.flat(eta), dims)
        xt = SB.es_vector(ER, EL, lam, eta)
        want = OP.densities(U, kappa, eta, x - xt).reshape(9, -1).sum(axis=-1) + add
        g = got["per_noise"][6][n]
        assert np.all(np.abs(g - want) <= 1e-10 * np.abs(want).max()), n
