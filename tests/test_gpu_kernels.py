"""GPU parity of the single-step kernels against the oracle, element by element, on seeded inputs:
Z(4) noise (bit-exact), the Wilson operator in all four forms, the contractions, the PS and POLY
series, the deflation projection, 1/xi', the Min-Res coefficients and the hopping traces.
Lattices span several thread blocks and ragged tails (odd extents, V not a multiple of 128)."""
import numpy as np
import pytest

from oracle import lattice as L, operators as O, rng, subtract as S
from paper_1903_06986_gb300 import synth
from tests.gpu_util import context, dev, host, rel_err

pytestmark = pytest.mark.gpu

DIMS = [(2, 2, 2, 2), (4, 4, 4, 4), (3, 5, 2, 7), (8, 8, 8, 16)]
FP64_TOL = 1e-14       # one operator application: a few roundings per output
CONTRACT_TOL = 1e-13   # sums of 12 V terms with compensated accumulation


def rand_fields(dims, n, seed):
    r = np.random.default_rng(seed)
    shp = L.field_shape(dims, (n,))
    return r.standard_normal(shp) + 1j * r.standard_normal(shp)


@pytest.mark.parametrize("dims", DIMS)
def test_noise_bit_exact(dims):
    ctx = context(dims)
    for seed, first, n in [(1, 0, 3), ((7 << 40) + 12345, 1000, 2), (99, rng.NOISE_SPECIAL, 2)]:
        got = host(ctx.noise_z4(seed, first, n))
        ref = rng.z4_block(seed, first, n, dims)
        assert np.array_equal(got, ref)


@pytest.mark.parametrize("dims", DIMS)
def test_wilson_all_forms(dims):
    ctx = context(dims)
    U = synth.su3_links(dims, 0.45, 3)
    kappa = 0.1537
    psi = rand_fields(dims, 3, 4)
    Ud, pd = dev(U), dev(psi)
    forms = {0: lambda f: L.wilson(U, kappa, f), 1: lambda f: L.wilson_g5(U, kappa, f),
             2: lambda f: L.wilson_dag(U, kappa, f), 3: lambda f: L.hop(U, f)}
    for flag, ref in forms.items():
        got = host(ctx.wilson_apply(Ud, kappa, pd, flags=flag))
        assert rel_err(got, ref(psi)) < FP64_TOL, flag
    # FP32 arithmetic on the same data, and FP32 storage (the inner operator of mixed precision)
    got = host(ctx.wilson_apply(Ud, kappa, pd, flags=0, prec=1))
    assert rel_err(got, forms[0](psi)) < 2e-6
    U32, p32 = ctx.to_f32(Ud), ctx.to_f32(pd)
    for flag, ref in forms.items():
        got = host(ctx.wilson_apply_f32(U32, kappa, p32, flags=flag))
        assert rel_err(got, ref(psi)) < 2e-6, flag
    # packed FP32 operator, recon 18 and 12, 1, 2 (paired lanes) and 4 right-hand sides per thread
    packed = ctx.pack_f32(pd)
    assert np.array_equal(host(ctx.unpack_f32(packed)), psi.astype(np.complex64).astype(np.complex128))
    for recon in (18, 12):
        Up = ctx.pack_links_f32(Ud, recon)
        for nr in (1, 2, 3, 4):   # 3: paired lanes with asynchronously staged neighbours
            for flag, ref in forms.items():
                got = host(ctx.unpack_f32(ctx.wilson_apply_packed(Up, recon, kappa, packed, flags=flag,
                                                                  rhs_per_thread=nr)))
                assert rel_err(got, ref(psi)) < 2e-6, (recon, nr, flag)


# unit roundoff of the storage formats: 10 and 7 stored mantissa bits, round to nearest
HALF_U = {2: 2.0 ** -11, 3: 2.0 ** -8}


@pytest.mark.parametrize("prec", [2, 3], ids=["fp16", "bf16"])
@pytest.mark.parametrize("dims", DIMS[1:3])
def test_wilson_half_storage(dims, prec):
    """FP16 / BF16 packed fields with FP32 arithmetic.  Packing scales by a power of two (exact) and
    rounds each component once, so the round trip is within u |x| per component (u the format's
    unit roundoff; the FP64 -> FP32 -> half double rounding adds at most 2^-24 relative).  The
    operator's error is the input and output rounding: ||out - ref|| <= u (||M|| ||in|| + ||ref||)
    with ||M|| <= 1 + 16 kappa (eight hopping terms of norm 2), FP32 arithmetic far below that."""
    ctx = context(dims)
    U = synth.su3_links(dims, 0.45, 3)
    kappa = 0.1537
    psi = rand_fields(dims, 3, 4)
    Ud, pd = dev(U), dev(psi)
    u = HALF_U[prec]
    packed = ctx.pack_half(pd, prec)
    back = host(ctx.unpack_half(packed, prec))
    for part in (np.real, np.imag):
        assert np.all(np.abs(part(back) - part(psi)) <= (u + 2.0 ** -24) * np.abs(part(psi)) + 1e-12)
    forms = {0: lambda f: L.wilson(U, kappa, f), 1: lambda f: L.wilson_g5(U, kappa, f),
             2: lambda f: L.wilson_dag(U, kappa, f), 3: lambda f: L.hop(U, f)}
    for nr in (1, 2, 3):   # one right-hand side per thread, two in paired lanes, or paired and staged (3 fields: one pair + odd one)
        ctx.set_rhs_per_thread(nr)
        for recon in (18, 12):
            Up = ctx.pack_links_f32(Ud, recon)
            for flag, ref in forms.items():
                want = ref(psi)
                got = host(ctx.unpack_half(ctx.wilson_apply_half(Up, recon, kappa, packed, flags=flag, prec=prec),
                                           prec))
                for r in range(3):
                    bound = u * ((1 + 16 * kappa) * np.linalg.norm(psi[r]) + np.linalg.norm(want[r]))
                    assert np.linalg.norm(got[r] - want[r]) <= bound, (nr, recon, flag, r)
                # and it is not merely within the bound by luck of a loose bound: error of order u
                assert rel_err(got, want) > 1e-3 * u
    ctx.set_rhs_per_thread(0)


@pytest.mark.parametrize("dims", DIMS[:3])
def test_contract_all_operators(dims):
    ctx = context(dims)
    U = synth.su3_links(dims, 0.5, 5)
    kappa = 0.14
    eta, w = rand_fields(dims, 2, 6), rand_fields(dims, 2, 7)
    got = ctx.contract(dev(U), kappa, dev(eta), dev(w))
    ref = O.per_t(O.densities(U, kappa, eta, w)).transpose(1, 0, 2)   # [n, op, t]
    assert rel_err(got, ref) < CONTRACT_TOL


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (3, 5, 2, 7)])
def test_hop_series_and_poly(dims):
    ctx = context(dims)
    U = synth.su3_links(dims, 0.45, 8)
    kappa = 0.15
    eta = rng.z4_block(3, 0, 2, dims)
    Ud, ed = dev(U), dev(eta)
    got = host(ctx.hop_series(Ud, kappa, ed, 7))
    assert rel_err(got, S.hop_series(U, kappa, eta, 7)) < 1e-13
    c = np.array([1.0, 0.5 - 0.25j, 2.0, -1.0, 0.1j])
    got = host(ctx.hop_series(Ud, kappa, ed, 5, c))
    ref = sum(c[k] * S.hop_series(U, kappa, eta, k + 1) - (c[k] * S.hop_series(U, kappa, eta, k) if k else 0)
              for k in range(5))
    assert rel_err(got, ref) < 1e-13
    a = np.array([6.4, -20.6, 39.4, -47.6, 36.7, -17.5, 4.7]) + 0.01j
    got = host(ctx.poly_apply(Ud, kappa, ed, a))
    assert rel_err(got, S.poly_apply(lambda f: L.wilson(U, kappa, f), a, eta)) < 1e-13


def _orthonormal(n, k, seed):
    r = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(r.standard_normal((n, k)) + 1j * r.standard_normal((n, k)))
    return Q


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (3, 5, 2, 7)])
def test_deflate_project_and_xi(dims):
    ctx = context(dims)
    U = synth.su3_links(dims, 0.45, 9)
    kappa = 0.15
    n = 12 * L.volume(dims)
    E = _orthonormal(n, 6, 10)
    lam = np.array([0.11, -0.12, 0.2, -0.25, 0.3, 0.31], dtype=np.complex128)
    defl = ctx.defl_import(dev(E.T), lam)
    eta = rng.z4_block(4, 0, 3, dims)
    d = 1.0 / lam - 0.3j
    got = host(ctx.deflate_project(defl, dev(eta), d))
    assert rel_err(got, S.defl_vector(E, d, eta)) < 1e-13
    Ud = dev(U)
    got = ctx.xi_inverse(Ud, kappa, defl, 2, 7)      # LQCD_SUB_PERT
    ref = S.xi_inverse(E, lambda f: S.hop_series(U, kappa, f, 7), dims)
    assert rel_err(got, ref) < 1e-12
    a = np.array([3.0, -4.0 + 0.1j, 2.5, -0.7])
    got = ctx.xi_inverse(Ud, kappa, defl, 4, 4, a)    # LQCD_SUB_POLY
    ref = S.xi_inverse(E, lambda f: S.poly_apply(lambda g: L.wilson(U, kappa, g), a, f), dims)
    assert rel_err(got, ref) < 1e-12


def test_poly_coeffs_minimiser():
    dims = (4, 4, 4, 4)
    ctx = context(dims)
    U = synth.su3_links(dims, 0.3, 1)
    kappa, n, seed = 0.15, 6, 17
    got = ctx.poly_coeffs(dev(U), kappa, seed, n)
    A = lambda f: L.wilson(U, kappa, f)
    b = rng.z4_noise(seed, rng.NOISE_POLY, dims)
    ref = S.poly_coeffs(A, b, n)
    # the same minimiser: residual norms agree, and P(M) b agrees
    r_got = np.linalg.norm(b - A(S.poly_apply(A, got, b)))
    r_ref = np.linalg.norm(b - A(S.poly_apply(A, ref, b)))
    assert abs(r_got - r_ref) <= 1e-10 * r_ref
    assert rel_err(S.poly_apply(A, got, b), S.poly_apply(A, ref, b)) < 1e-9
    assert rel_err(got, ref) < 1e-7


@pytest.mark.parametrize("dims,K", [((4, 4, 4, 4), 5), ((2, 2, 2, 8), 3), ((3, 2, 2, 6), 4), ((4, 4, 4, 8), 3),
                                    ((8, 4, 4, 8), 3), ((3, 3, 3, 6), 1), ((6, 6, 6, 6), 2)])
def test_hop_traces_small(dims, K):
    """The GPU probes with a sublattice colouring where the extents allow it (sum residue mod 2, the
    scaled D4 lattice, for (4,4,4,8) and (8,4,4,8) with K = 3; mod 3 for (3,3,3,6) with K = 1 and
    (6,6,6,6) with K = 2) and a Cartesian one otherwise; the oracle always uses its own Cartesian
    classes.  Probing is exact only if no two sites of a class are within K hops, so any colouring
    error shows up as a difference."""
    ctx = context(dims)
    U = synth.su3_links(dims, 0.5, 11)
    kappa = 0.13
    ref = O.per_t(S.hop_traces(U, kappa, K, dims))          # [k, op, t]
    # meet in the middle: full applications up to the depth, local completion of the orders above
    # it (0 = depth by cost, K - 1 = every order a full application)
    for depth in sorted({0, 1, 2, max(1, K - 1)}):
        ctx.set_probe_depth(depth)
        got = ctx.hop_traces(dev(U), kappa, K)
        assert rel_err(got, ref) < 1e-13, depth


def test_hop_traces_full_size_properties():
    """8^3 x 16 with K = 7 (the PS order of the paper): free field against the momentum-space
    closed form, and for an interacting field the vanishing orders (Sec. 5.1) and t_0 = 12 V."""
    from tests.test_oracle_traces import free_hop_traces
    dims, K, kappa = (8, 8, 8, 16), 7, 0.157
    ctx = context(dims)
    got = ctx.hop_traces(dev(synth.unit_links(dims)), kappa, K).sum(axis=-1)
    ref = free_hop_traces(dims, kappa, K)
    assert rel_err(got, ref) < 1e-12
    t = ctx.hop_traces(dev(synth.su3_links(dims, 0.437, 2)), kappa, K).sum(axis=-1)
    scale = abs(t[0, 0])
    assert t[0, 0] == 12 * L.volume(dims)
    for k in (1, 2, 3, 5):
        assert np.abs(t[k, 0:5]).max() < 1e-12 * scale
    for k in (0, 2, 4, 6):
        assert np.abs(t[k, 5:9]).max() < 1e-12 * scale
    assert abs(t[4, 0]) > 1.0 and abs(t[6, 0]) > 1.0
    # the meet-in-the-middle default (2 full applications, orders 3..6 completed within 4..1 hops
    # of the 16 members of each of the 512 classes) against every order applied in full
    ctx.set_probe_depth(K - 1)
    t_full = ctx.hop_traces(dev(synth.su3_links(dims, 0.437, 2)), kappa, K).sum(axis=-1)
    assert rel_err(t, t_full) < 1e-13
    ctx.set_probe_depth(0)
