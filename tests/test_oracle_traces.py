"""Pins of the oracle's traces: free-field closed forms in momentum space (an independent route to
Tr(Theta M^{-1}) and to t_k = Tr(Theta P^k)), brute-force dense traces, the vanishing orders of the
hopping expansion (Sec. 5.1), and the Re/Im structure implied by gamma_5-hermiticity (Sec. 6)."""
import itertools

import numpy as np
import pytest

from oracle import exact, lattice as L, operators as O, subtract as S
from paper_1903_06986_gb300 import synth


def momenta(dims):
    return itertools.product(*[[2 * np.pi * n / l for n in range(l)] for l in dims])


def P_of_p(p):
    """Spin matrix of the free hopping operator on exp(i p.x) u:  sum_mu (1-g)e^{ip} + (1+g)e^{-ip}."""
    return sum((L.ONE4 - L.G[m]) * np.exp(1j * p[m]) + (L.ONE4 + L.G[m]) * np.exp(-1j * p[m])
               for m in range(4))


def free_hop_traces(dims, kappa, K):
    out = np.zeros((K, O.NOPS), dtype=np.complex128)
    for p in momenta(dims):
        Pp = P_of_p(p)
        Pk = np.eye(4, dtype=np.complex128)
        for k in range(K):
            if k > 0:
                Pk = Pk @ Pp
            out[k, 0] += 3 * np.trace(Pk)
            for mu in range(4):
                out[k, 1 + mu] += 3 * np.trace(L.G[mu] @ Pk)
                out[k, 5 + mu] += 3 * kappa * (np.exp(-1j * p[mu]) * np.trace((L.ONE4 + L.G[mu]) @ Pk)
                                               - np.exp(1j * p[mu]) * np.trace((L.ONE4 - L.G[mu]) @ Pk))
    return out


def free_inverse_traces(dims, kappa):
    out = np.zeros(O.NOPS, dtype=np.complex128)
    for p in momenta(dims):
        Mp = np.eye(4) - kappa * P_of_p(p)
        W = np.linalg.inv(Mp)
        out[0] += 3 * np.trace(W)
        for mu in range(4):
            out[1 + mu] += 3 * np.trace(L.G[mu] @ W)
            out[5 + mu] += 3 * kappa * (np.exp(-1j * p[mu]) * np.trace((L.ONE4 + L.G[mu]) @ W)
                                        - np.exp(1j * p[mu]) * np.trace((L.ONE4 - L.G[mu]) @ W))
    return out


@pytest.mark.parametrize("dims,K", [((2, 4, 2, 4), 5), ((4, 4, 2, 6), 4)])
def test_free_field_hop_traces(dims, K):
    kappa = 0.13
    U = synth.unit_links(dims)
    t = S.hop_traces(U, kappa, K, dims).sum(axis=(-1, -2, -3, -4))
    ref = free_hop_traces(dims, kappa, K)
    assert np.allclose(t, ref, atol=1e-10 * max(1.0, np.abs(ref).max()))


def test_free_field_scalar_closed_form():
    """Tr M^{-1} = sum_p 12 A / (A^2 + |B|^2); vector traces vanish (odd in p)."""
    dims = (2, 2, 4, 4)
    kappa = 0.1
    U = synth.unit_links(dims)
    tr = exact.exact_traces(U, kappa, dims)
    closed = 0.0
    for p in momenta(dims):
        A = 1 - 2 * kappa * sum(np.cos(q) for q in p)
        B2 = sum((2 * kappa * np.sin(q)) ** 2 for q in p)
        closed += 12 * A / (A * A + B2)
    assert abs(tr[0] - closed) < 1e-11 * abs(closed)
    assert np.allclose(tr, free_inverse_traces(dims, kappa), atol=1e-11)
    assert np.abs(tr[1:]).max() < 1e-11


def test_hop_traces_brute_force_dense():
    dims = (2, 2, 2, 2)
    U = synth.su3_links(dims, 0.7, 4)
    kappa, K = 0.12, 5
    t = S.hop_traces(U, kappa, K, dims).sum(axis=(-1, -2, -3, -4))
    P = L.dense(lambda v: L.hop(U, v), dims)
    for op in range(O.NOPS):
        Th = exact.dense_theta(U, kappa, op, dims)
        Pk = np.eye(P.shape[0], dtype=np.complex128)
        for k in range(K):
            if k > 0:
                Pk = Pk @ P
            assert abs(np.trace(Th @ Pk) - t[k, op]) < 1e-10 * max(1.0, abs(t[k, op]))


def test_hop_traces_vanishing_orders():
    """Closed paths only (Sec. 5.1): on even extents >= 4, local t_1..t_3 and all odd local orders
    vanish, point-split even orders vanish; local t_4 (plaquettes) and point-split t_3 do not."""
    dims = (4, 4, 4, 4)
    U = synth.su3_links(dims, 0.5, 11)
    kappa, K = 0.15, 6
    t = S.hop_traces(U, kappa, K, dims).sum(axis=(-1, -2, -3, -4))
    scale = abs(t[0, 0])
    for k in (1, 2, 3, 5):
        assert np.abs(t[k, 0:5]).max() < 1e-12 * scale
    for k in (0, 2, 4):
        assert np.abs(t[k, 5:9]).max() < 1e-12 * scale
    assert abs(t[4, 0]) > 1.0
    assert np.abs(t[3, 5:9]).min() > 1e-3
    assert t[0, 0] == 12 * 256


def test_coloured_probing_equals_unit_probing():
    dims = (2, 2, 2, 8)
    U = synth.su3_links(dims, 0.6, 12)
    kappa, K = 0.14, 3
    full = S.hop_traces(U, kappa, K, dims, spacing=dims)
    assert S.default_spacing(dims, K) == (2, 2, 2, 4)
    col = S.hop_traces(U, kappa, K, dims)
    assert np.allclose(full, col, atol=1e-13)


def test_exact_trace_symmetries():
    """gamma_5-hermiticity makes Tr(M^{-1}) real and every vector trace imaginary (Sec. 6);
    traces are gauge invariant."""
    dims = (2, 2, 4, 4)
    U = synth.su3_links(dims, 0.5, 13)
    kappa = 0.14
    tr = exact.exact_traces(U, kappa, dims)
    assert abs(tr[0].imag) < 1e-11 * abs(tr[0])
    assert np.abs(tr[1:].real).max() < 1e-11 * abs(tr[0])
    g = synth.su3_links(dims, 2.0, 14)[0]
    Ug = np.empty_like(U)
    for mu in range(4):
        gfwd = np.roll(g, -1, axis=L.SITE_AXIS[mu])
        Ug[mu] = g @ U[mu] @ np.conj(np.swapaxes(gfwd, -1, -2))
    assert np.allclose(exact.exact_traces(Ug, kappa, dims), tr, atol=1e-11)


@pytest.mark.parametrize("dims,K", [((4, 2, 2, 4), 5), ((8, 2, 2, 2), 3), ((10, 2, 3, 2), 4), ((2, 2, 2, 2), 7)])
def test_meet_in_the_middle_traces_equal_probing(dims, K):
    """The meet-in-the-middle form (local operators from two half-depth probe blocks joined by
    gamma_5-hermiticity, point-split operators completed only near the class members) gives the
    per-site densities of full-depth probing, including classes with several members ((8,2,2,2),
    (10,2,3,2)), odd extents and windings (2^4, K = 7)."""
    U = synth.su3_links(dims, 0.6, 21)
    kappa = 0.14
    ref = S.hop_traces(U, kappa, K, dims)
    got = S.hop_traces_meet(U, kappa, K, dims)
    assert np.abs(got - ref).max() < 1e-12 * max(1.0, np.abs(ref).max())


def test_meet_in_the_middle_needs_its_completion_radius():
    """Cutting the completed orders one hop closer to the members than max(1, K - k) changes the
    point-split traces: the radius is the smallest that keeps them exact (odd extents, so that the
    even point-split orders, which the cut reaches, do not vanish)."""
    dims, K = (3, 2, 2, 3), 5
    U = synth.su3_links(dims, 0.6, 22)
    kappa = 0.14
    ref = S.hop_traces(U, kappa, K, dims).sum(axis=(-1, -2, -3, -4))
    cut = S.hop_traces_meet(U, kappa, K, dims, completion_radius=lambda K_, k: max(1, K_ - k) - 1)
    cut = cut.sum(axis=(-1, -2, -3, -4))
    assert np.abs(cut[:, 5:] - ref[:, 5:]).max() > 1e-3
    assert np.abs(cut[:, :5] - ref[:, :5]).max() < 1e-11 * np.abs(ref).max()
