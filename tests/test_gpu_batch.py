"""Batching on the GPU: CUDA-graph replay of the Krylov cycles, the block-width autotuner, and
concurrent loop estimates of lattices of uneven size.  Each batched or replayed result is compared
with the direct single-problem path (which the pipeline tests compare with the oracle) and, for
one lattice, with the oracle itself."""
import numpy as np
import pytest

from oracle import estimate as E, pipeline as PL, rng
from paper_1903_06986_gb300 import lqcd, synth
from tests.gpu_util import context, dev, host, rel_err

pytestmark = pytest.mark.gpu

KAPPA = 0.14


def test_graph_replay_is_bit_identical():
    """The Arnoldi steps replayed from a captured graph run the same kernels on the same data: the
    GMRES-DR and GMRES-Proj iterates agree bit for bit with direct launches (FP64 and the FP32,
    FP16 and BF16 inner solvers, one after another on one context, so graphs of one storage type
    are never replayed for another), and the launch count is the same."""
    dims = (4, 4, 4, 4)
    ctx = context(dims)
    U = dev(synth.su3_links(dims, 0.3, 5))
    b = ctx.noise_z4(3, 0, 4)
    out = {}
    for graphs in (False, True):
        ctx.set_graphs(graphs)
        l0 = ctx.launches
        x, info, defl = ctx.gmresdr_solve(U, KAPPA, b[:1].contiguous(), 20, 5, 1e-12, 200, want_defl=True)
        res = [host(x), info["cycles"]]
        for prec in (0, 1, 2, 3, 0):      # the repeat replays graphs cached by the first call
            y, pinfo = ctx.proj_solve(U, KAPPA, defl, b, 15, 1e-10, 200, prec=prec)
            assert pinfo["converged"] and pinfo["true_resid"] <= 1e-10, prec
            res += [host(y), pinfo["cycles"]]
        out[graphs] = res + [ctx.launches - l0]
    for a, g in zip(out[False], out[True]):
        assert np.array_equal(a, g)


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_autotune_picks_the_fastest_candidate(prec):
    dims = (4, 4, 4, 4)
    ctx = context(dims)
    U = dev(synth.su3_links(dims, 0.3, 6))
    b0 = ctx.noise_z4(1, rng.NOISE_SPECIAL, 1)
    _, _, defl = ctx.gmresdr_solve(U, KAPPA, b0, 20, 5, 1e-12, 200, want_defl=True)
    best, secs = ctx.autotune_block(U, KAPPA, defl, 15, candidates=(2, 4, 8), prec=prec)
    assert best in (2, 4, 8) and all(v > 0 for v in secs.values())
    assert secs[best] == min(secs.values())


def test_autotuned_block_gives_the_same_estimates():
    """block = 0 (autotuned among 8 and 16 for 16 noises) and a fixed block width solve every noise
    independently to the same tolerance: the estimates agree within the solver tolerance."""
    dims = (4, 4, 4, 4)
    ctx = context(dims)
    U = dev(synth.su3_links(dims, 0.3, 6))
    kw = dict(seed=4, nnoise=16, m=20, k=5, K=4, npoly=3, tol=1e-11, tol_special=1e-12)
    auto = ctx.loop_estimate(U, KAPPA, block=0, **kw)
    fixed = ctx.loop_estimate(U, KAPPA, block=4, **kw)
    assert auto["block"] in (8, 16) and fixed["block"] == 4
    assert auto["converged"] and fixed["converged"]
    assert rel_err(auto["per_noise"], fixed["per_noise"]) < 1e-9


def test_batch_of_uneven_lattices_matches_single_runs_and_oracle():
    """Three lattices of different shapes solved concurrently: every estimate equals the one of the
    same problem run alone (same kernels, same data, deterministic reductions), and the smallest
    lattice matches the oracle's loop estimate."""
    shapes = [(2, 2, 2, 4), (4, 4, 2, 4), (2, 4, 4, 6)]
    kw = dict(seed=7, nnoise=6, block=6, m=80, k=8, K=4, npoly=3, tol=1e-13, tol_special=1e-14, eig_tol=1e-13)
    probs, single = [], []
    for i, dims in enumerate(shapes):
        ctx = context(dims)
        U = dev(synth.su3_links(dims, 0.4, 20 + i))
        single.append(ctx.loop_estimate(U, KAPPA, **kw))
        probs.append(dict(ctx=lqcd.Context(dims), links=U, kappa=KAPPA, **kw))
    res = lqcd.batch_loop_estimate(probs)
    for r, s in zip(res, single):
        assert r["status"] == lqcd.OK and r["converged"]
        assert np.array_equal(r["per_noise"], s["per_noise"])
        assert np.array_equal(r["mean"], s["mean"])
    dims = shapes[0]
    ref, _, _ = PL.loop_estimate(synth.su3_links(dims, 0.4, 20), KAPPA, dims, 7, 6, 80, 8, 4, 3, 1e-13, 1e-14,
                                 eig_tol=1e-13)
    for mi, mode in enumerate(E.MODES):
        # the Min-Res coefficients (POLY modes) agree only to cond(v) * eps; the other modes at 1e-11
        tol = 1e-9 if mode in ("poly", "defl_poly") else 1e-11
        got, want = res[0]["mean"][mi], ref[mode]["mean"]
        assert np.all(np.abs(got - want) <= tol * np.abs(want).max()), mode
