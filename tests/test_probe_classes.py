"""CPU checks of the probing colouring the GPU hopping traces use (host logic of the library, no
GPU): every class is a set of sites pairwise more than K hops apart on the torus (the condition
under which probing gives the exact t_k, Sec. 5.1: K - 1 hops of P^k plus the one hop of a
point-split operator), every class is used, and the sublattice colourings give the expected,
small class counts."""
import shutil

import numpy as np
import pytest

from paper_1903_06986_gb300 import build, lqcd


@pytest.fixture(scope="module", autouse=True)
def lib():
    if shutil.which("nvcc") is None and not __import__("os").path.exists(build.LIB):
        pytest.skip("nvcc not available")
    build.build()


def min_same_class_distance(dims, cls):
    """Smallest torus L1 distance between two distinct sites of one class (brute force per class)."""
    lx, ly, lz, lt = dims
    t, z, y, x = np.meshgrid(np.arange(lt), np.arange(lz), np.arange(ly), np.arange(lx), indexing="ij")
    coords = np.stack([x.ravel(), y.ravel(), z.ravel(), t.ravel()], axis=1)
    ext = np.array(dims)
    flat = cls.ravel()
    best = np.inf
    for c in np.unique(flat):
        pts = coords[flat == c]
        if len(pts) < 2:
            continue
        d = np.abs(pts[:, None, :] - pts[None, :, :])
        d = np.minimum(d, ext - d).sum(axis=-1)
        np.fill_diagonal(d, np.iinfo(d.dtype).max)
        best = min(best, d.min())
    return best


@pytest.mark.parametrize("dims,K,expect", [
    ((8, 8, 8, 16), 7, 2 * 4 ** 4),       # scaled D4 (sum residue mod 2)
    ((12, 12, 12, 12), 7, 3 * 4 ** 4),    # sum residue mod 3
    ((12, 12, 12, 24), 7, 3 * 4 ** 4),
    ((16, 16, 16, 16), 7, 2 * 4 ** 4),
    ((6, 6, 6, 6), 2, 3 * 2 ** 4),
    ((3, 3, 3, 6), 1, 3),
    ((4, 4, 4, 8), 3, 2 * 2 ** 4),
    ((4, 4, 4, 4), 5, 4 ** 4),            # Cartesian fallback: every site its own class
    ((3, 2, 2, 6), 4, 3 * 2 * 2 * 6),
    ((10, 5, 7, 14), 3, 5 * 5 * 7 * 7),   # Cartesian periods 5, 5, 7, 7
])
def test_classes_are_far_apart_and_small_in_number(dims, K, expect):
    n, cls = lqcd.probe_classes(dims, K)
    assert n == expect
    assert cls.min() == 0 and cls.max() == n - 1 and len(np.unique(cls)) == n
    assert min_same_class_distance(dims, cls) > K


def test_bad_arguments_are_rejected():
    with pytest.raises(lqcd.LqcdError):
        lqcd.probe_classes((1, 4, 4, 4), 3)
    with pytest.raises(lqcd.LqcdError):
        lqcd.probe_classes((4, 4, 4, 4), 0)


def ball_size(r):
    """Number of points of Z^4 within taxicab distance r (counted directly)."""
    rng_ = np.arange(-r, r + 1)
    g = np.stack(np.meshgrid(rng_, rng_, rng_, rng_, indexing="ij"), axis=-1)
    return int((np.abs(g).sum(axis=-1) <= r).sum())


def site_updates(h, K, per_member):
    """Site updates per probe and lattice volume of the meet-in-the-middle traces at depth h: h full
    applications, then order k evaluated within max(1, K - k) hops of each class member (or in full
    where that ball holds more sites than a member's share of the lattice)."""
    return h + sum(min(1.0, ball_size(max(1, K - k)) / per_member) for k in range(h + 1, K))


@pytest.mark.parametrize("dims,K,expect", [((24, 24, 24, 32), 7, 2), ((8, 8, 8, 16), 7, 2), ((16, 16, 16, 32), 7, 2),
                                           ((12, 12, 12, 24), 7, None), ((2, 2, 2, 4), 7, None), ((4, 4, 4, 4), 5, None),
                                           ((8, 4, 4, 8), 3, 1), ((6, 6, 6, 6), 2, 1), ((3, 3, 3, 6), 1, 0)])
def test_probe_depth_minimises_site_updates(dims, K, expect):
    """The depth of the hopping traces (meet in the middle, Sec. 5.1 add-back): a depth of least site
    updates per probe, every completion ball within 8 hops, the first order above it a real local
    completion (its ball smaller than a member's share of the lattice): the depth counts the full
    applications, 2 of the 6 orders at K = 7 with 512 classes."""
    depth = lqcd.probe_depth(dims, K)
    if expect is not None:
        assert depth == expect
    if K <= 2:
        assert depth == K - 1
        return
    ncls, _ = lqcd.probe_classes(dims, K)
    costs = {h: site_updates(h, K, ncls) for h in range(1, K) if max(1, K - h - 1) <= 8}
    best = min(costs.values())
    assert costs[depth] <= best + 1e-9
    if depth < K - 1:
        assert ball_size(max(1, K - depth - 1)) < ncls


def test_probe_depth_fixed_values():
    """A fixed depth is capped at K - 1 and raised where a completion would reach beyond 8 hops."""
    assert lqcd.probe_depth((8, 8, 8, 16), 7, fixed=1) == 1
    assert lqcd.probe_depth((8, 8, 8, 16), 7, fixed=9) == 6
    assert lqcd.probe_depth((16, 16, 16, 32), 20, fixed=1) == 11
    with pytest.raises(lqcd.LqcdError):
        lqcd.probe_depth((8, 8, 8, 16), 7, fixed=-1)
    with pytest.raises(lqcd.LqcdError):
        lqcd.probe_depth((1, 8, 8, 16), 7)
