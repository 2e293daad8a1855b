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
