"""Pins of the oracle's counter generator (published Philox-4x32-10 known answers) and of the
Z(4) noise properties used in Sec. 2-3 (<eta> = 0, <eta_i eta_j^*> = delta_ij, <eta^2> = 0)."""
import os

import numpy as np

from oracle import rng

GOLD = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def load_kat():
    rows = []
    for line in open(GOLD):
        if line.startswith("#") or not line.strip():
            continue
        v = [int(t, 16) for t in line.split()]
        rows.append((v[0:4], v[4:6], v[6:10]))
    return rows


def test_philox_known_answers():
    for ctr, key, out in load_kat():
        got = rng.philox4x32_10(np.array(ctr, dtype=np.uint64), np.array(key, dtype=np.uint64))
        assert [int(g) for g in got] == out


def test_z4_values_and_norm():
    dims = (4, 4, 2, 2)
    eta = rng.z4_noise(12345, 7, dims)
    vals = set(np.round(eta.ravel(), 12).tolist())
    assert vals <= {1, 1j, -1, -1j}
    assert np.vdot(eta, eta).real == 12 * 64


def test_z4_reproducible_and_distinct():
    dims = (2, 2, 2, 2)
    a = rng.z4_noise(1, 0, dims)
    assert np.array_equal(a, rng.z4_noise(1, 0, dims))
    assert not np.array_equal(a, rng.z4_noise(1, 1, dims))
    assert not np.array_equal(a, rng.z4_noise(2, 0, dims))


def test_z4_moments():
    dims = (2, 2, 2, 4)
    N = 400
    etas = rng.z4_block(99, 0, N, dims).reshape(N, -1)
    n = etas.shape[1]
    # <eta_i> = 0 and <eta_i^2> = 0: each mean has standard error 1/sqrt(N)
    assert np.abs(etas.mean(axis=0)).max() < 5.5 / np.sqrt(N)
    assert np.abs((etas ** 2).mean(axis=0)).max() < 5.5 / np.sqrt(N)
    # <eta_i eta_j^*> = delta_ij: diagonal exactly 1, off-diagonal O(1/sqrt(N))
    X = etas.T @ etas.conj() / N
    assert np.allclose(np.diag(X), 1.0)
    off = X - np.diag(np.diag(X))
    assert np.abs(off).max() < 5.5 / np.sqrt(N)
    # the four values are equally likely (chi-square, 3 dof, 99.9% quantile 16.27)
    codes = np.round(np.angle(etas) / (np.pi / 2)).astype(int) % 4
    cnt = np.bincount(codes.ravel(), minlength=4)
    e = codes.size / 4
    assert ((cnt - e) ** 2 / e).sum() < 16.27
