"""Z(4) noise (Sec. 2; the paper uses Z(N) noise with N = 4) from a counter-based generator.

Test infrastructure (see ``oracle/__init__.py``).

The paper does not name its random number generator.  Reading: Philox-4x32-10 of Salmon,
Moraes, Dror and Shaw, "Parallel random numbers: as easy as 1, 2, 3" (SC'11), written here from
that paper's definition:
  * state: four 32-bit counter words (c0, c1, c2, c3) and two 32-bit key words (k0, k1);
  * one round: (hi0, lo0) = 0xD2511F53 * c0 and (hi1, lo1) = 0xCD9E8D57 * c2 as 64-bit products,
    then  (c0, c1, c2, c3) <- (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0);
  * ten rounds; between rounds the key is bumped by the Weyl constants (0x9E3779B9, 0xBB67AE85).

Noise entry (reading): key = (seed & 0xffffffff, seed >> 32); counter = (noise index n, site s,
0, 0); word 0 of the output supplies the 12 entries of the site, entry c = 3*spin + colour taking
bits 2c and 2c+1, mapped 0 -> 1, 1 -> i, 2 -> -1, 3 -> -i.  Entries are uniform in {1, i, -1, -i}
as Sec. 2 / Sec. 3 require (<eta_i eta_j^*> = delta_ij, <eta_i> = 0, <eta_i^2> = 0).
"""
import numpy as np

PHILOX_M0 = np.uint64(0xD2511F53)
PHILOX_M1 = np.uint64(0xCD9E8D57)
PHILOX_W0 = np.uint64(0x9E3779B9)
PHILOX_W1 = np.uint64(0xBB67AE85)
MASK32 = np.uint64(0xFFFFFFFF)

# reserved noise indices for the two special right-hand sides (readings of Sec. 5.2 / Sec. 7)
NOISE_POLY = 0xFFFFFFFF          # the "single noise vector" of the Min-Res polynomial
NOISE_SPECIAL = 0xFFFFFFFE       # the super-convergence right-hand side of GMRES-DR / MINRES-DR


def philox4x32_10(ctr, key):
    """ctr: uint array (..., 4); key: uint array (..., 2) (broadcastable).  Returns uint32 (..., 4)."""
    c = [np.asarray(ctr[..., i], dtype=np.uint64) & MASK32 for i in range(4)]
    k0 = np.asarray(key[..., 0], dtype=np.uint64) & MASK32
    k1 = np.asarray(key[..., 1], dtype=np.uint64) & MASK32
    for r in range(10):
        if r > 0:
            k0 = (k0 + PHILOX_W0) & MASK32
            k1 = (k1 + PHILOX_W1) & MASK32
        p0 = PHILOX_M0 * c[0]            # < 2^64: exact in uint64
        p1 = PHILOX_M1 * c[2]
        hi0, lo0 = p0 >> np.uint64(32), p0 & MASK32
        hi1, lo1 = p1 >> np.uint64(32), p1 & MASK32
        c = [(hi1 ^ c[1] ^ k0) & MASK32, lo1, (hi0 ^ c[3] ^ k1) & MASK32, lo0]
    return np.stack(c, axis=-1).astype(np.uint32)


Z4_VALUES = np.array([1, 1j, -1, -1j], dtype=np.complex128)


def z4_noise(seed, noise_index, dims):
    """One Z(4) noise field of shape (T, Z, Y, X, 4, 3) for the given seed and noise index."""
    v = int(np.prod(dims))
    s = np.arange(v, dtype=np.uint64)
    ctr = np.zeros((v, 4), dtype=np.uint64)
    ctr[:, 0] = np.uint64(noise_index)
    ctr[:, 1] = s
    key = np.array([seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF], dtype=np.uint64)
    w0 = philox4x32_10(ctr, key[None, :])[:, 0].astype(np.uint64)
    codes = np.stack([(w0 >> np.uint64(2 * c)) & np.uint64(3) for c in range(12)], axis=-1)
    vals = Z4_VALUES[codes.astype(np.int64)]
    lx, ly, lz, lt = dims
    return vals.reshape(lt, lz, ly, lx, 4, 3)


def z4_block(seed, first_noise, count, dims):
    """Noises first_noise .. first_noise+count-1 stacked on a leading axis."""
    return np.stack([z4_noise(seed, first_noise + n, dims) for n in range(count)])
