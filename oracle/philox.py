"""Philox4x32-10 counter-based RNG and the Z4 noise vectors (oracle side).

Philox4x32-10 is the generator of Salmon, Moraes, Dror and Shaw, "Parallel
random numbers: as easy as 1, 2, 3" (SC'11): a 4x32-bit counter and a 2x32-bit
key, ten rounds; each round multiplies counter words 0 and 2 by the constants
0xD2511F53 and 0xCD9E8D57, splits the 64-bit products into (hi, lo) and
recombines them with the other two words and the key by XOR; the key is
advanced by the Weyl increments (0x9E3779B9, 0xBB67AE85) between rounds.
The CUDA path implements the same published definition separately.

Noise definition (the Z4 vectors of Eq. (test) and Eq. (fs_trace_est), entries
drawn from {1, -1, i, -i} with equal probability):
  key     = (seed mod 2^32, seed >> 32)
  counter = (site, sample, level, job)       site in canonical order
  out     = Philox4x32-10(counter, key)
  for spin s, colour c, j = 3 s + c:  k = (out[0] >> 2 j) & 3,  z = i^k.
A gamma_5-rotated vector gamma_5 z flips the sign of spins 2 and 3.
Independent vectors per level (Sec. 4.1: noise "independent for each level")
come from the distinct `level` counter word. `variance_sample` uses the level
word VARIANCE_SAMPLE_LEVEL.
"""

import numpy as np

PHILOX_M0 = 0xD2511F53
PHILOX_M1 = 0xCD9E8D57
PHILOX_W0 = 0x9E3779B9
PHILOX_W1 = 0xBB67AE85
MASK32 = 0xFFFFFFFF

VARIANCE_SAMPLE_LEVEL = 0x80000000


def _mulhilo(a, b):
    prod = np.uint64(a) * b.astype(np.uint64)
    return (prod >> np.uint64(32)).astype(np.uint64), (prod & np.uint64(MASK32)).astype(np.uint64)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Vectorised Philox4x32-10. Counter words are uint arrays (broadcast), key scalars.

    Returns four uint32 arrays.
    """
    c = [np.asarray(w, dtype=np.uint64) & np.uint64(MASK32) for w in (c0, c1, c2, c3)]
    c = np.broadcast_arrays(*c)
    c = [w.copy() for w in c]
    k0 = int(k0) & MASK32
    k1 = int(k1) & MASK32
    for rnd in range(10):
        if rnd > 0:
            k0 = (k0 + PHILOX_W0) & MASK32
            k1 = (k1 + PHILOX_W1) & MASK32
        hi0, lo0 = _mulhilo(PHILOX_M0, c[0])
        hi1, lo1 = _mulhilo(PHILOX_M1, c[2])
        c = [hi1 ^ c[1] ^ np.uint64(k0), lo1, hi0 ^ c[3] ^ np.uint64(k1), lo0]
    return [w.astype(np.uint32) for w in c]


def z4_codes(volume, seed, job, level, sample):
    """Integer codes k in {0,1,2,3} (z = i^k), uint8[V][4][3]."""
    site = np.arange(volume, dtype=np.uint64)
    out0 = philox4x32_10(site, sample, level, job, seed & MASK32, (seed >> 32) & MASK32)[0]
    out0 = out0.astype(np.uint64)
    j = np.arange(12, dtype=np.uint64)
    k = (out0[:, None] >> (np.uint64(2) * j[None, :])) & np.uint64(3)
    return k.astype(np.uint8).reshape(volume, 4, 3)


def z4_noise(volume, seed, job, level, sample, gamma5=False):
    """Z4 noise vector complex128[V][4][3]; gamma5=True returns gamma_5 z."""
    k = z4_codes(volume, seed, job, level, sample)
    z = (1j ** k.astype(np.int64)).astype(np.complex128)
    if gamma5:
        z[:, 2:, :] *= -1.0
    return z
