"""Philox4x32-10 counter-based generator, written from its published definition
(Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3",
SC'11, section 3 and table 2).

Test infrastructure only: this module belongs to the oracle and is imported by
nothing but ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU
baseline.

The paper draws its Poisson macro-events and energies at random but names no
generator (Sec. II.D); both the oracle and the CUDA path key one Philox4x32-10
stream by (seed, step, cell, particle, stream) so that their draws coincide.

Pinned by: the generator's published known-answer vectors
(tests/golden/philox4x32_10_kat.txt) and a uniformity chi-square test.
"""
import numpy as np

_M0 = np.uint64(0xD2511F53)
_M1 = np.uint64(0xCD9E8D57)
_W0 = 0x9E3779B9
_W1 = 0xBB67AE85
_MASK = np.uint64(0xFFFFFFFF)
_S32 = np.uint64(32)


def philox4x32_10(ctr, key):
    """Apply ten Philox rounds.

    ctr: uint32 array of shape (..., 4); key: two uint32 words (k0, k1).
    Returns a uint32 array of the same shape as ctr.
    One round maps (c0, c1, c2, c3) to
    (hi(M1*c2) ^ c1 ^ k0, lo(M1*c2), hi(M0*c0) ^ c3 ^ k1, lo(M0*c0)),
    and the key is bumped by the Weyl constants between rounds.
    """
    c = np.asarray(ctr, dtype=np.uint32).astype(np.uint64)
    c0, c1, c2, c3 = c[..., 0], c[..., 1], c[..., 2], c[..., 3]
    k0 = int(key[0]) & 0xFFFFFFFF
    k1 = int(key[1]) & 0xFFFFFFFF
    for r in range(10):
        p0 = _M0 * c0
        p1 = _M1 * c2
        hi0, lo0 = p0 >> _S32, p0 & _MASK
        hi1, lo1 = p1 >> _S32, p1 & _MASK
        c0 = hi1 ^ c1 ^ np.uint64(k0)
        c1 = lo1
        c2 = hi0 ^ c3 ^ np.uint64(k1)
        c3 = lo0
        k0 = (k0 + _W0) & 0xFFFFFFFF
        k1 = (k1 + _W1) & 0xFFFFFFFF
    out = np.stack([c0, c1, c2, c3], axis=-1)
    return out.astype(np.uint32)


def uniform23(word):
    """Map a 32-bit word to a uniform in (0, 1): ((word >> 9) + 0.5) * 2**-23.

    The top 23 bits are used so that the value, and every comparison made
    with it, is exact in binary32 as well as binary64.
    """
    w = np.asarray(word, dtype=np.uint32)
    return ((w >> np.uint32(9)).astype(np.float64) + 0.5) * (2.0 ** -23)


def split_seed(seed):
    """Key words (k0, k1) = (low, high) 32 bits of a 64-bit seed."""
    s = int(seed) & 0xFFFFFFFFFFFFFFFF
    return (s & 0xFFFFFFFF, s >> 32)
