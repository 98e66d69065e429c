"""Philox4x64-10 counter-based generator (oracle; test infrastructure only).

Written from the published definition (Salmon, Moraes, Dror, Shaw, "Parallel
random numbers: as easy as 1, 2, 3", SC'11): a 4x64-bit counter and a 2x64-bit
key; each of 10 rounds multiplies counter words 0 and 2 by two fixed 64-bit
constants, keeps the high and low halves of the 128-bit products and mixes
them with counter words 1, 3 and the key; the key is advanced by two Weyl
constants between rounds.  The paper does not say how its particles are
sampled (Sec. 3.1.3, Sec. 5.2.2); using a counter-based generator is a
reading made so that the CPU oracle and the CUDA path draw the same numbers
without sharing state.  Pinned against numpy.random.Philox (a 4x64-10
implementation) in tests/test_oracle_rng.py.
"""
import numpy as np

M0 = np.uint64(0xD2E7470EE14C6C93)
M1 = np.uint64(0xCA5A826395121157)
W0 = np.uint64(0x9E3779B97F4A7C15)
W1 = np.uint64(0xBB67AE8584CAA73B)
_LO32 = np.uint64(0xFFFFFFFF)
_S32 = np.uint64(32)

# purposes of the key's stream word (high byte)
PURPOSE_LOAD = 1
PURPOSE_INJECT = 2
PURPOSE_PHOTO = 3


def _mulhilo(a, b):
    """Full 64x64 -> 128-bit product of uint64 arrays: (hi, lo)."""
    a = np.asarray(a, dtype=np.uint64)
    b = np.asarray(b, dtype=np.uint64)
    al, ah = a & _LO32, a >> _S32
    bl, bh = b & _LO32, b >> _S32
    p0 = al * bl
    p1 = al * bh
    p2 = ah * bl
    p3 = ah * bh
    mid = (p0 >> _S32) + (p1 & _LO32) + (p2 & _LO32)
    lo = (p0 & _LO32) | ((mid & _LO32) << _S32)
    hi = p3 + (p1 >> _S32) + (p2 >> _S32) + (mid >> _S32)
    return hi, lo


def philox4x64(c0, c1, c2, c3, k0, k1, rounds=10):
    """Philox4x64 with `rounds` rounds on broadcastable uint64 arrays."""
    with np.errstate(over="ignore"):
        c0, c1, c2, c3 = (np.asarray(v, dtype=np.uint64) for v in (c0, c1, c2, c3))
        k0 = np.asarray(k0, dtype=np.uint64)
        k1 = np.asarray(k1, dtype=np.uint64)
        for r in range(rounds):
            if r > 0:
                k0 = k0 + W0
                k1 = k1 + W1
            hi0, lo0 = _mulhilo(M0, c0)
            hi1, lo1 = _mulhilo(M1, c2)
            c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return c0, c1, c2, c3


def stream_key(purpose, species, face, step):
    """Second key word: purpose (8 bits) | species (8) | face (8) | step (40)."""
    return np.uint64((int(purpose) << 56) | (int(species) << 48) | (int(face) << 40)
                     | (int(step) & ((1 << 40) - 1)))


def uniform(x):
    """Open-interval uniform from the top 52 bits: ((x >> 12) + 0.5) * 2^-52.

    Every operation is exact in FP64, so both implementations agree bit for bit.
    """
    return ((np.asarray(x, dtype=np.uint64) >> np.uint64(12)).astype(np.float64) + 0.5) * (2.0 ** -52)


def box_muller(u1, u2):
    """Two standard normals from two open uniforms (Box & Muller 1958)."""
    r = np.sqrt(-2.0 * np.log(u1))
    t = (2.0 * np.pi) * u2
    return r * np.cos(t), r * np.sin(t)
