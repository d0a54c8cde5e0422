"""Gaussian sketch stream for the randomized SVDs (Sec. 1 and Table 1: RSVD with q iterations).

The paper draws Gaussian test matrices but does not say how; both the oracle and the CUDA
library implement the same counter-based generator so that their sketches agree:

* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2,
  3", SC'11): a 4x32-bit counter and a 2x32-bit key, ten rounds.  One round maps
  (c0,c1,c2,c3) with key (k0,k1) to (hi(M1*c2)^c1^k0, lo(M1*c2), hi(M0*c0)^c3^k1,
  lo(M0*c0)) with multipliers M0=0xD2511F53, M1=0xCD9E8D57; between rounds the key
  advances by the Weyl increments (0x9E3779B9, 0xBB67AE85).
* Two 53-bit uniforms in (0,1) from the four output words,
  u = ((w_a >> 5) * 2^26 + (w_b >> 6) + 0.5) * 2^-53.
* Box-Muller: z0 = sqrt(-2 ln u1) cos(2 pi u2), z1 = sqrt(-2 ln u1) sin(2 pi u2).

Stream layout: element e of a row-major [rows, cols] sketch uses counter
(lo32(e >> 1), hi32(e >> 1), replica, hi32(seed)) and key (lo32(seed), stream_id) and takes
z_{e mod 2}.  ``stream_id = (step << 8) | kind`` names the sketch inside an RG step.
"""
import numpy as np

M0 = np.uint64(0xD2511F53)
M1 = np.uint64(0xCD9E8D57)
W0 = np.uint32(0x9E3779B9)
W1 = np.uint32(0xBB67AE85)
_MASK32 = np.uint64(0xFFFFFFFF)

# sketch kinds inside one RG step
KIND_SWAP = 0
KIND_TRIAD = {"A": 1, "X": 2, "Y": 3, "D": 4}
KIND_SQ_LEFT = 5    # + (leg position - 1), leg positions 1..3
KIND_SQ_RIGHT = 8   # + (leg position - 1)


def stream_id(step, kind):
    return ((int(step) << 8) | int(kind)) & 0xFFFFFFFF


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Ten Philox rounds on uint32 arrays (broadcast); returns the four output words."""
    c0 = np.asarray(c0, dtype=np.uint32)
    c1 = np.asarray(c1, dtype=np.uint32)
    c2 = np.asarray(c2, dtype=np.uint32)
    c3 = np.asarray(c3, dtype=np.uint32)
    k0 = np.uint32(k0)
    k1 = np.uint32(k1)
    with np.errstate(over="ignore"):
        for rnd in range(10):
            if rnd > 0:
                k0 = np.uint32(k0 + W0)
                k1 = np.uint32(k1 + W1)
            p0 = M0 * c0.astype(np.uint64)
            p1 = M1 * c2.astype(np.uint64)
            hi0 = (p0 >> np.uint64(32)).astype(np.uint32)
            lo0 = (p0 & _MASK32).astype(np.uint32)
            hi1 = (p1 >> np.uint64(32)).astype(np.uint32)
            lo1 = (p1 & _MASK32).astype(np.uint32)
            c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return c0, c1, c2, c3


def _uniform53(wa, wb):
    a = (wa >> np.uint32(5)).astype(np.float64)
    b = (wb >> np.uint32(6)).astype(np.float64)
    return (a * 67108864.0 + b + 0.5) * (1.0 / 9007199254740992.0)


def philox_words(seed, sid, first_pair, npairs, replica=0):
    """Raw output words for counters first_pair .. first_pair+npairs-1."""
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    idx = np.arange(first_pair, first_pair + npairs, dtype=np.uint64)
    c0 = (idx & _MASK32).astype(np.uint32)
    c1 = (idx >> np.uint64(32)).astype(np.uint32)
    c2 = np.full(npairs, replica & 0xFFFFFFFF, dtype=np.uint32)
    c3 = np.full(npairs, seed >> 32, dtype=np.uint32)
    return philox4x32_10(c0, c1, c2, c3, seed & 0xFFFFFFFF, sid)


def gaussian(seed, sid, rows, cols, replica=0):
    """Row-major [rows, cols] float64 sketch of N(0,1) entries (element e -> pair e//2)."""
    n = int(rows) * int(cols)
    npairs = (n + 1) // 2
    w0, w1, w2, w3 = philox_words(seed, sid, 0, npairs, replica)
    u1 = _uniform53(w0, w1)
    u2 = _uniform53(w2, w3)
    rad = np.sqrt(-2.0 * np.log(u1))
    ang = 2.0 * np.pi * u2
    out = np.empty(2 * npairs, dtype=np.float64)
    out[0::2] = rad * np.cos(ang)
    out[1::2] = rad * np.sin(ang)
    return out[:n].reshape(rows, cols)
