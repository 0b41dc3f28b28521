"""Philox4x32-10 counter-based generator, written from its published definition
(Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11).

Test infrastructure: part of the CPU oracle.  Only tests, the smoke check and the
benchmark's CPU-baseline leg use it.  The CUDA path carries its own implementation.

The DQMC proposal stream: one Philox block per proposal.  Counter words are
(event, sweep, chain, tag) and the 64-bit seed is the key (low word first).
Local moves use event = l*N + i (slice l, 0-based, site i) and tag 0; global moves
use event = i and tag 1.  The four output words give two uniforms on the 2^-53 grid:
u1 = ((w0 >> 5) * 2^26 + (w1 >> 6)) * 2^-53 and u2 likewise from (w2, w3).
"""
import numpy as np

PHILOX_M0 = 0xD2511F53
PHILOX_M1 = 0xCD9E8D57
PHILOX_W0 = 0x9E3779B9
PHILOX_W1 = 0xBB67AE85
MASK32 = 0xFFFFFFFF

TAG_LOCAL = 0
TAG_GLOBAL = 1


def philox4x32_10(counter, key):
    """Ten Philox rounds on an array of counters.

    counter: integer array of shape (..., 4) holding 32-bit words; key: two 32-bit words.
    Returns a uint64 array of shape (..., 4) holding the four 32-bit output words.
    Each round multiplies words 0 and 2 by the two round constants, keeps the high and
    low halves, and mixes in words 1 and 3 and the key; the key is bumped by the
    Weyl constants between rounds.
    """
    c = np.asarray(counter, dtype=np.uint64) & np.uint64(MASK32)
    c0, c1, c2, c3 = c[..., 0], c[..., 1], c[..., 2], c[..., 3]
    k0 = np.uint64(key[0] & MASK32)
    k1 = np.uint64(key[1] & MASK32)
    m0 = np.uint64(PHILOX_M0)
    m1 = np.uint64(PHILOX_M1)
    mask = np.uint64(MASK32)
    s32 = np.uint64(32)
    for _ in range(10):
        p0 = m0 * c0            # < 2^64: exact in uint64
        p1 = m1 * c2
        hi0, lo0 = p0 >> s32, p0 & mask
        hi1, lo1 = p1 >> s32, p1 & mask
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
        k0 = (k0 + np.uint64(PHILOX_W0)) & mask
        k1 = (k1 + np.uint64(PHILOX_W1)) & mask
    return np.stack([c0, c1, c2, c3], axis=-1)


def words_to_uniform(wa, wb):
    """53-bit uniform in [0, 1) from two 32-bit words (27 high bits of wa, 26 of wb)."""
    wa = np.asarray(wa, dtype=np.uint64)
    wb = np.asarray(wb, dtype=np.uint64)
    m = (wa >> np.uint64(5)) * np.uint64(1 << 26) + (wb >> np.uint64(6))
    return m.astype(np.float64) * (1.0 / 9007199254740992.0)


def proposal_uniforms(seed, chain, sweep, events, tag):
    """(u1, u2) arrays for the given proposal events of one chain and sweep."""
    events = np.atleast_1d(np.asarray(events, dtype=np.uint64))
    ctr = np.zeros(events.shape + (4,), dtype=np.uint64)
    ctr[..., 0] = events
    ctr[..., 1] = np.uint64(sweep)
    ctr[..., 2] = np.uint64(chain)
    ctr[..., 3] = np.uint64(tag)
    w = philox4x32_10(ctr, (seed & MASK32, (seed >> 32) & MASK32))
    return words_to_uniform(w[..., 0], w[..., 1]), words_to_uniform(w[..., 2], w[..., 3])
