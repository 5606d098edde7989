"""Stochastic rounding of FP32 values to BF16 storage, with the random bits
drawn from the Philox4x32 counter-based generator (Salmon, Moraes, Dror and
Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC 2011), 7 rounds.

TEST INFRASTRUCTURE ONLY (imported by tests; never by the product library).

The paper stores f_1 in double precision and draws no random numbers; BF16
storage of delta f is this implementation's precision pattern.  Its rounding
rule: add 16 uniformly drawn bits r to the low half of the FP32 bit pattern
and keep the high half, so x rounds away from its truncation with probability
(discarded fraction) and the stored value equals x in expectation.  The bits
of a stored 16-byte vector (8 nodes) come from one generator call with the
counter (row, vector index, step mod 2^32, step >> 32) and the key
(seed mod 2^32, seed >> 32): output word q holds node 2q in its low and node
2q + 1 in its high 16 bits.  This module writes both the generator and the
rule out from their definitions, vectorised over numpy arrays.

Parity pins (tests/test_oracle_sr.py): the rule's expectation is x exactly
(exact rational arithmetic over all 2^16 draws); draws 0 and 2^16 - 1 give
the two bracketing BF16 values; the generator's round is a bijection of the
counter for a fixed key, its 16-bit fields are uniform (chi-square) and one
flipped counter bit changes half the output bits on average (avalanche).
"""
from __future__ import annotations

import numpy as np

# Philox4x32 constants (Salmon et al. 2011): the two round multipliers and
# the Weyl-sequence key increments (golden ratio and sqrt(3) - 1 in 0.32 fixed point).
PHILOX_M0 = 0xD2511F53
PHILOX_M1 = 0xCD9E8D57
PHILOX_W0 = 0x9E3779B9
PHILOX_W1 = 0xBB67AE85
MASK32 = 0xFFFFFFFF


def _mulhilo(m: int, x: np.ndarray):
    p = np.uint64(m) * x.astype(np.uint64)
    return (p >> np.uint64(32)).astype(np.uint64), (p & np.uint64(MASK32)).astype(np.uint64)


def philox4x32(ctr, key, rounds: int = 7):
    """Philox4x32-R on counters ctr [..., 4] and keys key [..., 2] (broadcast),
    as uint32 words.  One round: (hi, lo) = M0 * c0 and M1 * c2 as 64-bit
    products; c <- (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0); the key is bumped by
    the Weyl increments between rounds."""
    ctr = np.asarray(ctr, dtype=np.uint64)
    key = np.asarray(key, dtype=np.uint64)
    c0, c1, c2, c3 = (ctr[..., i] for i in range(4))
    k0, k1 = key[..., 0], key[..., 1]
    for r in range(rounds):
        if r:
            k0 = (k0 + np.uint64(PHILOX_W0)) & np.uint64(MASK32)
            k1 = (k1 + np.uint64(PHILOX_W1)) & np.uint64(MASK32)
        hi0, lo0 = _mulhilo(PHILOX_M0, c0)
        hi1, lo1 = _mulhilo(PHILOX_M1, c2)
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return np.stack([c0, c1, c2, c3], axis=-1).astype(np.uint32)


def bf16_sr(x, r16):
    """FP32 values x (any shape) rounded to BF16 bit patterns (uint16) with the
    draws r16 (same shape, 0 <= r16 < 2^16).  Infinities and NaNs keep their
    high half."""
    b = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    special = (b & np.uint64(0x7F800000)) == np.uint64(0x7F800000)
    up = (b + np.asarray(r16, dtype=np.uint64)) >> np.uint64(16)
    return np.where(special, b >> np.uint64(16), up).astype(np.uint16)


def bf16_value(code):
    """BF16 bit patterns to their values (float64, exact)."""
    c = np.asarray(code, dtype=np.uint32) << np.uint32(16)
    return c.view(np.float32).astype(np.float64)


def row_draws(rows, nnodes: int, step: int, seed: int):
    """The 16-bit draws of nodes 0..nnodes-1 (a multiple of 8) of the given
    delta-f rows at time step `step`: array [len(rows), nnodes]."""
    rows = np.asarray(rows, dtype=np.uint64)
    nvec = nnodes // 8
    vi = np.arange(nvec, dtype=np.uint64)
    ctr = np.zeros((rows.size, nvec, 4), dtype=np.uint64)
    ctr[..., 0] = (rows & np.uint64(MASK32))[:, None]
    ctr[..., 1] = vi[None, :]
    ctr[..., 2] = step & MASK32
    ctr[..., 3] = (step >> 32) & MASK32
    key = np.array([seed & MASK32, (seed >> 32) & MASK32], dtype=np.uint64)
    w = philox4x32(ctr, key).astype(np.uint32)                  # [rows, nvec, 4]
    lo, hi = w & np.uint32(0xFFFF), w >> np.uint32(16)
    return np.stack([lo, hi], axis=-1).reshape(rows.size, nvec * 8)   # node 8 v + 2 q + h
