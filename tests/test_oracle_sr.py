"""Pins of the oracle's stochastic-rounding reference (oracle/sr_bf16.py): the
rounding rule against exact rational arithmetic and the Philox4x32-7
generator against the properties its construction guarantees."""
from fractions import Fraction

import numpy as np
import pytest

from oracle.sr_bf16 import bf16_sr, bf16_value, philox4x32, row_draws


def _finite_f32(rng, n):
    x = rng.standard_normal(n) * 10.0 ** rng.uniform(-30, 30, n)
    return x.astype(np.float32)


def test_rule_is_unbiased_exactly():
    """Over all 2^16 draws the mean stored value is x itself, in exact
    arithmetic: x rounds up with probability (discarded low half) / 2^16."""
    rng = np.random.default_rng(1)
    r = np.arange(1 << 16, dtype=np.uint64)
    for x in _finite_f32(rng, 40):
        codes = bf16_sr(np.full(r.size, x, dtype=np.float32), r)
        vals, counts = np.unique(codes, return_counts=True)
        assert vals.size <= 2
        mean = sum(Fraction(float(bf16_value(v))) * int(c) for v, c in zip(vals, counts)) / (1 << 16)
        assert mean == Fraction(float(x)), x


def test_rule_extreme_draws_bracket_x():
    """Draw 0 truncates (toward zero in magnitude); draw 2^16 - 1 gives the next
    BF16 value away from zero unless x is already a BF16 value; infinities and
    NaNs pass through."""
    rng = np.random.default_rng(2)
    x = _finite_f32(rng, 2000)
    lo = bf16_value(bf16_sr(x, np.zeros(x.size, dtype=np.uint64)))
    hi = bf16_value(bf16_sr(x, np.full(x.size, 0xFFFF, dtype=np.uint64)))
    xd = x.astype(np.float64)
    assert np.all(np.abs(lo) <= np.abs(xd)) and np.all(np.abs(hi) >= np.abs(xd))
    exact = (x.view(np.uint32) & 0xFFFF) == 0
    assert np.array_equal(lo[exact], xd[exact]) and np.array_equal(hi[exact], xd[exact])
    ulp = np.abs(hi - lo)[~exact]
    assert np.all(ulp == np.ldexp(1.0, np.frexp(np.abs(lo[~exact]))[1] - 8))   # 8 significant bits
    special = np.array([np.inf, -np.inf, np.nan], dtype=np.float32)
    out = bf16_sr(special, np.array([0xFFFF] * 3, dtype=np.uint64))
    assert list(out[:2]) == [0x7F80, 0xFF80] and (out[2] & 0x7F80) == 0x7F80 and (out[2] & 0x7F) != 0


def test_philox_round_is_a_bijection_of_the_counter():
    """Each round is invertible for a fixed key (odd multipliers; the xor with
    the key and the swap are permutations), so distinct counters give distinct
    outputs."""
    n = 1 << 16
    ctr = np.zeros((n, 4), dtype=np.uint64)
    ctr[:, 0] = np.arange(n)
    ctr[:, 2] = np.arange(n)[::-1]
    out = philox4x32(ctr, np.array([12345, 678], dtype=np.uint64))
    words = out.astype(np.uint64)
    packed = {tuple(w) for w in words.tolist()}
    assert len(packed) == n


def test_philox_fields_uniform_and_avalanche():
    rng = np.random.default_rng(3)
    draws = row_draws(np.arange(4096), 64, step=17, seed=2022)          # 262 144 16-bit fields
    counts = np.bincount((draws >> 8).ravel(), minlength=256)           # top byte of each draw
    expected = draws.size / 256
    chi2 = float(((counts - expected) ** 2 / expected).sum())
    assert 180 < chi2 < 340, chi2                                       # 255 dof: mean 255, sd 22.6
    base = rng.integers(0, 1 << 32, size=(2000, 4), dtype=np.uint64)
    key = np.array([7, 9], dtype=np.uint64)
    flips = []
    for bit in range(128):
        c = base.copy()
        c[:, bit // 32] ^= np.uint64(1 << (bit % 32))
        d = philox4x32(base, key) ^ philox4x32(c, key)
        flips.append(np.unpackbits(d.view(np.uint8), axis=-1).sum(axis=-1).mean())
    flips = np.array(flips)
    assert abs(flips.mean() - 64.0) < 0.5 and flips.min() > 60.0, (flips.mean(), flips.min())


def test_row_draws_layout():
    """Node 8 v + 2 q + h of a row takes half h of output word q of the call
    with counter (row, v, step lo, step hi)."""
    d = row_draws([5, 6], 16, step=(3 << 32) + 11, seed=(4 << 32) + 99)
    w = philox4x32(np.array([6, 1, 11, 3], dtype=np.uint64), np.array([99, 4], dtype=np.uint64))
    for q in range(4):
        assert d[1, 8 + 2 * q] == w[q] & 0xFFFF and d[1, 8 + 2 * q + 1] == w[q] >> 16
    assert not np.array_equal(d[0], d[1])


@pytest.mark.parametrize("seed", [0, 1, 2**40 + 3])
def test_seed_changes_every_draw_stream(seed):
    a = row_draws(np.arange(64), 64, 0, seed)
    b = row_draws(np.arange(64), 64, 0, seed + 1)
    assert np.mean(a == b) < 0.01
