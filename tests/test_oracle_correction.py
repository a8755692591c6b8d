"""Pins of the oracle's detector correction (Section 1.2; Eq. 1 numerator):
gain-level decode, closed-form photon values, and the two-rounding binary32
definition checked against exact rational arithmetic."""
from fractions import Fraction

import numpy as np
import pytest

import oracle


def rn32(q: Fraction) -> float:
    """Round an exact rational to the nearest binary32 (ties to even), written
    from the IEEE 754 definition (normal range only)."""
    if q == 0:
        return 0.0
    s = -1 if q < 0 else 1
    a = abs(q)
    e = a.numerator.bit_length() - a.denominator.bit_length()
    if Fraction(2) ** e > a:
        e -= 1
    ulp = Fraction(2) ** (e - 23)
    m = a / ulp                      # in [2^23, 2^24)
    lo = m.numerator // m.denominator
    rem = m - lo
    if rem > Fraction(1, 2) or (rem == Fraction(1, 2) and lo % 2 == 1):
        lo += 1
    return float(s * lo * ulp)


def test_decode_levels():
    # levels 0, 1, 2 from the two top bits; code 2 is read as level 2
    ped = np.array([[100.0] * 4, [200.0] * 4, [300.0] * 4], np.float32)
    gain = np.array([[1.0] * 4, [1.0] * 4, [1.0] * 4], np.float32)
    raw = np.array([0x0000 | 1000, 0x4000 | 1000, 0x8000 | 1000, 0xC000 | 1000], np.uint16)
    out = oracle.jf_photons(raw, ped, gain)
    assert out.tolist() == [900.0, 800.0, 700.0, 700.0]


def test_closed_form_photons():
    # level 0: (1400 - 1000) / 40 = 10; level 1 (negative gain): (13850 - 14000) / -1.5 = 100
    # level 2: (10000 - 15000) / RN32(-0.1) = 49999.99925... -> RN32 = 50000
    raw = np.array([1400, 0x4000 | 13850, 0xC000 | 10000], np.uint16)
    ped = np.array([[1000, 0, 0], [0, 14000, 0], [0, 0, 15000]], np.float32)
    gain = np.array([[40, 1, 1], [1, -1.5, 1], [1, 1, -0.1]], np.float32)
    assert oracle.jf_photons(raw, ped, gain).tolist() == [10.0, 100.0, 50000.0]


def test_all_raw_codes_two_binary32_roundings():
    """Every 16-bit raw word against exact rationals with the rounding applied
    twice, once after the subtraction and once after the division."""
    rng = np.random.default_rng(7)
    n = 1 << 16
    raw = np.arange(n, dtype=np.uint16)
    ped = np.stack([rng.normal(m, s, n) for m, s in ((1500, 50), (14000, 200), (15000, 200))]).astype(np.float32)
    gain = np.stack([40 * (1 + rng.uniform(-.02, .02, n)), -1.5 * (1 + rng.uniform(-.02, .02, n)),
                     -0.1 * (1 + rng.uniform(-.02, .02, n))]).astype(np.float32)
    out = oracle.jf_photons(raw, ped, gain)
    lvl = np.where(raw >> 14 == 0, 0, np.where(raw >> 14 == 1, 1, 2))
    adc = (raw & 0x3FFF).astype(np.int64)
    differs_from_single_rounding = 0
    for i in range(0, n, 7):  # a stride keeps the exact-rational loop quick
        p = Fraction(float(ped[lvl[i], i]))
        g = Fraction(float(gain[lvl[i], i]))
        x = rn32(Fraction(int(adc[i])) - p)
        want = rn32(Fraction(x) / g)
        assert out[i] == want, (i, out[i], want)
        if rn32((Fraction(int(adc[i])) - p) / g) != want:
            differs_from_single_rounding += 1
    # the definition matters: rounding once (e.g. in binary64, then to
    # binary32) would give other values for some of these words
    assert differs_from_single_rounding > 0
