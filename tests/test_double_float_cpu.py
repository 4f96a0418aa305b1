"""Host restatement (numpy float32) of the double-float arithmetic of the
top-k panel products that need float64 accuracy (DF, panel_in<DF> and
panel_fma<DF> in paper_1511_00152_gb300/csrc/topk.cu), checked against exact
rational arithmetic and float64.

Split: a float64 x becomes h + l, h = x rounded toward zero to float32 (from
the bit pattern), l = the dropped low 29 mantissa bits rounded to float32.
Product and accumulation: p = fl(a.h b.h), e = the exact error of that
product (an FMA), plus the cross terms a.h b.l and a.l b.h; the pair
(p, e) is added to the accumulator (s.h, s.l) with Knuth's TwoSum on s.h
and p.  The claims pinned here: h + l equals x to 2^-48 relative; one
product is within about 2^-44 of the exact product of the two float64
inputs; a 4096-term dot product lands within 1e-12 (relative to the sum
of the products' magnitudes) of the exact value, over a thousand times
closer than the float32 sum of the rounded products."""
from fractions import Fraction

import numpy as np
import pytest

f32 = np.float32


def to_f32_rz(x):
    """float64 -> float32 rounded toward zero, from the bits (normal range)."""
    u = np.float64(x).view(np.uint64)
    sign = int(u >> np.uint64(63))
    e = int((u >> np.uint64(52)) & np.uint64(0x7FF)) - 1023 + 127
    mant = int((u >> np.uint64(29)) & np.uint64(0x7FFFFF))
    if e <= 0:
        return f32(0.0)
    assert e < 255
    bits = (sign << 31) | (e << 23) | mant
    return np.array([bits], dtype=np.uint32).view(np.float32)[0]


def f64_tail(x):
    """The low 29 mantissa bits of x as a float32 (rounded to nearest)."""
    u = int(np.float64(x).view(np.uint64))
    e = ((u >> 52) & 0x7FF) - 1023 - 52
    m29 = u & 0x1FFFFFFF
    if m29 == 0 or e < -126 or e > 127 - 29:
        return f32(0.0)
    v = f32(m29) * f32(2.0) ** e  # m29 -> float32 rounds to nearest; the scale is exact
    return -v if (u >> 63) else v


def split(x):
    h = to_f32_rz(x)
    return (h, f32(0.0) if h == 0 else f64_tail(x))


def round_f32(q):
    """The float32 nearest to the rational q (ties to even)."""
    f = f32(float(q))
    cands = [np.nextafter(f, f32(-np.inf)), f, np.nextafter(f, f32(np.inf))]
    best = min(cands, key=lambda c: (abs(Fraction(float(c)) - q),
                                     int(np.array([c], dtype=np.float32).view(np.uint32)[0]) & 1))
    return f32(best)


def fma32(a, b, c):
    """Single-rounding float32 fused multiply-add (exact product and sum in
    rationals, one rounding to float32 at the end)."""
    return round_f32(Fraction(float(a)) * Fraction(float(b)) + Fraction(float(c)))


def df_fma(a, b, acc):
    p = f32(a[0] * b[0])
    e = fma32(a[0], b[0], -p)
    e = fma32(a[0], b[1], e)
    e = fma32(a[1], b[0], e)
    t = f32(acc[0] + p)
    z = f32(t - acc[0])
    err = f32(f32(acc[0] - f32(t - z)) + f32(p - z))
    return (t, f32(acc[1] + f32(err + e)))


def value(d):
    return Fraction(float(d[0])) + Fraction(float(d[1]))


def test_split_is_exact_to_2_pow_48():
    rng = np.random.default_rng(1)
    for x in np.concatenate([rng.standard_normal(2000) * 10.0 ** rng.integers(-8, 8, 2000),
                             [1.0, -1.0, 0.1, 1 / 3, np.pi, 2.0 ** -100, 1e30]]):
        h, l = split(x)
        err = abs(Fraction(float(x)) - (Fraction(float(h)) + Fraction(float(l))))
        assert err <= abs(Fraction(float(x))) * Fraction(1, 2 ** 48), x
        # h carries the leading 24 bits: |l| below one ulp of h
        assert abs(float(l)) <= np.spacing(np.float32(abs(h))) or h == 0


def test_one_product_within_2_pow_44():
    rng = np.random.default_rng(2)
    xs = rng.standard_normal(400) * 10.0 ** rng.integers(-4, 4, 400)
    ys = rng.standard_normal(400)
    for x, y in zip(xs, ys):
        r = df_fma(split(x), split(y), (f32(0.0), f32(0.0)))
        exact = Fraction(float(x)) * Fraction(float(y))
        assert abs(value(r) - exact) <= abs(exact) * Fraction(1, 2 ** 44), (x, y)


@pytest.mark.parametrize("n", [256, 4096])
def test_dot_product_to_float64_accuracy(n):
    rng = np.random.default_rng(n)
    c = rng.standard_normal(n)
    v = rng.standard_normal(n) / np.sqrt(n)
    acc = (f32(0.0), f32(0.0))
    plain = f32(0.0)
    for x, y in zip(c, v):
        acc = df_fma(split(x), split(y), acc)
        plain = f32(plain + f32(f32(x) * f32(y)))
    exact = sum(Fraction(float(x)) * Fraction(float(y)) for x, y in zip(c, v))
    scale = sum(abs(Fraction(float(x)) * Fraction(float(y))) for x, y in zip(c, v))
    err_df = float(abs(value(acc) - exact) / scale)
    err_f32 = float(abs(Fraction(float(plain)) - exact) / scale)
    assert err_df <= 1e-12, err_df
    # what the float32 panels would give: many orders of magnitude worse
    assert err_f32 > 1e3 * err_df
