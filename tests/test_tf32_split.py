"""The arithmetic of the fine pass's TF32 operands, checked on the CPU: the
integer rounding the converters use (half an ulp of the 11-bit significand
added to the magnitude bits, 13 low bits cleared) is round-to-nearest with ties
away from zero, each part carries at most 11 significant bits (zero low 13
bits, what kind::tf32 reads), and x = x_h + x_m + x_l to 2^-33 |x|; the six
products of order >= 2^-22 give a b to about 2^-32 relative."""
import numpy as np


def tf32_round(x):
    b = np.asarray(x, dtype=np.float32).view(np.uint32)
    return ((b + np.uint32(0x1000)) & np.uint32(0xFFFFE000)).view(np.float32)


def nearest_tf32_ties_away(x):
    # independent route in fp64: the two TF32 neighbours of x and the closer one
    x = np.asarray(x, dtype=np.float64)
    e = np.floor(np.log2(np.abs(x)))
    ulp = 2.0 ** (e - 10)  # 11 significant bits
    lo = np.floor(np.abs(x) / ulp) * ulp
    hi = lo + ulp
    d_lo, d_hi = np.abs(x) - lo, hi - np.abs(x)
    mag = np.where(d_hi <= d_lo, hi, lo)  # a tie goes up in magnitude: away from zero
    return np.sign(x) * mag


def _samples(n=200000, seed=0):
    rng = np.random.default_rng(seed)
    x = (rng.standard_normal(n) * np.exp(rng.uniform(-30, 30, n))).astype(np.float32)
    # exact ties: 11 significant bits plus a half unit
    t = (rng.integers(1 << 10, 1 << 11, 2000).astype(np.float64) + 0.5) * 2.0 ** rng.integers(-20, 20, 2000)
    t *= rng.choice([-1.0, 1.0], 2000)
    return np.concatenate([x, t.astype(np.float32)])


def test_integer_rounding_is_nearest_ties_away():
    x = _samples()
    x = x[np.abs(x) > 1e-30]
    h = tf32_round(x)
    assert np.all((h.view(np.uint32) & np.uint32(0x1FFF)) == 0)
    assert np.array_equal(h.astype(np.float64), nearest_tf32_ties_away(x.astype(np.float64)))


def test_three_part_split_is_exact_to_2_33():
    x = _samples(seed=1)
    h = tf32_round(x)
    r1 = (x - h).astype(np.float32)
    # x - h is exact in fp32 (h is within half a TF32 ulp of x)
    assert np.array_equal(r1.astype(np.float64), x.astype(np.float64) - h.astype(np.float64))
    m = tf32_round(r1)
    l = tf32_round((r1 - m).astype(np.float32))
    for part in (h, m, l):
        assert np.all((part.view(np.uint32) & np.uint32(0x1FFF)) == 0)
    err = np.abs(x.astype(np.float64) - (h.astype(np.float64) + m + l))
    assert np.all(err <= 2.0 ** -33 * np.abs(x.astype(np.float64)))


def test_six_products_reproduce_the_product():
    rng = np.random.default_rng(2)
    a = rng.standard_normal(100000).astype(np.float32)
    b = rng.standard_normal(100000).astype(np.float32)

    def parts(x):
        h = tf32_round(x)
        r = (x - h).astype(np.float32)
        m = tf32_round(r)
        return h.astype(np.float64), m.astype(np.float64), tf32_round((r - m).astype(np.float32)).astype(np.float64)

    ah, am, al = parts(a)
    bh, bm, bl = parts(b)
    six = am * bm + al * bh + ah * bl + am * bh + ah * bm + ah * bh
    exact = a.astype(np.float64) * b.astype(np.float64)
    assert np.all(np.abs(six - exact) <= 2.0 ** -30 * np.abs(exact))
