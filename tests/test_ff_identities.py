"""The float-float identity the FP32-bulk Halpern step with reflection 1
relies on, checked in IEEE single precision on the CPU: the TwoSum-based
difference of two (hi, lo) pairs is odd in its arguments,

    sub(a, b) == -sub(b, a)   (bit for bit, except the sign of a zero),

because the TwoSum error term is exact and round-to-nearest is symmetric.
The primal step therefore takes z_0 - x_bar as the negated anchor difference
x_bar - z_0 it already formed.  (The pair operations are restated here from
their published definition, Knuth's TwoSum followed by a renormalisation.)"""
import numpy as np

f32 = np.float32


def two_sum_sub(ah, al, bh, bl):
    # (ah, al) - (bh, bl): TwoSum of the high parts, low parts added, renormalised
    s = f32(ah - bh)
    bb = f32(s - ah)
    err = f32(f32(ah - f32(s - bb)) + f32(f32(-bh) - bb))
    t = f32(err + f32(al - bl))
    h = f32(s + t)
    b2 = f32(h - s)
    lo = f32(f32(s - f32(h - b2)) + f32(t - b2))
    return h, lo


def _pairs(rng, n, scale):
    hi = (rng.standard_normal(n) * scale).astype(np.float32)
    lo = (hi.astype(np.float64) * rng.uniform(-2.0 ** -25, 2.0 ** -25, n)).astype(np.float32)
    return hi, lo


def test_pair_difference_is_odd_bit_for_bit():
    rng = np.random.default_rng(3)
    with np.errstate(all="ignore"):
        for scale_a, scale_b in ((1.0, 1.0), (1e-3, 1.0), (1.0, 1e-6), (1e4, 1e4), (1e-20, 1e-20)):
            ah, al = _pairs(rng, 20000, scale_a)
            bh, bl = _pairs(rng, 20000, scale_b)
            # near-cancelling pairs too
            bh[:5000] = ah[:5000] * f32(1.0 + 2.0 ** -20)
            h1, l1 = two_sum_sub(ah, al, bh, bl)
            h2, l2 = two_sum_sub(bh, bl, ah, al)
            for u, v in ((h1, h2), (l1, l2)):
                assert np.array_equal(u, -v)  # equal values (a zero may differ in sign)
                nz = u != 0
                assert np.array_equal(u[nz].view(np.uint32), (-v[nz]).view(np.uint32))


def test_pair_difference_keeps_the_exact_difference():
    # the pair (h, lo) carries the difference to within about 2^-48 of the
    # operands' size, the precision the float-float iterates rely on
    rng = np.random.default_rng(5)
    ah, al = _pairs(rng, 20000, 1.0)
    bh, bl = _pairs(rng, 20000, 0.5)
    h, lo = two_sum_sub(ah, al, bh, bl)
    exact = (ah.astype(np.float64) + al) - (bh.astype(np.float64) + bl)
    got = h.astype(np.float64) + lo.astype(np.float64)
    size = np.abs(ah.astype(np.float64)) + np.abs(bh.astype(np.float64))
    assert np.max(np.abs(got - exact) / size) < 2.0 ** -46
