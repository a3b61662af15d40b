"""The library converts between FP64 and FP32 with integer operations (GB300 runs the conversion
instructions on its scarce FP64 pipe): f32_rn rounds to nearest even for results in the normal FP32
range and zeros, f64_of widens normal numbers and zeros. A numpy restatement of the same integer
steps equals numpy's own conversions (IEEE round to nearest even) on random doubles, on exact
half-way cases, at the edges of the normal range and across the carry into the exponent."""
import numpy as np

LO, HI, REBIAS = 0x3810000000000000, 0x47F0000000000000, 0x3800000000000000


def f32_rn_int(x):
    b = np.asarray(x, np.float64).view(np.uint64)
    a = b & np.uint64(0x7FFFFFFFFFFFFFFF)
    sgn = ((b >> np.uint64(32)) & np.uint64(0x80000000)).astype(np.uint32)
    inr = (a - np.uint64(LO)) < np.uint64(HI - LO)
    m = a - np.uint64(REBIAS)
    m = m + np.uint64(0x0FFFFFFF) + ((m >> np.uint64(29)) & np.uint64(1))
    f = (m >> np.uint64(29)).astype(np.uint32) | sgn
    f = np.where(a == 0, sgn, f)
    return f.view(np.float32), inr | (a == 0)


def f64_of_int(f):
    u = np.asarray(f, np.float32).view(np.uint32)
    a = u & np.uint32(0x7FFFFFFF)
    sgn = (u & np.uint32(0x80000000)).astype(np.uint64) << np.uint64(32)
    normal = (a - np.uint32(0x00800000)) < np.uint32(0x7F800000 - 0x00800000)
    m = ((a.astype(np.uint64) << np.uint64(29)) + np.uint64(REBIAS)) | sgn
    m = np.where(a == 0, sgn, m)
    return m.view(np.float64), normal | (a == 0)


def test_narrowing_equals_round_to_nearest_even():
    rng = np.random.default_rng(7)
    x = np.concatenate([
        rng.standard_normal(200000) * 10.0 ** rng.uniform(-40, 40, 200000),
        rng.uniform(-1, 1, 50000),
        [0.0, -0.0, 1.0, -1.0, 2.0 ** -126, -(2.0 ** -126), np.finfo(np.float32).max],
    ])
    # exact half-way points between neighbouring floats (ties to even) and their neighbours
    f = rng.standard_normal(50000).astype(np.float32)
    nxt = np.nextafter(f, np.float32(np.inf))
    half = (f.astype(np.float64) + nxt.astype(np.float64)) / 2.0
    x = np.concatenate([x, half, np.nextafter(half, np.inf), np.nextafter(half, -np.inf)])
    # the largest floats: rounding past FLT_MAX gives infinity
    big = np.float64(np.finfo(np.float32).max)
    x = np.concatenate([x, [big * (1 + 2.0 ** -25), big * (1 + 2.0 ** -23), 2.0 ** 127 * 1.99999999999]])
    got, handled = f32_rn_int(x)
    with np.errstate(over="ignore"):
        want = x.astype(np.float32)
    assert handled.sum() > 200000
    assert np.array_equal(got[handled].view(np.uint32), want[handled].view(np.uint32))


def test_widening_is_exact():
    rng = np.random.default_rng(8)
    f = np.concatenate([(rng.standard_normal(200000) * 10.0 ** rng.uniform(-37, 37, 200000)).astype(np.float32),
                        np.array([0.0, -0.0, 1.0, np.finfo(np.float32).tiny, np.finfo(np.float32).max], np.float32)])
    got, handled = f64_of_int(f)
    assert handled.sum() > 199000          # the rest (denormals, infinities) go to the instruction
    assert np.array_equal(got[handled].view(np.uint64), f[handled].astype(np.float64).view(np.uint64))
