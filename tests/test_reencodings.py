"""The integer re-encodings between binary32 and binary64 that the mixed
shape-tensor inverse uses in place of the hardware conversions (which issue
on the FP64 pipe), restated on the host with numpy integer operations and
checked bit for bit against numpy's IEEE conversions (binary32 -> binary64
exact; binary64 -> binary32 round to nearest, ties to even).

- binary32 -> binary64 (flushed): for |f| >= 2^-40 the exponent is re-biased
  by 1023 - 127 and the 23-bit fraction moves to the top of the 52-bit one;
  smaller |f| (zero, subnormals) give a zero of the same sign.
- binary64 -> binary32 (regular range): a funnel shift keeps the top 23
  fraction bits below the low 9 exponent bits, adding 2^30 re-biases that
  exponent modulo 2^9, the 29 dropped bits decide the rounding (above half:
  up; exactly half: up when the kept lsb is odd), and a carry out of the
  fraction moves into the exponent.  Valid for zero and for values whose
  rounded result is a normal binary32 number.

No GPU is used."""
import numpy as np

M32 = np.uint64(0xFFFFFFFF)


def f32_to_f64_flushed(f):
    u = np.asarray(f, np.float32).view(np.uint32).astype(np.uint64)
    mag = u & np.uint64(0x7FFFFFFF)
    keep = mag >= np.uint64(0x2B800000)                      # |f| >= 2^-40
    hi = (u & np.uint64(0x80000000)) | np.where(keep, (mag >> np.uint64(3)) + np.uint64(0x38000000),
                                                np.uint64(0))
    lo = np.where(keep, (u << np.uint64(29)) & M32, np.uint64(0))
    return ((hi << np.uint64(32)) | lo).view(np.float64)


def f64_to_f32_regular(d):
    b = np.asarray(d, np.float64).view(np.uint64)
    hi, lo = b >> np.uint64(32), b & M32
    f = (((hi << np.uint64(3)) | (lo >> np.uint64(29))) + np.uint64(0x40000000)) & M32
    rem = lo & np.uint64(0x1FFFFFFF)
    f = f + ((rem + (f & np.uint64(1))) > np.uint64(0x10000000)).astype(np.uint64)
    f = np.where((hi & np.uint64(0x7FFFFFFF)) != 0, f & M32, np.uint64(0))
    return (f | (hi & np.uint64(0x80000000))).astype(np.uint32).view(np.float32)


def test_binary32_to_binary64_is_exact_over_every_exponent():
    rng = np.random.default_rng(1)
    # every exponent and sign, random fractions, plus the fraction extremes
    e = np.repeat(np.arange(256, dtype=np.uint32), 4096)
    frac = rng.integers(0, 1 << 23, e.size, dtype=np.uint32)
    frac[::4096] = 0
    frac[1::4096] = (1 << 23) - 1
    sign = rng.integers(0, 2, e.size, dtype=np.uint32) << np.uint32(31)
    f = (sign | (e << np.uint32(23)) | frac).view(np.float32)
    f = f[np.isfinite(f)]
    got = f32_to_f64_flushed(f)
    kept = np.abs(f) >= np.float32(2.0 ** -40)
    want = np.where(kept, f.astype(np.float64), np.copysign(0.0, f.astype(np.float64)))
    assert np.array_equal(got.view(np.uint64), want.view(np.uint64))
    assert 0.6 < kept.mean() < 0.7              # exponents 87..254 of 0..254 kept


def test_binary64_to_binary32_rounds_to_nearest_even():
    rng = np.random.default_rng(2)
    n = 1 << 20
    # random binary64 values whose binary32 rounding stays normal
    e = rng.integers(1023 - 126, 1023 + 128, n).astype(np.uint64)
    frac = rng.integers(0, 1 << 52, n, dtype=np.uint64)
    sign = rng.integers(0, 2, n).astype(np.uint64) << np.uint64(63)
    d = (sign | (e << np.uint64(52)) | frac).view(np.float64)
    # ties and near-ties on the 29 dropped bits, and all-ones fractions (carry
    # into the exponent)
    base = d[: n // 4].view(np.uint64) & ~np.uint64((1 << 29) - 1)
    ties = [base | np.uint64(1 << 28), base | np.uint64((1 << 28) - 1), base | np.uint64((1 << 28) + 1)]
    carry = (d[: n // 8].view(np.uint64) | np.uint64((1 << 52) - 1))
    d = np.concatenate([d] + [t.view(np.float64) for t in ties] + [carry.view(np.float64),
                                                                   np.array([0.0, -0.0])])
    with np.errstate(over="ignore"):
        want = d.astype(np.float32)
    ok = np.isfinite(want) & ((np.abs(want) >= np.float32(2.0 ** -126)) | (d == 0))
    got = f64_to_f32_regular(d[ok])
    assert np.array_equal(got.view(np.uint32), want[ok].view(np.uint32))
    assert ok.mean() > 0.95


def test_round_trip_of_binary32_numbers_in_range():
    rng = np.random.default_rng(3)
    bits = rng.integers(0x2B800000, 0x7F800000, 1 << 20, dtype=np.uint32)
    bits |= rng.integers(0, 2, bits.size, dtype=np.uint32) << np.uint32(31)
    f = bits.view(np.float32)
    assert np.array_equal(f64_to_f32_regular(f32_to_f64_flushed(f)).view(np.uint32), bits)


def test_a_truncating_rounding_would_be_caught():
    # the plausible mistake: dropping the rounding step (truncation) differs
    # from round-to-nearest on about half of random inputs
    rng = np.random.default_rng(4)
    d = rng.uniform(1.0, 2.0, 4096)
    b = d.view(np.uint64)
    hi, lo = b >> np.uint64(32), b & M32
    trunc = ((((hi << np.uint64(3)) | (lo >> np.uint64(29))) + np.uint64(0x40000000)) & M32)
    trunc = trunc.astype(np.uint32).view(np.float32)
    assert np.mean(trunc != d.astype(np.float32)) > 0.3
    assert np.array_equal(f64_to_f32_regular(d), d.astype(np.float32))
