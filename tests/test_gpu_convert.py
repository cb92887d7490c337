"""The integer-pipe conversions inlined by the mixed form's kernels
(double <-> float, int64 * 2^e -> double, double * 2^e) against the hardware
conversions, on about a million crafted bit patterns each: round-to-nearest
ties in both parities, carries into the exponent, the smallest-normal
boundary, subnormals, overflow, signed zeros, infinities and NaNs.  The only
differences allowed are the ones the header documents (magnitudes below
2^-126 give a signed zero in the double -> float conversion)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def omm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    from paper_2209_05934_gb300 import omm as _omm
    _omm.lib()
    return _omm


def _doubles_from_bits(bits):
    return np.asarray(bits, dtype=np.uint64).view(np.float64)


def _d2f_inputs(rng):
    parts = []
    n = 200_000
    # random doubles with exponents across and beyond the float range
    e = rng.integers(1023 - 160, 1023 + 140, n).astype(np.uint64)
    m = rng.integers(0, 1 << 52, n, dtype=np.uint64)
    s = rng.integers(0, 2, n).astype(np.uint64)
    parts.append((s << np.uint64(63)) | (e << np.uint64(52)) | m)
    # exact ties (the 29 dropped bits = 1 followed by zeros), both parities of the kept bits
    e = rng.integers(1023 - 126, 1023 + 128, n).astype(np.uint64)
    keep = rng.integers(0, 1 << 23, n, dtype=np.uint64)
    parts.append((e << np.uint64(52)) | (keep << np.uint64(29)) | np.uint64(1 << 28))
    # one below and one above the tie
    parts.append((e << np.uint64(52)) | (keep << np.uint64(29)) | np.uint64((1 << 28) - 1))
    parts.append((e << np.uint64(52)) | (keep << np.uint64(29)) | np.uint64((1 << 28) + 1))
    # carries into the exponent: all 23 kept bits set, at and above the tie
    e2 = rng.integers(1023 - 126, 1023 + 128, 50_000).astype(np.uint64)
    low = rng.integers(1 << 28, 1 << 29, 50_000, dtype=np.uint64)
    parts.append((e2 << np.uint64(52)) | (np.uint64((1 << 23) - 1) << np.uint64(29)) | low)
    # around the smallest normal float 2^-126 and into the subnormal range
    x = np.ldexp(rng.uniform(0.25, 2.0, 100_000), -126) * rng.choice([-1.0, 1.0], 100_000)
    parts.append(x.view(np.uint64))
    # around the largest float and overflow
    x = np.float64(np.finfo(np.float32).max) * rng.uniform(0.999, 1.001, 50_000)
    parts.append(x.view(np.uint64))
    special = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, 1e300, -1e300, 1e-300, -1e-300,
                        2.0 ** -126, -(2.0 ** -126), 2.0 ** -149, 2.0 ** 128, 3.4028235677973366e38])
    parts.append(special.view(np.uint64))
    return _doubles_from_bits(np.concatenate(parts))


def test_double_to_float(omm):
    rng = np.random.default_rng(0)
    x = torch.from_numpy(_d2f_inputs(rng)).cuda()
    out = torch.empty(x.numel(), dtype=torch.float32, device="cuda")
    assert omm.op_convert(0, x, out) == omm.OK
    hw = x.float()
    torch.cuda.synchronize()
    got, ref, xs = out.cpu().numpy(), hw.cpu().numpy(), x.cpu().numpy()
    small = np.abs(xs) < 2.0 ** -126
    nan = np.isnan(xs)
    # documented: below 2^-126 a signed zero
    assert np.all(got[small] == 0.0) and np.all(np.signbit(got[small]) == np.signbit(xs[small]))
    assert np.all(np.isnan(got[nan]))
    rest = ~small & ~nan
    np.testing.assert_array_equal(got[rest].view(np.uint32), ref[rest].view(np.uint32))
    assert rest.sum() > 900_000


def test_float_to_double(omm):
    rng = np.random.default_rng(1)
    bits = np.concatenate([rng.integers(0, 1 << 32, 1_000_000, dtype=np.uint64).astype(np.uint32),
                           np.arange(0, 1 << 16, dtype=np.uint32),                 # small subnormals
                           (1 << 23) - np.arange(1, 1 << 12, dtype=np.uint32),     # largest subnormals
                           np.array([0x80000001, 0x807FFFFF, 0x7F800000, 0xFF800000, 0x7FC00000,
                                     0x00800000, 0x7F7FFFFF], dtype=np.uint32)])
    x = torch.from_numpy(bits.view(np.float32)).cuda()
    out = torch.empty(x.numel(), dtype=torch.float64, device="cuda")
    assert omm.op_convert(1, x, out) == omm.OK
    hw = x.double()
    torch.cuda.synchronize()
    got, ref = out.cpu().numpy(), hw.cpu().numpy()
    nan = np.isnan(ref)
    assert np.all(np.isnan(got[nan]))
    np.testing.assert_array_equal(got[~nan].view(np.uint64), ref[~nan].view(np.uint64))


def test_int64_scaled_to_double(omm):
    rng = np.random.default_rng(2)
    n = 400_000
    mags = rng.integers(1, 63, n)
    v = (rng.integers(0, 1 << 62, n, dtype=np.int64) >> (62 - mags)).astype(np.int64)
    v[v == 0] = 1
    # exact ties: 2^53 + 1 style values at several magnitudes (one dropped bit = half)
    sh = rng.integers(1, 9, 100_000)
    tie = ((rng.integers(1 << 52, 1 << 53, 100_000, dtype=np.int64) << sh) | (np.int64(1) << (sh - 1)))
    # carries: 2^53 - 1 shifted, with the dropped bits at or above half
    carry = (((np.int64(1) << 53) - 1) << 5) | rng.integers(16, 32, 50_000, dtype=np.int64)
    vals = np.concatenate([v, tie, carry, np.array([1, -1, 2 ** 62, -(2 ** 62), 2 ** 63 - 1, -(2 ** 63) + 1])])
    vals = vals * rng.choice([-1, 1], vals.size)
    e = rng.integers(-900, 900, vals.size).astype(np.int32)
    tv, te = torch.from_numpy(vals).cuda(), torch.from_numpy(e).cuda()
    out = torch.empty(vals.size, dtype=torch.float64, device="cuda")
    assert omm.op_convert(2, tv, out, e=te) == omm.OK
    # host reference: one rounding (int64 -> double, round to nearest even), then an exact
    # ldexp (the results stay normal)
    ref = np.ldexp(vals.astype(np.float64), e)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(out.cpu().numpy().view(np.uint64), ref.view(np.uint64))


def test_scale_by_power_of_two(omm):
    rng = np.random.default_rng(3)
    n = 1_000_000
    x = rng.standard_normal(n) * np.ldexp(1.0, rng.integers(-1070, 1000, n))
    x[:1000] = 0.0
    x[1000:2000] = np.ldexp(rng.uniform(1, 2, 1000), -1074 + rng.integers(0, 50, 1000))   # subnormal
    x[2000:2010] = [np.inf, -np.inf, np.nan, -0.0, 1e308, -1e308, 5e-324, 2.2250738585072014e-308, 1.0, -1.0]
    e = rng.integers(-80, 80, n).astype(np.int32)
    tx, te = torch.from_numpy(x).cuda(), torch.from_numpy(e).cuda()
    out = torch.empty(n, dtype=torch.float64, device="cuda")
    assert omm.op_convert(3, tx, out, e=te) == omm.OK
    r = np.ldexp(x, e)                              # host reference, correctly rounded
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    nan = np.isnan(r)
    assert np.all(np.isnan(got[nan]))
    np.testing.assert_array_equal(got[~nan].view(np.uint64), r[~nan].view(np.uint64))
