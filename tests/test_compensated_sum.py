"""The arithmetic of the refinement residual's compensated FP32 product, restated
in numpy float32 (round-to-nearest, one rounding per operation), against an
exact FP64 sum: complex64 matrix entries times complex128 vectors split into
complex64 hi + lo, the two main products of each component split exactly
(product + FMA residual), TwoSum into one FP32 sum and every error and low
product into a second.  The pair must carry ~48 bits (1e-12 of sum |a x| over a
few thousand terms spanning 7 decades), where a plain FP32 sum carries ~24.

This checks the method the kernel follows, not the kernel (the GPU parity tests
check the refined solves against the oracle)."""
import numpy as np

f32 = np.float32


def _fma(a, b, c):
    # a*b of two float32 values is exact in float64; one rounding to float32
    return f32(np.float64(a) * np.float64(b) + np.float64(c))


def _two_sum_into(s, c, p):
    t = f32(s + p)
    bp = f32(t - s)
    e = f32(f32(s - f32(t - bp)) + f32(p - bp))
    return t, f32(c + e)


def _comp_mac(s, c, a1, b1, a2, b2, b1lo, b2lo):
    p1, p2 = f32(a1 * b1), f32(a2 * b2)
    e1, e2 = _fma(a1, b1, -p1), _fma(a2, b2, -p2)
    s, c = _two_sum_into(s, c, p1)
    s, c = _two_sum_into(s, c, p2)
    c = f32(c + f32(e1 + e2))
    c = _fma(a1, b1lo, c)
    return s, _fma(a2, b2lo, c)


def _compensated_dot(A, x):
    sr = cr = si = ci = f32(0)
    for a, v in zip(A, x):
        ar, ai = f32(a.real), f32(a.imag)
        hr, hi = f32(v.real), f32(v.imag)
        lr, li = f32(v.real - np.float64(hr)), f32(v.imag - np.float64(hi))
        sr, cr = _comp_mac(sr, cr, ar, hr, -ai, hi, lr, li)
        si, ci = _comp_mac(si, ci, ar, hi, ai, hr, li, lr)
    return complex(np.float64(sr) + np.float64(cr), np.float64(si) + np.float64(ci))


def test_compensated_fp32_dot_carries_48_bits():
    rng = np.random.default_rng(2106)
    n = 2000
    scale = np.exp(rng.uniform(-8, 8, n))
    A = ((rng.standard_normal(n) + 1j * rng.standard_normal(n)) * scale).astype(np.complex64)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    exact = np.sum(A.astype(np.complex128) * x)
    mag = np.sum(np.abs(A.astype(np.complex128) * x))
    got = _compensated_dot(A, x)
    assert abs(got - exact) < 1e-12 * mag, abs(got - exact) / mag
    # a plain FP32 running sum of the same products is ~1e4 times further off
    plain = np.complex64(0)
    for a, v in zip(A, x.astype(np.complex64)):
        plain = np.complex64(plain + np.complex64(a * v))
    assert abs(complex(plain) - exact) > 1e3 * abs(got - exact)


def test_split_of_complex128_entry_is_exact_to_2_pow_48():
    rng = np.random.default_rng(7)
    v = rng.standard_normal(1000) * np.exp(rng.uniform(-20, 20, 1000))
    hi = v.astype(np.float32)
    lo = (v - hi.astype(np.float64)).astype(np.float32)
    err = np.abs(v - (hi.astype(np.float64) + lo.astype(np.float64)))
    assert np.all(err <= 2.0 ** -48 * np.abs(v))
