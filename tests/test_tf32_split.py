"""The arithmetic of the tensor-core product's 3 x TF32 split, restated in numpy
and checked against exact FP64 results.

TF32 keeps 10 stored mantissa bits.  Rounding an FP32 value v to nearest TF32
(ties away from zero) on its bit pattern -- add half of the dropped unit, 0x1000,
letting the carry run into the exponent, then clear the 13 low bits -- gives hi
with |v - hi| <= 2^-11 |v|; lo = tf32(v - hi) leaves |v - hi - lo| <= 2^-22 |v|.
With D = hi(a) hi(b) + lo(a) hi(b) + hi(a) lo(b), the dropped lo(a) lo(b) and the
roundings of lo keep each product term within 3 x 2^-22 |a||b|, where one TF32
product alone is off by up to ~2^-10.  The tolerances of the GPU tensor-core
tests (4e-6 relative per column against the CUDA-core product) rest on this
bound.

This checks the method the kernel follows, not the kernel (the GPU tests compare
the kernel with the CUDA-core product and the oracle)."""
import numpy as np

f32 = np.float32


def tf32_rn(v):
    """Round float32 values to TF32 on the bit pattern (finite inputs below ~3.4e38)."""
    u = np.asarray(v, f32).view(np.uint32)
    return ((u + np.uint32(0x1000)) & np.uint32(0xFFFFE000)).view(f32)


def tf32_split(v):
    v = np.asarray(v, f32)
    hi = tf32_rn(v)
    lo = tf32_rn((v - hi).astype(f32))
    return hi, lo


def _rn_reference(v):
    """Round to 11 significant bits (10 stored), ties away from zero, in float64 arithmetic."""
    v = np.asarray(v, np.float64)
    m, e = np.frexp(np.abs(v))          # |v| = m 2^e, m in [0.5, 1)
    q = np.floor(m * 2048.0 + 0.5)      # 11 significant bits
    return np.sign(v) * np.ldexp(q, e - 11)


def _samples(n, seed):
    rng = np.random.default_rng(seed)
    v = rng.standard_normal(n) * np.exp(rng.uniform(-30, 30, n))
    return v.astype(f32)


def test_tf32_rounding_is_round_to_nearest():
    v = _samples(200_000, 1)
    hi = tf32_rn(v)
    assert np.all((hi.view(np.uint32) & np.uint32(0x1FFF)) == 0)        # a TF32 value
    assert np.array_equal(hi.astype(np.float64), _rn_reference(v))      # nearest, ties away from zero
    err = np.abs(v.astype(np.float64) - hi.astype(np.float64))
    assert np.all(err <= 2.0 ** -11 * np.abs(v.astype(np.float64)))


def test_tf32_rounding_edge_cases():
    # the carry of a full mantissa runs into the exponent: just below 2 rounds to 2
    assert tf32_rn(f32(np.nextafter(f32(2.0), f32(0.0)))) == f32(2.0)
    # an exact tie (half of the dropped unit) rounds away from zero
    one_half_ulp = f32(1.0 + 2.0 ** -11)
    assert tf32_rn(one_half_ulp) == f32(1.0 + 2.0 ** -10)
    assert tf32_rn(-one_half_ulp) == f32(-(1.0 + 2.0 ** -10))
    # TF32 values and zero are fixed points
    for x in (0.0, -0.0, 1.0, -3.5, 2.0 ** -100, 1.0 + 2.0 ** -10):
        assert tf32_rn(f32(x)) == f32(x)


def test_split_reconstructs_to_22_bits():
    v = _samples(200_000, 2)
    hi, lo = tf32_split(v)
    assert np.all((lo.view(np.uint32) & np.uint32(0x1FFF)) == 0)
    vd = v.astype(np.float64)
    assert np.all(np.abs(vd - hi.astype(np.float64) - lo.astype(np.float64)) <= 2.0 ** -22 * np.abs(vd))


def test_three_products_keep_each_term_within_3_ulp22():
    a, b = _samples(100_000, 3), _samples(100_000, 4)
    ah, al = tf32_split(a)
    bh, bl = tf32_split(b)
    d = lambda x: x.astype(np.float64)  # noqa: E731  products of TF32 values are exact in FP64
    three = d(ah) * d(bh) + d(al) * d(bh) + d(ah) * d(bl)
    exact = d(a) * d(b)
    mag = np.abs(exact)
    assert np.all(np.abs(three - exact) <= 3 * 2.0 ** -22 * mag)
    # one TF32 product (up to ~2^-10 off) or the split with a term left out (~2^-11) fails the bound
    one = d(ah) * d(bh)
    missing = d(ah) * d(bh) + d(ah) * d(bl)
    for wrong in (one, missing):
        assert np.max(np.abs(wrong - exact) / mag) > 100 * 3 * 2.0 ** -22


def test_complex_product_as_real_gemm_with_split():
    """A complex64 block read as interleaved FP32 (2n columns) times a real B'
    holding +re, -im / +im, +re of each vector gives Re and Im of y = A x in two
    columns; with the 3 x TF32 split every output stays within 3 x 2^-22 of
    sum |a||x| (FP64 accumulation here isolates the products' error)."""
    rng = np.random.default_rng(5)
    m, n, nrhs = 64, 300, 4
    A = (rng.standard_normal((m, n)) + 1j * rng.standard_normal((m, n))).astype(np.complex64)
    X = (rng.standard_normal((n, nrhs)) + 1j * rng.standard_normal((n, nrhs))).astype(np.complex64)
    Ar = A.view(f32)                                   # m x 2n: re, im interleaved
    Bp = np.zeros((2 * n, 2 * nrhs), f32)
    Bp[0::2, 0::2], Bp[1::2, 0::2] = X.real, -X.imag   # Re y = re a re x - im a im x
    Bp[0::2, 1::2], Bp[1::2, 1::2] = X.imag, X.real    # Im y = re a im x + im a re x
    ah, al = tf32_split(Ar)
    bh, bl = tf32_split(Bp)
    d = lambda x: x.astype(np.float64)  # noqa: E731
    D = d(ah) @ d(bh) + d(al) @ d(bh) + d(ah) @ d(bl)
    Y = D[:, 0::2] + 1j * D[:, 1::2]
    exact = A.astype(np.complex128) @ X.astype(np.complex128)
    mag = np.abs(d(Ar)) @ np.abs(d(Bp))
    assert np.all(np.abs(Y.real - exact.real) <= 3 * 2.0 ** -22 * mag[:, 0::2])
    assert np.all(np.abs(Y.imag - exact.imag) <= 3 * 2.0 ** -22 * mag[:, 1::2])
    # relative to the column norms: FP32 level, far below one TF32 product's error
    rel = np.linalg.norm(Y - exact, axis=0) / np.linalg.norm(exact, axis=0)
    assert np.all(rel < 4e-6), rel
    one = (d(ah) @ d(bh))
    rel1 = np.linalg.norm(one[:, 0::2] + 1j * one[:, 1::2] - exact, axis=0) / np.linalg.norm(exact, axis=0)
    assert np.all(rel1 > 30 * rel)
