"""The tensor-core multi-RHS product (tcgen05, 3 x TF32 with FP32 accumulation)
against the CUDA-core product of the same complex64 operator, through the C ABI.

With the policy forced to 9 (sldm_set_tc_policy), 9 to 32 right-hand sides per
pass go to the tensor cores (by default the crossover is measured per operator,
checked last): every block as a
real FP32 GEMM (complex64 storage read as interleaved FP32), 128-row tiles,
K chunks of 32 FP32 columns, ragged rows and columns zero-filled by TMA, long
tiles split into two K halves that add into Y atomically.  The split into
round-to-nearest TF32 high and low parts keeps near-FP32 accuracy: each product
term carries at most 3 x 2^-22 of |a||x| (the dropped lo x lo term and the
roundings of lo), so the two products differ by 4e-6 relative per column at
most, and against the FP64 product of the same stored blocks the tensor-core
result is as accurate as the CUDA-core one (within 2x); a structural mistake (a
missing split term, a wrong swizzle or sign, a K half added twice or not at
all) gives 1e-3 or more.  The split halves add into zero, which commutes, so a
product repeated on the same inputs is bit-identical.  FP64
operators take 8 right-hand sides per CUDA-core launch and must agree with
single products to 1e-13.
"""
import copy

import numpy as np
import pytest

from oracle import system as S
from oracle.topology import Mesh as OMesh
from workloads.meshes import cylinder_array, ellipsoid, icosphere, merge

pytestmark = pytest.mark.gpu


def _sl():
    import torch  # noqa: F401
    from paper_2106_06184_gb300 import sldm
    return sldm


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


CASES = {
    "sphere": lambda: (*icosphere(2, 0.1), None, [(4.0, 1.0, 0.0)], 300e6),
    "two_lossy": lambda: (*merge(ellipsoid(1, (0.06, 0.04, 0.05), (0, 0, 0)), icosphere(1, 0.05, (0.15, 0.02, 0.0))),
                          [(6.0, 1.0, 0.05), (2.5, 1.0, 0.0)], 500e6),
    "cyl4": lambda: (*cylinder_array(2, 2, 120e-9, 300e-9, 500e-9), [(6.0, 1.0, 0.0)] * 4, 299792458.0 / 1e-6),
}


def _op(sl, name, prec, tc_from=9):
    xyz, tri, obj, mats, f = CASES[name]()
    m = sl.Mesh(xyz, tri, obj)
    st = sl.Stack([(1.0, 1.0, 0.0, 0.0)])
    sl.set_tc_policy(tc_from)
    try:
        return sl.Operator(m, st, mats, f, precision=prec)
    finally:
        sl.set_tc_policy(0)


@pytest.mark.parametrize("name", ["sphere", "two_lossy", "cyl4"])
@pytest.mark.parametrize("nrhs", [9, 16, 31, 32])
def test_tensor_core_product_matches_cuda_core(name, nrhs):
    sl = _sl()
    op = _op(sl, name, 1)
    rng = np.random.default_rng(1000 + nrhs)
    X = np.ascontiguousarray(rng.standard_normal((nrhs, op.N)) + 1j * rng.standard_normal((nrhs, op.N)))
    Y = np.zeros_like(X)
    sl.timers_reset()
    sl.timers_enable(True)
    op.apply(X, Y, nrhs=nrhs)
    sl.timers_enable(False)
    t = sl.timers_read()
    assert t.get("gemm_tc", (0, 0))[1] >= 2, t   # the Y stage and the main stage ran on the tensor cores
    for r in range(nrhs):
        y1 = np.zeros(op.N, complex)
        op.apply(np.ascontiguousarray(X[r]), y1, nrhs=1)
        assert rel(Y[r], y1) < 4e-6, (r, rel(Y[r], y1))


def test_tensor_core_product_is_bit_reproducible():
    sl = _sl()
    op = _op(sl, "cyl4", 1)
    rng = np.random.default_rng(77)
    X = np.ascontiguousarray(rng.standard_normal((32, op.N)) + 1j * rng.standard_normal((32, op.N)))
    Y1 = np.zeros_like(X)
    Y2 = np.zeros_like(X)
    op.apply(X, Y1, nrhs=32)
    for _ in range(3):
        op.apply(X, Y2, nrhs=32)
        assert np.array_equal(Y1, Y2)


def test_tensor_core_product_is_fp32_accurate():
    """Both products of the stored complex64 blocks against their exact (FP64)
    product, formed by the oracle's final_matrix from the copied-out blocks."""
    sl = _sl()
    xyz, tri, obj, mats, f = CASES["sphere"]()
    op = _op(sl, "sphere", 1)
    A = S.assemble(OMesh(xyz, tri, obj), [S.Material(*m) for m in mats], S.Material(), f)
    A32 = copy.copy(A)
    A32.LAm, A32.LPm, A32.Ix = op.block(sl.BLOCK_LAM), op.block(sl.BLOCK_LPM), op.block(sl.BLOCK_IX)
    A32.blocks = [dict(bl, LA=op.block(sl.BLOCK_LA, o), LP=op.block(sl.BLOCK_LP, o), K=op.block(sl.BLOCK_K, o),
                       Y11=op.block(sl.BLOCK_Y11, o), Y21=op.block(sl.BLOCK_Y21, o)) for o, bl in enumerate(A.blocks)]
    Z32 = S.final_matrix(A32)
    rng = np.random.default_rng(5)
    X = np.ascontiguousarray(rng.standard_normal((32, op.N)) + 1j * rng.standard_normal((32, op.N)))
    Y = np.zeros_like(X)
    op.apply(X, Y, nrhs=32)
    ref = (Z32 @ X.T).T
    e_tc = max(rel(Y[r], ref[r]) for r in range(32))
    e_cc = 0.0
    for r in range(32):
        y1 = np.zeros(op.N, complex)
        op.apply(np.ascontiguousarray(X[r]), y1, nrhs=1)
        e_cc = max(e_cc, rel(y1, ref[r]))
    assert e_tc < 2.0 * e_cc + 1e-7, (e_tc, e_cc)


@pytest.mark.parametrize("nrhs", [9, 32])
def test_fp64_passes_of_eight_match_single(nrhs):
    sl = _sl()
    op = _op(sl, "two_lossy", 0)
    rng = np.random.default_rng(7 + nrhs)
    X = np.ascontiguousarray(rng.standard_normal((nrhs, op.N)) + 1j * rng.standard_normal((nrhs, op.N)))
    Y = np.zeros_like(X)
    op.apply(X, Y, nrhs=nrhs)
    for r in range(nrhs):
        y1 = np.zeros(op.N, complex)
        op.apply(np.ascontiguousarray(X[r]), y1, nrhs=1)
        assert rel(Y[r], y1) < 1e-13, (r, rel(Y[r], y1))


@pytest.mark.parametrize("prec", [1, 2])
def test_32_lockstep_solves_match_single_solves(prec):
    """32 plane waves in one lockstep block (tensor-core products in the GMRES
    cycles, FP64-residual refinement) against separate single solves."""
    sl = _sl()
    op = _op(sl, "cyl4", prec)
    th = np.radians(2.5 * np.arange(32))
    khat = np.stack([np.sin(th), 0 * th, -np.cos(th)], axis=1)
    pol = np.stack([np.where(np.arange(32) % 2 == 0, 0.0, np.cos(th)), np.where(np.arange(32) % 2 == 0, 1.0, 0.0),
                    np.where(np.arange(32) % 2 == 0, 0.0, np.sin(th))], axis=1)
    b = np.zeros((32, op.N), complex)
    op.rhs_planewave(khat, pol, b)
    x = np.zeros_like(b)
    sl.timers_reset()
    sl.timers_enable(True)
    info = op.solve(b, x, nrhs=32, tol=1e-10)
    sl.timers_enable(False)
    assert sl.timers_read().get("gemm_tc", (0, 0))[1] > 0
    assert info["relres"] < 1e-10
    for r in (0, 5, 17, 31):
        xr = np.zeros(op.N, complex)
        op.solve(np.ascontiguousarray(b[r]), xr, tol=1e-10)
        assert rel(x[r], xr) < 1e-7, (r, rel(x[r], xr))


@pytest.mark.parametrize("name", ["sphere", "cyl4"])
def test_autotuned_crossover(name):
    """Default policy: the operator records the measured crossover (9, 17 or 33),
    a 16-column product goes to the tensor cores exactly when the crossover says
    so, and agrees with the forced tensor-core product to FP32 accuracy."""
    sl = _sl()
    op = _op(sl, name, 1, tc_from=0)
    assert op.tc_from in (9, 17, 33)
    forced = _op(sl, name, 1, tc_from=9)
    assert forced.tc_from == 9
    rng = np.random.default_rng(5)
    X = np.ascontiguousarray(rng.standard_normal((16, op.N)) + 1j * rng.standard_normal((16, op.N)))
    Y, Yf = np.zeros_like(X), np.zeros_like(X)
    sl.timers_reset()
    sl.timers_enable(True)
    op.apply(X, Y, nrhs=16)
    sl.timers_enable(False)
    ran_tc = sl.timers_read().get("gemm_tc", (0, 0))[1] > 0
    assert ran_tc == (op.tc_from <= 16)
    forced.apply(X, Yf, nrhs=16)
    assert rel(Y, Yf) < 4e-6
