"""Failure paths of the library on the GPU, made without faulting the GPU.

* A bounded device wait that runs out: the batched direct solver's first CTA is
  made to wait on a flag that nothing sets (sldm_test_inject); the wait gives up
  after its iteration limit, every CTA leaves, sldm_assemble returns
  SLDM_ETIMEOUT, and the context stays usable (the next assembly is correct).
* The device-memory budget: an assembly that would exceed it returns
  SLDM_ENOMEM and releases what it took.
* GMRES that cannot reach the tolerance within maxit returns SLDM_ENOTCONV.
* Two identical runs agree to rounding (the fill accumulates the four
  triangle-pair contributions of an edge pair with atomics, so the order of the
  additions may differ between runs).
"""
import numpy as np
import pytest

from workloads.meshes import icosphere

pytestmark = pytest.mark.gpu


def _sl():
    import torch  # noqa: F401
    from paper_2106_06184_gb300 import sldm
    return sldm


def _sphere_op(sl, sub=1, prec=0):
    v, f = icosphere(sub, 0.1)
    m = sl.Mesh(v, f)
    st = sl.Stack([(1.0, 1.0, 0.0, 0.0)])
    return m, st, sl.Operator(m, st, [(4.0, 1.0, 0.0)], 300e6, precision=prec)


def _solve(sl, op, **kw):
    import torch
    b = torch.zeros(op.N, dtype=torch.complex128, device="cuda")
    op.rhs_planewave([0, 0, -1.0], [1.0, 0, 0], b)
    x = torch.zeros_like(b)
    info = op.solve(b, x, **kw)
    return x.cpu().numpy(), info


def test_lu_wait_runs_out_and_context_survives():
    sl = _sl()
    m, st, ref_op = _sphere_op(sl)
    x_ref, _ = _solve(sl, ref_op, tol=1e-10)
    sl.test_inject(sl.INJECT_LU_STALL, 1)
    try:
        with pytest.raises(sl.SldmError) as e:
            sl.Operator(m, st, [(4.0, 1.0, 0.0)], 300e6, precision=sl.PREC_F64)
        assert e.value.code == sl.ETIMEOUT
    finally:
        sl.test_inject(sl.INJECT_LU_STALL, 0)
    op = sl.Operator(m, st, [(4.0, 1.0, 0.0)], 300e6, precision=sl.PREC_F64)
    x, info = _solve(sl, op, tol=1e-10)
    assert np.linalg.norm(x - x_ref) <= 1e-10 * np.linalg.norm(x_ref)  # atomics: summation order only


def test_budget_exceeded_returns_enomem_and_releases():
    sl = _sl()
    v, f = icosphere(2, 0.1)
    m = sl.Mesh(v, f)
    st = sl.Stack([(1.0, 1.0, 0.0, 0.0)])
    held = sl.device_bytes()
    sl.set_device_budget(held + (1 << 20))  # 1 MiB more than the mesh: far below one operator
    try:
        with pytest.raises(sl.SldmError) as e:
            sl.Operator(m, st, [(4.0, 1.0, 0.0)], 300e6, precision=sl.PREC_F64)
        assert e.value.code == sl.ENOMEM and "budget" in str(e.value)
        assert sl.device_bytes() == held
    finally:
        sl.set_device_budget(0)
    op = sl.Operator(m, st, [(4.0, 1.0, 0.0)], 300e6, precision=sl.PREC_F64)
    assert sl.device_bytes() > held
    _, info = _solve(sl, op, tol=1e-8)
    assert info["code"] == sl.OK


def test_gmres_not_converged_is_reported():
    sl = _sl()
    _, _, op = _sphere_op(sl, sub=2)
    _, info = _solve(sl, op, tol=1e-12, maxit=3, check=False)
    assert info["code"] == sl.ENOTCONV and info["status"] == sl.ENOTCONV
    assert info["relres"] > 1e-12 and info["iters"] == 3


@pytest.mark.parametrize("prec", [0, 2])
def test_two_runs_agree(prec):
    """Two identical runs: the operators agree to FP64 rounding (the atomic
    accumulation order of the fill is the only difference) and the solutions
    to the solve tolerance times the conditioning (GMRES stops at 1e-10 of the
    residual, so two nearby operators may stop a few iterations apart)."""
    sl = _sl()
    xs, blocks = [], []
    for _ in range(2):
        _, _, op = _sphere_op(sl, sub=2, prec=prec)
        blocks.append([op.block(w) for w in (sl.BLOCK_LAM, sl.BLOCK_LPM)] + [op.block(sl.BLOCK_Y11, 0)])
        x, info = _solve(sl, op, tol=1e-10)
        xs.append(x)
        assert info["code"] == sl.OK
    for a, b in zip(*blocks):
        assert np.max(np.abs(a - b)) <= 1e-13 * np.max(np.abs(a))
    assert np.linalg.norm(xs[0] - xs[1]) <= 1e-8 * np.linalg.norm(xs[0])
