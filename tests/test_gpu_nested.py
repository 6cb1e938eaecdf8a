"""Y E by inner solves for large objects (Sec. III: direct factorisation only
below ~1000 triangles): an FP32 approximate inverse of M_l with FP64 iterative
refinement to 1e-13 inside every product, in place of the formed Y11, Y21.

* the 512-triangle box (M_l of order 1,279) with the inner-solve threshold
  lowered to 1,000: Y is not formed (op_block says so), the structured product
  equals the direct path's to 1e-12, the solution matches the oracle to 1e-8;
* two copies of the box (the second reuses the first's M_l and inverse): the
  product equals the direct path's;
* the full copper wire (M_l of order 5,119, inner solves by default) at 1 MHz
  and 50 GHz: the solution equals the direct path's to the solve tolerance.
"""
import numpy as np
import pytest

from oracle import system as S
from oracle.topology import Mesh as OMesh
from workloads.meshes import box, copper_wire, merge

pytestmark = pytest.mark.gpu


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.fixture(scope="module")
def box512():
    xyz, tri = box(0.2, 0.15, 0.1, 8, 8, 4, jitter=0.05, seed=11)
    om = OMesh(xyz, tri)
    A = S.assemble(om, [S.Material(4.0, 1.0, 0.01)], S.Material(), 300e6)
    b = S.rhs(A)
    return xyz, tri, S.solve(A, b)


def _ops(xyz, tri, mats, stack_layers=((1.0, 1.0, 0.0, 0.0),), freq=300e6, obj=None, **kw):
    import torch  # noqa: F401
    from paper_2106_06184_gb300 import sldm
    m = sldm.Mesh(xyz, tri, obj)
    st = sldm.Stack(list(stack_layers), **kw)
    inner = sldm.Operator(m, st, mats, freq, precision=0, nested_min=1000)
    direct = sldm.Operator(m, st, mats, freq, precision=0, nested_min=-1)
    return sldm, m, st, inner, direct


def _apply_match(op1, op2, nr=3, seed=0):
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((nr, op1.N)) + 1j * rng.standard_normal((nr, op1.N))
    y1, y2 = np.zeros_like(x), np.zeros_like(x)
    op1.apply(x, y1, nrhs=nr)
    op2.apply(x, y2, nrhs=nr)
    return rel(y1, y2)


def test_inner_solves_box(box512):
    xyz, tri, x_ref = box512
    sl, m, st, inner, direct = _ops(xyz, tri, [(4.0, 1.0, 0.01)])
    with pytest.raises(sl.SldmError) as e:
        inner.block(sl.BLOCK_Y11, 0)
    assert e.value.code == sl.ENOTSUP
    assert _apply_match(inner, direct) < 1e-12
    b = np.zeros(inner.N, complex)
    inner.rhs_planewave([0, 0, -1.0], [1.0, 0, 0], b)
    x = np.zeros(inner.N, complex)
    info = inner.solve(b, x, tol=1e-10)
    assert info["relres"] < 1e-10
    assert rel(x, x_ref) < 1e-8, rel(x, x_ref)


def test_inner_solves_repeated_objects():
    v, f = box(0.2, 0.15, 0.1, 8, 8, 4, jitter=0.05, seed=11)
    v2 = v + np.array([0.5, 0.0, 0.0])
    xyz, tri, obj = merge((v, f), (v2, f))
    sl, m, st, inner, direct = _ops(xyz, tri, [(4.0, 1.0, 0.01)] * 2, obj=obj)
    assert _apply_match(inner, direct, nr=2, seed=1) < 1e-12


@pytest.mark.parametrize("freq", [1e6, 50e9], ids=["1MHz", "50GHz"])
def test_inner_solves_full_wire(freq):
    import torch  # noqa: F401
    from paper_2106_06184_gb300 import sldm
    xyz, tri = copper_wire()
    m = sldm.Mesh(xyz, tri)
    st = sldm.Stack([(1.0, 1.0, 0.0, 0.0), (3.9, 1.0, 0.0, 10e-6), (11.9, 1.0, 10.0, 200e-6)], z_top=0.0,
                    bottom=sldm.BOTTOM_PEC)
    mats = [(1.0, 1.0, 5.8e7, 1)]
    xs = []
    for nmin in (0, -1):  # default (inner solves for this object) and the formed Y
        op = sldm.Operator(m, st, mats, freq, precision=0, nested_min=nmin)
        b = np.zeros(op.N, complex)
        op.rhs_planewave([0, 0, -1.0], [1.0, 0, 0], b)
        x = np.zeros(op.N, complex)
        info = op.solve(b, x, tol=1e-10, maxit=6000)
        assert info["relres"] < 1e-10
        xs.append(x)
        if nmin == 0:
            with pytest.raises(sldm.SldmError):
                op.block(sldm.BLOCK_Y11, 0)
        del op
    assert rel(xs[0], xs[1]) < 1e-7, rel(xs[0], xs[1])
