"""Parity of the blocked LU (objects whose M_l has order 1024 or more) with the
oracle's dense solve: Y11, Y21 = M_l^-1 [Kbar_l + I_x/2; 0] and the solution of
the final system, on a dielectric box of 512 triangles (M_l of order 1,279,
20 panels of 64 columns with a ragged last panel).

Tolerances: Y11, Y21 1e-9 relative to the block's largest entry (M_l's
conditioning times FP64 rounding); solution 1e-8 (GMRES to 1e-10), as for the
unblocked path.  In complex64 the solution is held to 5e-4, as the FP32 path
of the other parity tests.
"""
import numpy as np
import pytest

from oracle import system as S
from oracle.topology import Mesh as OMesh
from workloads.meshes import box

pytestmark = pytest.mark.gpu


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def relmax(a, b):
    return np.max(np.abs(a - b)) / np.max(np.abs(b))


@pytest.fixture(scope="module")
def box512():
    xyz, tri = box(0.2, 0.15, 0.1, 8, 8, 4, jitter=0.05, seed=11)
    om = OMesh(xyz, tri)
    assert om.ne + om.nt - 1 >= 1024
    A = S.assemble(om, [S.Material(4.0, 1.0, 0.01)], S.Material(), 300e6)
    b = S.rhs(A)
    return xyz, tri, om, A, b, S.solve(A, b)


def _op(xyz, tri, prec):
    import torch  # noqa: F401
    from paper_2106_06184_gb300 import sldm
    m = sldm.Mesh(xyz, tri)
    return sldm, m, sldm.Operator(m, sldm.Stack([(1.0, 1.0, 0.0, 0.0)]), [(4.0, 1.0, 0.01)], 300e6, precision=prec)


def test_blocked_lu_blocks_and_solution(box512):
    xyz, tri, om, A, b_ref, x_ref = box512
    sl, m, op = _op(xyz, tri, 0)
    blk = A.blocks[0]
    for name, got, ref in (("Y11", op.block(sl.BLOCK_Y11, 0), blk["Y11"]), ("Y21", op.block(sl.BLOCK_Y21, 0), blk["Y21"])):
        assert relmax(got, ref) < 1e-9, (name, relmax(got, ref))
    b = np.zeros(op.N, complex)
    op.rhs_planewave([0, 0, -1.0], [1.0, 0, 0], b)
    x = np.zeros(op.N, complex)
    info = op.solve(b, x, tol=1e-10)
    assert info["relres"] < 1e-10
    assert rel(x, x_ref) < 1e-8, rel(x, x_ref)


def test_blocked_lu_complex64(box512):
    xyz, tri, om, A, b_ref, x_ref = box512
    sl, m, op = _op(xyz, tri, 1)
    b = np.zeros(op.N, complex)
    op.rhs_planewave([0, 0, -1.0], [1.0, 0, 0], b)
    x = np.zeros(op.N, complex)
    info = op.solve(b, x, tol=1e-5)
    assert info["relres"] < 1e-5
    assert rel(x, x_ref) < 5e-4, rel(x, x_ref)
