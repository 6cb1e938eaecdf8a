"""Parity of the layered-background path (multilayer kernel of the external
problem) with the oracle: Sommerfeld remainder tables, L^A_m and L^phi_m, the
stack-transferred plane wave and the solution.

Both sides integrate the same Sommerfeld path (elliptic arc + Gauss-Legendre
panels, same node rule) with their own Bessel functions and summation order, so
the tables agree to 1e-9 of their largest entry.  The TM - TE difference of the
scalar-potential kernel cancels as k_rho -> 0, which leaves rounding noise of
about 1e-10 of the kernel in a table that should vanish (PEC ground), so the
blocks built from the tables are compared at 3e-9; everything else matches the
homogeneous path's 1e-10.
"""
import numpy as np
import pytest

from oracle import layered as LY
from oracle import system as S
from oracle.topology import Mesh as OMesh
from workloads.meshes import icosphere

pytestmark = pytest.mark.gpu


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def relmax(a, b):
    return np.max(np.abs(a - b)) / np.max(np.abs(b))


class LCase:
    def __init__(self, xyz, tri, mats, layers, z_top, bottom, layer, freq):
        self.xyz, self.tri, self.mats, self.freq = xyz, tri, mats, freq
        self.layers, self.z_top, self.bottom, self.layer = layers, z_top, bottom, layer
        self.om = OMesh(xyz, tri)
        self.stack = LY.Stack(layers, z_top=z_top, bottom=bottom)
        self.A = S.assemble(self.om, [S.Material(*m[:3]) for m in mats], self.stack, freq, layer=layer)
        self.b = S.rhs(self.A)
        self.x = S.solve(self.A, self.b)

    def gpu(self, prec=0):
        import torch  # noqa: F401
        from paper_2106_06184_gb300 import sldm
        m = sldm.Mesh(self.xyz, self.tri)
        st = sldm.Stack([(l[0], l[1], l[2], l[3] if np.isfinite(l[3]) else 0.0) for l in self.layers], z_top=self.z_top,
                        bottom=sldm.BOTTOM_PEC if self.bottom == "pec" else sldm.BOTTOM_HALFSPACE)
        op = sldm.Operator(m, st, [tuple(mm[:3]) + (self.layer,) for mm in self.mats], self.freq, precision=prec)
        return sldm, m, st, op


@pytest.fixture(scope="module")
def over_pec():
    v, f = icosphere(1, 0.1, (0.0, 0.0, 0.15))
    return LCase(v, f, [(4.0, 1.0, 0.0)], [(1.0, 1.0, 0.0, np.inf)], 0.0, "pec", 0, 300e6)


@pytest.fixture(scope="module")
def in_slab():
    v, f = icosphere(1, 0.08, (0.0, 0.0, -0.2))
    layers = [(1.0, 1.0, 0.0, np.inf), (4.0, 1.0, 0.0, 0.4), (11.9, 1.0, 0.1, np.inf)]
    return LCase(v, f, [(2.5, 1.0, 0.01)], layers, 0.0, "halfspace", 1, 300e6)


@pytest.mark.parametrize("which", ["over_pec", "in_slab"])
def test_layered_blocks_and_solution(which, request):
    c = request.getfixturevalue(which)
    sl, m, st, op = c.gpu(0)
    A = c.A
    for name, got, ref, tol in (("LAm", op.block(sl.BLOCK_LAM), A.LAm, 3e-9), ("LPm", op.block(sl.BLOCK_LPM), A.LPm, 3e-9),
                                ("Y11", op.block(sl.BLOCK_Y11), A.blocks[0]["Y11"], 1e-10),
                                ("K", op.block(sl.BLOCK_K), A.blocks[0]["K"], 1e-10)):
        assert relmax(got, ref) < tol and rel(got, ref) < tol, (name, relmax(got, ref))
    b = np.zeros(op.N, complex)
    op.rhs_planewave([0, 0, -1.0], [1.0, 0, 0], b)
    assert rel(b, c.b) < 1e-12
    x = np.zeros(op.N, complex)
    op.solve(b, x, tol=1e-11)
    assert rel(x, c.x) < 1e-8


@pytest.mark.parametrize("which", ["over_pec", "in_slab"])
def test_layered_oblique_incidence(which, request):
    """Oblique TE, TM and mixed plane waves through the stack (one batched call of
    five right-hand sides, incl. grazing 80 degrees and normal incidence) against
    the oracle's stack-transferred field, then the solution of one of them."""
    c = request.getfixturevalue(which)
    sl, m, st, op = c.gpu(0)
    waves = []
    for th, ph, a_te, a_tm in ((35.0, 20.0, 1.0, 0.0), (35.0, 20.0, 0.0, 1.0), (60.0, -130.0, 0.6, 0.8),
                               (80.0, 45.0, 0.8, -0.6), (0.0, 0.0, 0.0, 1.0)):
        t, p = np.radians(th), np.radians(ph)
        khat = np.array([np.sin(t) * np.cos(p), np.sin(t) * np.sin(p), -np.cos(t)])
        e_te = np.array([-np.sin(p), np.cos(p), 0.0])
        waves.append((khat, a_te * e_te + a_tm * np.cross(e_te, khat)))
    K = np.array([w[0] for w in waves])
    P = np.array([w[1] for w in waves])
    b = np.zeros((len(waves), op.N), complex)
    op.rhs_planewave(K, P, b)
    for r, (khat, pol) in enumerate(waves):
        ref = S.rhs(c.A, khat=khat, pol=pol)
        assert rel(b[r], ref) < 1e-12, (r, rel(b[r], ref))
    x = np.zeros(op.N, complex)
    op.solve(b[2], x, tol=1e-11)
    xr = S.solve(c.A, S.rhs(c.A, khat=waves[2][0], pol=waves[2][1]))
    assert rel(x, xr) < 1e-8


def test_layered_tables_match_oracle(in_slab):
    c = in_slab
    sl, m, st, op = c.gpu(0)
    T = c.A.layered[2]
    ta, ga = op.table(0)
    tb, gb = op.table(1)
    assert np.allclose(ga, [np.log(T.rho[0]), np.log(T.rho[-1]), T.s[0], T.s[-1], T.d[-1]], rtol=1e-13, atol=1e-15)
    for k, comp in enumerate(LY.COMPONENTS):
        scale = max(np.abs(T.A[comp]).max(), 1e-300)
        assert np.abs(ta[k] - T.A[comp]).max() <= 1e-9 * scale, comp
        scale_b = max(np.abs(T.B[comp]).max(), 1e-300)
        assert np.abs(tb[k] - T.B[comp]).max() <= 1e-9 * scale_b, comp


def test_layered_fp32_and_invalid_cases(in_slab, over_pec):
    sl, m, st, op = in_slab.gpu(1)
    assert relmax(op.block(sl.BLOCK_LAM), in_slab.A.LAm) < 1e-5
    # far field is free-space only; a wave must come from the upper half-space
    x = np.zeros(op.N, complex)
    with pytest.raises(sl.SldmError):
        op.farfield(x, np.array([0.1]), np.array([0.0]))
    with pytest.raises(sl.SldmError):
        op.rhs_planewave([1.0, 0, 0], [0, 0, 1.0], np.zeros(op.N, complex))
    # an object crossing an interface is rejected
    v, f = icosphere(1, 0.1, (0.0, 0.0, 0.05))
    mm = sl.Mesh(v, f)
    st2 = sl.Stack([(1.0, 1.0, 0.0, 0.0)], z_top=0.0, bottom=sl.BOTTOM_PEC)
    with pytest.raises(sl.SldmError):
        sl.Operator(mm, st2, [(4.0, 1.0, 0.0, 0)], 300e6)
