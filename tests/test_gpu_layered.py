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
    # above a stack the far field is taken in the upper half-space only; a wave
    # must come from the upper half-space
    x = np.zeros(op.N, complex)
    with pytest.raises(sl.SldmError):
        op.farfield(x, np.array([np.pi / 2 + 0.1]), np.array([0.0]))
    with pytest.raises(sl.SldmError):
        op.rhs_planewave([1.0, 0, 0], [0, 0, 1.0], np.zeros(op.N, complex))
    # an object crossing an interface is rejected
    v, f = icosphere(1, 0.1, (0.0, 0.0, 0.05))
    mm = sl.Mesh(v, f)
    st2 = sl.Stack([(1.0, 1.0, 0.0, 0.0)], z_top=0.0, bottom=sl.BOTTOM_PEC)
    with pytest.raises(sl.SldmError):
        sl.Operator(mm, st2, [(4.0, 1.0, 0.0, 0)], 300e6)


# ---------------------------------------------------------------- objects resting on an interface
LAM_OPT = 1e-6
F_OPT = 299792458.0 / LAM_OPT
GLASS = [(1.0, 1.0, 0.0, np.inf), (2.25, 1.0, 0.0, np.inf)]


@pytest.fixture(scope="module")
def on_glass():
    """One cylinder (r = 120 nm, h = 300 nm, eps 6) resting on a glass half-space at 1 um."""
    from workloads.meshes import cylinder
    v, f = cylinder(120e-9, 300e-9)
    return LCase(v, f, [(6.0, 1.0, 0.0)], GLASS, 0.0, "halfspace", 0, F_OPT)


@pytest.fixture(scope="module")
def array_on_glass():
    """2 x 2 such cylinders at a 500 nm period: the oracle's L^A_m, L^phi_m only
    (homogeneous fill + reflected part), to check the copied repeated blocks."""
    from oracle import fill as OF
    from workloads.meshes import cylinder_array
    v, f, obj = cylinder_array(2, 2, 120e-9, 300e-9, 500e-9)
    c = LCase.__new__(LCase)
    c.xyz, c.tri, c.mats, c.freq, c.obj = v, f, [(6.0, 1.0, 0.0)] * 4, F_OPT, obj
    c.layers, c.z_top, c.bottom, c.layer = GLASS, 0.0, "halfspace", 0
    c.om = OMesh(v, f, obj)
    c.stack = LY.Stack(GLASS, z_top=0.0)
    w = 2 * np.pi * F_OPT
    k0 = w / 299792458.0
    tris = np.arange(c.om.nt)
    LA, LP = OF.fill_L(c.om, k0, tris)
    LAr, LPr = LY.fill_reflected(c.om, c.stack, 0, w, S.default_tables(c.om, c.stack, 0, w), tris)
    c.LAm, c.LPm = LA + LAr, LP + LPr
    return c


def _gpu_case(c, prec=0):
    import torch  # noqa: F401
    from paper_2106_06184_gb300 import sldm
    m = sldm.Mesh(c.xyz, c.tri, getattr(c, "obj", None))
    st = sldm.Stack([(l[0], l[1], l[2], l[3] if np.isfinite(l[3]) else 0.0) for l in c.layers], z_top=c.z_top,
                    bottom=sldm.BOTTOM_HALFSPACE)
    op = sldm.Operator(m, st, [tuple(mm[:3]) + (c.layer,) for mm in c.mats], c.freq, precision=prec)
    return sldm, op


def test_resting_on_glass_blocks_and_oblique_solution(on_glass):
    """A cylinder resting on glass (images of pairs touching through the interface
    integrated apart, static z-rho images, Sommerfeld tail floor): L^A_m, L^phi_m
    against the oracle at the table bound, then 35-degree TM incidence solved."""
    c = on_glass
    sl, op = _gpu_case(c)
    A = c.A
    for name, got, ref in (("LAm", op.block(sl.BLOCK_LAM), A.LAm), ("LPm", op.block(sl.BLOCK_LPM), A.LPm)):
        assert relmax(got, ref) < 3e-9 and rel(got, ref) < 3e-9, (name, relmax(got, ref))
    t = np.radians(35.0)
    khat = np.array([np.sin(t), 0.0, -np.cos(t)])
    pol = np.array([np.cos(t), 0.0, np.sin(t)])
    b = np.zeros(op.N, complex)
    op.rhs_planewave(khat, pol, b)
    ref_b = S.rhs(A, khat=khat, pol=pol)
    assert rel(b, ref_b) < 1e-12
    x = np.zeros(op.N, complex)
    op.solve(b, x, tol=1e-11)
    assert rel(x, S.solve(A, ref_b)) < 1e-8


def test_resting_array_blocks(array_on_glass):
    """2 x 2 resting cylinders: the repeated blocks (filled once per relative
    placement, reflected part included, then copied) against the oracle."""
    c = array_on_glass
    sl, op = _gpu_case(c)
    for name, got, ref in (("LAm", op.block(sl.BLOCK_LAM), c.LAm), ("LPm", op.block(sl.BLOCK_LPM), c.LPm)):
        assert relmax(got, ref) < 3e-9 and rel(got, ref) < 3e-9, (name, relmax(got, ref))


def test_resting_on_glass_complex64_refined(on_glass):
    """The complex64 operator with the FP64-accurate residual (hi + lo) on the
    resting cylinder: currents within 1e-6 of the FP64 oracle."""
    from paper_2106_06184_gb300 import sldm
    c = on_glass
    sl, op = _gpu_case(c, prec=sldm.PREC_F32X2)
    b = S.rhs(c.A, khat=[0, 0, -1.0], pol=[1.0, 0, 0])
    x = np.zeros(op.N, complex)
    op.solve(b.copy(), x, tol=1e-10)
    assert rel(x, S.solve(c.A, b)) < 1e-6


def test_layered_rcs(on_glass, over_pec):
    """The far field above the stack against the oracle's (reciprocity with the
    stack's plane waves): the cylinder on glass under 35-degree TM incidence and the
    sphere over PEC, 6 upper-hemisphere directions in two azimuth planes each."""
    from oracle import farfield
    th = np.radians(np.linspace(0.0, 85.0, 6))
    t = np.radians(35.0)
    cases = [(on_glass, [np.sin(t), 0.0, -np.cos(t)], [np.cos(t), 0.0, np.sin(t)]),
             (over_pec, [0.0, 0.0, -1.0], [1.0, 0.0, 0.0])]
    for c, khat, pol in cases:
        op = _gpu_case(c)[1] if c is on_glass else c.gpu(0)[3]
        b = np.zeros(op.N, complex)
        op.rhs_planewave(khat, pol, b)
        x = np.zeros(op.N, complex)
        op.solve(b, x, tol=1e-11)
        xr = S.solve(c.A, S.rhs(c.A, khat=khat, pol=pol))
        for ph in (0.0, 1.0):
            got = op.farfield(x, th, np.full_like(th, ph))
            ref = farfield.rcs_layered(c.om, c.stack, c.layer, 2 * np.pi * c.freq, S.j_delta(c.A, xr), th, phi=ph)
            assert np.max(np.abs(got - ref)) <= 1e-7 * np.max(ref), (ph, got, ref)
