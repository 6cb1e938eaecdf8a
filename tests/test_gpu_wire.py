"""Parity of the multiscale-conductor configuration with the oracle, through the
C ABI: copper (5.8e7 S/m) in the middle of a 10 um SiO2 layer over 200 um of
lossy Si over a PEC ground, air above, at the ends and the middle of the
1 MHz - 50 GHz sweep.

* A 20 x 2 x 1 um bar (80 triangles) in that stack: every block, Y11 and the
  solution against the oracle's whole system (its sources are split at 50 GHz
  and 300 MHz, and far pairs are cut at 50 GHz).
* The full 100 x 2 x 1 um wire of the bench (2,048 graded triangles), in the
  launch configuration the bench times: sampled entries of the copper L^A,
  L^phi (split sources, cut pairs) and of the layered L^A_m, L^phi_m, each
  computed by the oracle one triangle pair at a time.

Tolerances: FP64 blocks 1e-10; blocks built from the Sommerfeld tables 3e-9 of
the block's largest entry (the tables agree to 1e-9, see test_gpu_layered);
Y11 1e-9; the right-hand side 1e-10 (see the test); the solution through the
length-scaled residual in the oracle's Z (1e-10) and to 1e-6.
"""
import numpy as np
import pytest

from oracle import fill as OFL
from oracle import layered as LY
from oracle import system as S
from oracle.topology import Mesh as OMesh
from workloads.meshes import box, copper_wire

pytestmark = pytest.mark.gpu

LAYERS = [(1.0, 1.0, 0.0, np.inf), (3.9, 1.0, 0.0, 10e-6), (11.9, 1.0, 10.0, 200e-6)]
COPPER = (1.0, 1.0, 5.8e7)
SWEEP = np.logspace(6.0, np.log10(50e9), 20)


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def relmax(a, b):
    return np.max(np.abs(a - b)) / np.max(np.abs(b))


def gpu_op(xyz, tri, freq):
    import torch  # noqa: F401
    from paper_2106_06184_gb300 import sldm
    m = sldm.Mesh(xyz, tri)
    st = sldm.Stack([(l[0], l[1], l[2], l[3] if np.isfinite(l[3]) else 0.0) for l in LAYERS], z_top=0.0,
                    bottom=sldm.BOTTOM_PEC)
    return sldm, m, st, sldm.Operator(m, st, [COPPER + (1,)], freq, precision=0)


class ShortBar:
    def __init__(self, freq):
        self.xyz, self.tri = box(20e-6, 2e-6, 1e-6, 6, 2, 1, center=(0.0, 0.0, -5e-6), jitter=0.01, seed=7)
        self.freq = freq
        self.om = OMesh(self.xyz, self.tri)
        self.stack = LY.Stack(LAYERS, z_top=0.0, bottom="pec")
        self.A = S.assemble(self.om, [S.Material(*COPPER)], self.stack, freq, layer=1)
        self.b = S.rhs(self.A)
        self.x = S.solve(self.A, self.b)


@pytest.fixture(scope="module", params=[0, 10, 19], ids=["1MHz", "297MHz", "50GHz"])
def bar(request):
    return ShortBar(SWEEP[request.param])


def test_short_bar_blocks_and_solution(bar):
    sl, m, st, op = gpu_op(bar.xyz, bar.tri, bar.freq)
    A, blk = bar.A, bar.A.blocks[0]
    for name, got, ref, tol in (("LAm", op.block(sl.BLOCK_LAM), A.LAm, 3e-9), ("LPm", op.block(sl.BLOCK_LPM), A.LPm, 3e-9),
                                ("LA", op.block(sl.BLOCK_LA, 0), blk["LA"], 1e-10),
                                ("LP", op.block(sl.BLOCK_LP, 0), blk["LP"], 1e-10),
                                ("K", op.block(sl.BLOCK_K, 0), blk["K"], 1e-10),
                                ("Y11", op.block(sl.BLOCK_Y11, 0), blk["Y11"], 1e-9)):
        assert relmax(got, ref) < tol, (name, relmax(got, ref))
    b = np.zeros(op.N, complex)
    op.rhs_planewave([0, 0, -1.0], [1.0, 0, 0], b)
    # the field in the SiO2 over grounded Si is a near-cancelling standing wave at low
    # frequency (|a + c| ~ 1e-4 |a|), which amplifies the rounding of the stack's
    # transfer coefficients by that ratio
    assert rel(b, bar.b) < 1e-10
    x = np.zeros(op.N, complex)
    info = op.solve(b, x, tol=1e-11, maxit=4000)
    assert info["relres"] < 1e-11
    om = bar.om
    ell = np.mean(np.linalg.norm(om.xyz[om.E.uv[:, 0]] - om.xyz[om.E.uv[:, 1]], axis=1))
    dr = np.ones(op.N)
    dr[2 * om.ne:] = ell
    assert np.linalg.norm(dr * (A.Z @ x - bar.b)) < 1e-10 * np.linalg.norm(dr * bar.b)
    assert rel(x, bar.x) < 1e-6, rel(x, bar.x)


# ---------------------------------------------------------------- full-size wire, sampled entries
@pytest.fixture(scope="module")
def wire():
    xyz, tri = copper_wire()
    return xyz, tri, OMesh(xyz, tri)


def _L_entry_pairs(om, k, tris_a, tris_b):
    """Oracle local blocks of the given triangle pairs, as oracle.fill.fill_L forms them:
    the source's split rule, and the far-pair cut when any source of the fill is split."""
    P = om.xyz[om.tri]
    split = OFL.needs_split(k, P).any()
    la = np.zeros((len(tris_a), 3, 3), complex)
    lp = np.zeros(len(tris_a), complex)
    keep = np.ones(len(tris_a), bool)
    if split:
        keep = OFL._kept(k, P[tris_a], P[tris_b], OFL._touch_primal(om.tri, tris_a, tris_b))
    for i in np.nonzero(keep)[0]:
        rule = None
        if split:
            pts, w = OFL.source_rule(P[tris_b[i]], k)
            rule = (pts[None], w[None])
        a, b = OFL._L_pairs(om, k, tris_a[i:i + 1], tris_b[i:i + 1], rule)
        la[i], lp[i] = a[0], b[0]
    return la, lp


def _edge_entry(om, la_fn, m, n):
    """Sum of the four triangle-pair contributions to the edge-pair entry (m, n)."""
    tm = [om.E.tp[m], om.E.tm[m]]
    tn = [om.E.tp[n], om.E.tm[n]]
    ta = np.array([a for a in tm for b in tn])
    tb = np.array([b for a in tm for b in tn])
    la = la_fn(ta, tb)
    out = 0.0
    for p in range(4):
        i = int(np.nonzero(om.E.tri_edge[ta[p]] == m)[0][0])
        j = int(np.nonzero(om.E.tri_edge[tb[p]] == n)[0][0])
        out = out + la[p, i, j]
    return out


@pytest.mark.parametrize("fi", [0, 19], ids=["1MHz", "50GHz"])
def test_full_wire_sampled_entries(wire, fi):
    xyz, tri, om = wire
    freq = SWEEP[fi]
    sl, m, st, op = gpu_op(xyz, tri, freq)
    k0 = 2 * np.pi * freq / S.C0
    kc = S.wavenumber(S.Material(*COPPER), k0)
    LA, LP = op.block(sl.BLOCK_LA, 0), op.block(sl.BLOCK_LP, 0)
    rng = np.random.default_rng(fi)
    # edge pairs: half random, half near neighbours (the touching and split-source regime)
    E = rng.integers(0, om.ne, (12, 2))
    nb = rng.integers(0, om.ne, 12)
    E = np.concatenate([E, np.stack([nb, om.E.tri_edge[om.E.tp[nb], rng.integers(0, 3, 12)]], axis=1)])
    for mm, nn in E:
        ref = _edge_entry(om, lambda a, b: _L_entry_pairs(om, kc, a, b)[0], mm, nn)
        assert abs(LA[mm, nn] - ref) <= 1e-10 * np.max(np.abs(LA)), (mm, nn, LA[mm, nn], ref)
    T = rng.integers(0, om.nt, (24, 2))
    T[12:, 1] = T[12:, 0]  # self pairs
    _, lp = _L_entry_pairs(om, kc, T[:, 0], T[:, 1])
    ref = lp / S.eps_c(S.Material(*COPPER), 2 * np.pi * freq)
    got = LP[T[:, 0], T[:, 1]]
    assert np.max(np.abs(got - ref)) <= 1e-10 * np.max(np.abs(LP))
    # layered external blocks: homogeneous SiO2 part + reflected part, one small triangle set at a time
    LAm, LPm = op.block(sl.BLOCK_LAM), op.block(sl.BLOCK_LPM)
    stack = LY.Stack(LAYERS, z_top=0.0, bottom="pec")
    omega = 2 * np.pi * freq
    tables = S.default_tables(om, stack, 1, omega)
    kb = S.wavenumber(S.Material(3.9), k0)
    for mm, nn in E[::3]:
        tris = np.unique([om.E.tp[mm], om.E.tm[mm], om.E.tp[nn], om.E.tm[nn]])
        la_h, lp_h = OFL.fill_L(om, kb, tris)
        la_r, lp_r = LY.fill_reflected(om, stack, 1, omega, tables, tris)
        edges = np.unique(om.E.tri_edge[tris])
        i, j = int(np.searchsorted(edges, mm)), int(np.searchsorted(edges, nn))
        ref = la_h[i, j] + la_r[i, j]
        assert abs(LAm[mm, nn] - ref) <= 3e-9 * np.max(np.abs(LAm)), (mm, nn)
        ti = [int(np.searchsorted(tris, t)) for t in tris]
        for a, ta in zip(ti, tris):
            for b, tb in zip(ti, tris):
                refp = lp_h[a, b] / 3.9 + lp_r[a, b]
                assert abs(LPm[ta, tb] - refp) <= 3e-9 * np.max(np.abs(LPm)), (ta, tb)
