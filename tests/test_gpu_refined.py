"""Mixed precision against the FP64 oracle, through the C ABI.

SLDM_PREC_F32X2 keeps an FP64 fill as complex64 pairs (hi + lo): GMRES cycles run
on hi in FP32 arithmetic and iterative refinement takes its residual from
hi + lo with compensated FP32 sums, so the refined currents converge to the
FP64 discrete system's: the stated bound is relative L2 1e-6 against the oracle
(observed: ~1e-9).  Blocks reconstructed from hi + lo match the oracle's FP64
blocks to 1e-10 (the FP64 fill's own parity bound).

SLDM_PREC_F32 (the FP32 bulk fill) is checked entry by entry: every entry of
L^A_m, L^phi_m, L^A, L^phi and K within 1e-5 of its own magnitude, plus an
absolute floor of 4 FP32 units of the block's largest entry (4 x 2^-24 x max)
for entries near the FP32 resolution of the block; and at the full 8 x 8
metasurface on sampled entries computed by the oracle one triangle pair at a
time.
"""
import numpy as np
import pytest

from oracle import farfield as OF
from oracle import fill as OFL
from oracle import system as S
from oracle.topology import Mesh as OMesh
from workloads.meshes import cylinder_array, ellipsoid, icosphere, merge

pytestmark = pytest.mark.gpu

FP32_FLOOR = 4 * 2.0 ** -24


def _sl():
    import torch  # noqa: F401
    from paper_2106_06184_gb300 import sldm
    return sldm


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


class Case:
    def __init__(self, xyz, tri, obj, mats, freq):
        self.xyz, self.tri, self.obj, self.mats, self.freq = xyz, tri, obj, mats, freq
        self.om = OMesh(xyz, tri, obj)
        self.A = S.assemble(self.om, [S.Material(*m[:3]) for m in mats], S.Material(), freq)
        self.b = S.rhs(self.A)
        self.x = S.solve(self.A, self.b)


@pytest.fixture(scope="module")
def sphere():
    v, f = icosphere(2, 0.1)
    return Case(v, f, None, [(4.0, 1.0, 0.0)], 300e6)


@pytest.fixture(scope="module")
def two_lossy():
    xyz, tri, obj = merge(ellipsoid(1, (0.06, 0.04, 0.05), (0, 0, 0)), icosphere(1, 0.05, (0.15, 0.02, 0.0)))
    return Case(xyz, tri, obj, [(6.0, 1.0, 0.05), (2.5, 1.0, 0.0)], 500e6)


@pytest.fixture(scope="module")
def cyl4():
    xyz, tri, obj = cylinder_array(2, 2, 120e-9, 300e-9, 500e-9)
    return Case(xyz, tri, obj, [(6.0, 1.0, 0.0)] * 4, 299792458.0 / 1e-6)


def build(case, prec):
    sl = _sl()
    m = sl.Mesh(case.xyz, case.tri, case.obj)
    st = sl.Stack([(1.0, 1.0, 0.0, 0.0)])
    return sl, sl.Operator(m, st, case.mats, case.freq, precision=prec)


def _blocks(case, op, sl, with_y=True):
    A = case.A
    out = [("LAm", op.block(sl.BLOCK_LAM), A.LAm), ("LPm", op.block(sl.BLOCK_LPM), A.LPm)]
    for o, b in enumerate(A.blocks):
        out += [(f"LA{o}", op.block(sl.BLOCK_LA, o), b["LA"]), (f"LP{o}", op.block(sl.BLOCK_LP, o), b["LP"]),
                (f"K{o}", op.block(sl.BLOCK_K, o), b["K"])]
        if with_y:
            out += [(f"Y11_{o}", op.block(sl.BLOCK_Y11, o), b["Y11"]), (f"Y21_{o}", op.block(sl.BLOCK_Y21, o), b["Y21"])]
    return out


@pytest.mark.parametrize("which", ["sphere", "two_lossy", "cyl4"])
def test_x2_blocks_are_the_fp64_blocks(which, request):
    case = request.getfixturevalue(which)
    sl, op = build(case, 2)
    assert op.precision == sl.PREC_F32X2
    for name, got, ref in _blocks(case, op, sl):
        err = np.max(np.abs(got - ref)) / np.max(np.abs(ref))
        assert rel(got, ref) < 1e-10 and err < 1e-10, (name, rel(got, ref), err)


@pytest.mark.parametrize("which", ["sphere", "two_lossy"])
@pytest.mark.parametrize("nrhs", [1, 3, 8])
def test_x2_apply_is_the_fp64_product(which, nrhs, request):
    case = request.getfixturevalue(which)
    sl, op = build(case, 2)
    rng = np.random.default_rng(11 + nrhs)
    X = np.ascontiguousarray(rng.standard_normal((nrhs, op.N)) + 1j * rng.standard_normal((nrhs, op.N)))
    Y = np.zeros_like(X)
    op.apply(X, Y, nrhs=nrhs)
    assert rel(Y, (case.A.Z @ X.T).T) < 1e-10


@pytest.mark.parametrize("which", ["sphere", "cyl4", "two_lossy"])
def test_x2_refined_currents_within_1e6_of_oracle(which, request):
    case = request.getfixturevalue(which)
    sl, op = build(case, 2)
    b = np.zeros(op.N, complex)
    op.rhs_planewave([0, 0, -1.0], [1.0, 0, 0], b)
    x = np.zeros(op.N, complex)
    info = op.solve(b, x, tol=1e-10)
    assert info["relres"] < 1e-10
    err = rel(x, case.x)
    assert err < 1e-6, err
    th = np.radians(np.arange(0, 181, 15.0))
    got = op.farfield(x, th, np.zeros_like(th))
    ref = OF.rcs(case.om, case.A.k0, S.j_delta(case.A, case.x), th)
    assert np.max(np.abs(10 * np.log10(got / ref))) < 0.05


def test_x2_lockstep_angles_within_1e6_of_oracle(cyl4):
    """Eight plane waves in one lockstep block, each refined to the FP64 system."""
    sl, op = build(cyl4, 2)
    th = np.radians(2.5 * np.arange(8))
    khat = np.stack([np.sin(th), 0 * th, -np.cos(th)], axis=1)
    pol = np.stack([np.cos(th), 0 * th, np.sin(th)], axis=1)
    b = np.zeros((8, op.N), complex)
    op.rhs_planewave(khat, pol, b)
    x = np.zeros_like(b)
    info = op.solve(b, x, nrhs=8, tol=1e-10)
    assert info["relres"] < 1e-10
    ref = np.linalg.solve(cyl4.A.Z, b.T).T
    for r in range(8):
        assert rel(x[r], ref[r]) < 1e-6, (r, rel(x[r], ref[r]))


def _entrywise(got, ref, name):
    floor = FP32_FLOOR * np.max(np.abs(ref))
    bad = np.abs(got - ref) > 1e-5 * np.abs(ref) + floor
    assert not bad.any(), (name, int(bad.sum()), float(np.max(np.abs(got - ref) / (np.abs(ref) + floor))))


@pytest.mark.parametrize("which", ["sphere", "two_lossy", "cyl4"])
def test_fp32_fill_entrywise(which, request):
    case = request.getfixturevalue(which)
    sl, op = build(case, 1)
    for name, got, ref in _blocks(case, op, sl, with_y=False):
        _entrywise(got, ref, name)


def _edge_entry(om, la_fn, m, n):
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


@pytest.mark.parametrize("prec", [1, 2])
def test_metasurface_8x8_sampled_entries(prec):
    """The full 8 x 8 metasurface (15,360 triangles) in the bench's configuration:
    sampled entries of L^A_m and L^phi_m, near and far, against the oracle one
    triangle pair at a time (FP32 fill: entrywise bound above; F32X2: 1e-10)."""
    import torch
    sl = _sl()
    xyz, tri, obj = cylinder_array(8, 8, 120e-9, 300e-9, 500e-9)
    om = OMesh(xyz, tri, obj)
    m = sl.Mesh(xyz, tri, obj)
    st = sl.Stack([(1.0, 1.0, 0.0, 0.0)])
    freq = 299792458.0 / 1e-6
    op = sl.Operator(m, st, [(6.0, 1.0, 0.0)] * 64, freq, precision=prec)
    k0 = 2 * np.pi * freq / S.C0
    rng = np.random.default_rng(64 + prec)
    # edges: random pairs over the whole array, plus pairs inside one cylinder and its neighbour
    E = rng.integers(0, om.ne, (16, 2))
    E2 = rng.integers(0, 360, (8, 2)) + np.array([[0, 360]])
    E = np.concatenate([E, E2])
    T = rng.integers(0, om.nt, (24, 2))
    T[:8, 1] = T[:8, 0] + rng.integers(-3, 4, 8)
    T = np.clip(T, 0, om.nt - 1)
    la_fn = lambda a, b: OFL._L_pairs(om, k0, a, b)[0]
    LAm = torch.empty((om.ne, om.ne), dtype=torch.complex128, device="cuda")
    op.block_into(sl.BLOCK_LAM, LAm)
    got_a = LAm[torch.as_tensor(E[:, 0]), torch.as_tensor(E[:, 1])].cpu().numpy()
    amax = float(LAm.abs().max())
    del LAm
    LPm = torch.empty((om.nt, om.nt), dtype=torch.complex128, device="cuda")
    op.block_into(sl.BLOCK_LPM, LPm)
    got_p = LPm[torch.as_tensor(T[:, 0]), torch.as_tensor(T[:, 1])].cpu().numpy()
    pmax = float(LPm.abs().max())
    del LPm
    torch.cuda.empty_cache()
    ref_a = np.array([_edge_entry(om, la_fn, mm, nn) for mm, nn in E])
    ref_p = OFL._L_pairs(om, k0, T[:, 0], T[:, 1])[1]
    if prec == 1:
        assert np.all(np.abs(got_a - ref_a) <= 1e-5 * np.abs(ref_a) + FP32_FLOOR * amax), np.abs(got_a / ref_a - 1)
        assert np.all(np.abs(got_p - ref_p) <= 1e-5 * np.abs(ref_p) + FP32_FLOOR * pmax), np.abs(got_p / ref_p - 1)
    else:
        assert np.max(np.abs(got_a - ref_a)) <= 1e-10 * amax
        assert np.max(np.abs(got_p - ref_p)) <= 1e-10 * pmax
