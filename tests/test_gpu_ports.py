"""Delta-gap edge ports through the C ABI against the oracle (oracle/ports.py;
Sec. IV-B, IV-C): the rings, the port right-hand sides and currents (exact
arithmetic on both sides: 1e-14), and the admittance and scattering matrices
of solved systems (GMRES to 1e-11 against the oracle's dense solve: 1e-6) for
a two-port lossy dipole in free space and a one-port dipole above a scaled
version of the paper's ground stack (Table I, sphere-array column, all sizes
and conductivities scaled from 200 MHz to 3 GHz).
"""
import numpy as np
import pytest

from oracle import layered as LY
from oracle import ports as PT
from oracle import system as S
from oracle.fill import C0
from oracle.topology import Mesh as OMesh
from workloads.meshes import box

pytestmark = pytest.mark.gpu

F = 3e9
LAM = C0 / F
LEN = 0.48 * LAM
SIGMA = 1e3
SC = 1 / 15  # 200 MHz -> 3 GHz


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _sl():
    import torch  # noqa: F401
    from paper_2106_06184_gb300 import sldm
    return sldm


class Case:
    pass


@pytest.fixture(scope="module")
def free2():
    c = Case()
    c.xyz, c.tri = box(0.04 * LAM, LEN, 0.04 * LAM, 2, 12, 2)
    c.om = OMesh(c.xyz, c.tri, np.zeros(len(c.tri), int))
    c.A = S.assemble(c.om, [S.Material(1.0, 1.0, SIGMA)], S.Material(), F)
    c.planes = [0.0, LEN / 4]
    c.oports = [PT.port_ring(c.om, 0, (0, 1, 0), p) for p in c.planes]
    c.Y = PT.y_matrix(c.A, c.oports, S.solve)
    return c


@pytest.fixture(scope="module")
def ground1():
    c = Case()
    c.xyz, c.tri = box(0.075 * SC, 0.75 * SC, 0.0375 * SC, 2, 8, 2, center=(0, 0, 0.49375 * SC))
    c.layers = [(1.0, 1.0, 0.0, np.inf), (3.47, 1.0, 0.001725 / SC, 0.525 * SC), (6.5, 1.0, 0.003338 / SC, np.inf)]
    c.z_top = 0.375 * SC
    c.om = OMesh(c.xyz, c.tri, np.zeros(len(c.tri), int))
    stack = LY.Stack(c.layers, z_top=c.z_top, bottom="halfspace")
    c.A = S.assemble(c.om, [S.Material(1.0, 1.0, SIGMA)], stack, F, layer=0)
    c.oports = [PT.port_ring(c.om, 0, (0, 1, 0), 0.0)]
    c.Y = PT.y_matrix(c.A, c.oports, S.solve)
    return c


def _gpu(sl, c, prec=0, layered=False):
    m = sl.Mesh(c.xyz, c.tri)
    if layered:
        st = sl.Stack([(l[0], l[1], l[2], l[3] if np.isfinite(l[3]) else 0.0) for l in c.layers], z_top=c.z_top,
                      bottom=sl.BOTTOM_HALFSPACE)
        op = sl.Operator(m, st, [(1.0, 1.0, SIGMA, 0)], F, precision=prec)
    else:
        st = sl.Stack([(1.0, 1.0, 0.0, 0.0)])
        op = sl.Operator(m, st, [(1.0, 1.0, SIGMA)], F, precision=prec)
    return m, st, op


def test_port_rings_match_oracle(free2):
    sl = _sl()
    m = sl.Mesh(free2.xyz, free2.tri)
    for p, op_ in zip(free2.planes, free2.oports):
        e, g = sl.port_ring(m, 0, (0.0, 2.0, 0.0), p)       # any length of the normal
        assert np.array_equal(e, op_.edges) and np.array_equal(g, op_.signs.astype(np.int8))
        e2, g2 = sl.port_ring(m, 0, (0.0, -1.0, 0.0), -p)   # the reversed plane flips every sign
        assert np.array_equal(e2, e) and np.array_equal(g2, -g)
    with pytest.raises(sl.SldmError):
        sl.port_ring(m, 0, (0.0, 1.0, 0.0), 0.5 * LEN / 12)  # no vertex row there
    with pytest.raises(sl.SldmError):
        sl.port_ring(m, 1, (0.0, 1.0, 0.0), 0.0)             # no such object


def test_port_rhs_and_currents_match_oracle(free2):
    sl = _sl()
    m, st, op = _gpu(sl, free2)
    ports = sl.Ports([(p.edges, p.signs) for p in free2.oports])
    rng = np.random.default_rng(11)
    V = rng.standard_normal((2, 3)) + 1j * rng.standard_normal((2, 3))
    b = np.zeros((3, op.N), complex)
    op.port_rhs(ports, V, b)
    bo = PT.port_rhs(free2.A, free2.oports, V)
    assert rel(b.T, bo) < 1e-14
    x = rng.standard_normal((3, op.N)) + 1j * rng.standard_normal((3, op.N))
    x = np.ascontiguousarray(x)
    I = op.port_currents(x, ports, ncols=3)
    Io = PT.port_currents(free2.A, x.T, free2.oports)
    assert rel(I, Io) < 1e-14
    # device buffers take the same path
    import torch
    bt = torch.zeros((3, op.N), dtype=torch.complex128, device="cuda")
    op.port_rhs(ports, V, bt)
    assert rel(bt.cpu().numpy().T, bo) < 1e-14
    xt = torch.from_numpy(x).cuda()
    assert rel(op.port_currents(xt, ports, ncols=3), Io) < 1e-14


def test_two_port_y_and_s_match_oracle(free2):
    sl = _sl()
    m, st, op = _gpu(sl, free2)
    ports = sl.Ports([(p.edges, p.signs) for p in free2.oports])
    b = np.zeros((2, op.N), complex)
    op.port_rhs(ports, np.eye(2), b)
    x = np.zeros_like(b)
    info = op.solve(b, x, nrhs=2, tol=1e-11)
    assert info["relres"] <= 1e-11
    Y = op.port_currents(x, ports, ncols=2)
    assert rel(Y, free2.Y) < 1e-6, (Y, free2.Y)
    assert abs(Y[0, 1] - Y[1, 0]) < 1e-3 * abs(Y[0, 1])
    Sg = sl.sparams(Y, 50.0)
    assert rel(Sg, PT.s_matrix(free2.Y, 50.0)) < 1e-6


@pytest.mark.parametrize("prec", [0, 2])
def test_s11_over_ground_stack_matches_oracle(ground1, prec):
    """FP64, and complex64 with the FP64-accurate refinement residual."""
    sl = _sl()
    m, st, op = _gpu(sl, ground1, prec=prec, layered=True)
    ports = sl.Ports([(p.edges, p.signs) for p in ground1.oports])
    b = np.zeros((1, op.N), complex)
    op.port_rhs(ports, [[1.0]], b)
    x = np.zeros_like(b)
    op.solve(b, x, nrhs=1, tol=1e-11)
    Y = op.port_currents(x, ports)
    assert abs(Y[0, 0] - ground1.Y[0, 0]) < 1e-6 * abs(ground1.Y[0, 0])
    s11 = sl.sparams(Y)[0, 0]
    assert abs(s11 - PT.s_matrix(ground1.Y)[0, 0]) < 1e-6


def test_port_arguments_rejected(free2):
    sl = _sl()
    m, st, op = _gpu(sl, free2)
    p = free2.oports[0]
    b = np.zeros((1, op.N), complex)
    bad = [sl.Ports([(p.edges, p.signs)]) for _ in range(3)]
    bad[0].ptr[0] = 1                        # CSR must start at 0
    bad[1].edges[0] = op.N                   # edge out of range
    bad[2].signs[0] = 0                      # sign must be +-1
    for ports in bad:
        with pytest.raises(sl.SldmError):
            op.port_rhs(ports, [[1.0]], b)
    with pytest.raises(sl.SldmError):
        sl.sparams(np.eye(2), 0.0)
    with pytest.raises(sl.SldmError):
        sl.sparams(-np.eye(1) / 50.0, 50.0)  # 1 + z0 Y singular
