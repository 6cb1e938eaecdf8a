"""Pins of the oracle's delta-gap ports (oracle/ports.py; Sec. IV-B, IV-C).

* The ring right-hand side against a brute-force surface integral of a finite
  gap field V/delta s on |s . r - c| < delta / 2: every RWG's integral over the
  band, clipped exactly out of its two triangles (f_n is linear there, so the
  integral is the clipped area times f_n at its centroid).  As delta -> 0 it
  tends to sigma_n V on the ring edges and to 0 elsewhere.
* Power balance of a lossy dipole (bar of sigma = 1e3 S/m, 0.48 wavelengths
  long, free space): the input power Re(V I*)/2 equals the power radiated to
  infinity (far field of j_Delta integrated over the sphere) plus the ohmic
  loss, estimated by the surface-impedance (Leontovich) formula
  Rs/2 int |J|^2 dS with Rs = sqrt(w mu0 / (2 sigma)) (skin depth 0.09 mm
  against a 4 mm cross-section).  A wrong sign on ring edges, a missing 1/eta0
  or 1/(j k0) changes the balance by far more than the 2% allowed.
* Reciprocity: Y12 = Y21 for two ports on the same dipole.
* S of a one-port is the reflection coefficient (Z - z0)/(Z + z0), and S of a
  matched port is 0.
"""
import numpy as np
import pytest

from oracle import system as S, ports as PT, quadrature as Q
from oracle.fill import C0, MU0
from oracle.topology import Mesh as OMesh
from workloads.meshes import box

F = 3e9
LAM = C0 / F
LEN = 0.48 * LAM
SIGMA = 1e3


def _bar(ny=12):
    xyz, tri = box(0.04 * LAM, LEN, 0.04 * LAM, 2, ny, 2)
    return OMesh(xyz, tri, np.zeros(len(tri), int))


def _clip(poly, s, lo, hi):
    """The part of a convex polygon (k x 3) with lo <= s . r <= hi."""
    for sgn, bound in ((1.0, hi), (-1.0, -lo)):
        out = []
        n = len(poly)
        for i in range(n):
            p, q = poly[i], poly[(i + 1) % n]
            dp, dq = sgn * (p @ s) - bound, sgn * (q @ s) - bound
            if dp <= 0:
                out.append(p)
            if dp * dq < 0:
                out.append(p + (q - p) * (dp / (dp - dq)))
        poly = np.array(out)
        if len(poly) < 3:
            return None
    return poly


def _area_centroid(poly):
    a, c = 0.0, np.zeros(3)
    for i in range(1, len(poly) - 1):
        t = np.cross(poly[i] - poly[0], poly[i + 1] - poly[0])
        ai = 0.5 * np.linalg.norm(t)
        a += ai
        c += ai * (poly[0] + poly[i] + poly[i + 1]) / 3
    return a, (c / a if a > 0 else c)


def test_port_rhs_matches_finite_gap_integral():
    m = _bar()
    s = np.array([0.0, 1.0, 0.0])
    port = PT.port_ring(m, 0, s, 0.0)
    h = LEN / 12
    V = 1.3 - 0.4j
    delta = 1e-7 * h
    brute = np.zeros(m.ne, complex)
    for n in range(m.ne):
        for t, loc, sg in ((m.E.tp[n], m.E.ip[n], 1.0), (m.E.tm[n], m.E.im[n], -1.0)):
            P = m.xyz[m.tri[t]]
            poly = _clip(P.copy(), s, -delta / 2, delta / 2)
            if poly is None:
                continue
            a, cen = _area_centroid(poly)
            f = sg * (cen - P[loc]) / (2 * m.area[t])
            brute[n] += a * (f @ s) * V / delta
    closed = np.zeros(m.ne, complex)
    closed[port.edges] = port.signs * V
    assert np.max(np.abs(brute - closed)) < 1e-5 * abs(V)
    # the oracle's right-hand side is that, in the system's scaling E / eta0
    a = S.Assembled(mesh=m, k0=2 * np.pi / LAM, LAm=None, LPm=None, Ix=None)
    b = PT.port_rhs(a, [port], [V])[:, 0]
    from oracle.fill import ETA0
    assert np.allclose(b[:m.ne] * ETA0, closed) and not np.any(b[m.ne:])


def test_port_ring_is_a_closed_loop_around_the_section():
    m = _bar()
    port = PT.port_ring(m, 0, (0, 1, 0), 0.0)
    assert len(port.edges) == 8           # 2 + 2 + 2 + 2 grid edges around the section
    verts = m.E.uv[port.edges].ravel()
    _, counts = np.unique(verts, return_counts=True)
    assert np.all(counts == 2)            # every ring vertex joins two ring edges
    assert np.allclose(m.xyz[verts, 1], 0.0)
    # a plane through no vertex row has no ring
    with pytest.raises(ValueError):
        PT.port_ring(m, 0, (0, 1, 0), 0.5 * LEN / 12)


@pytest.fixture(scope="module")
def dipole():
    m = _bar()
    a = S.assemble(m, [S.Material(1.0, 1.0, SIGMA)], S.Material(), F)
    ports = [PT.port_ring(m, 0, (0, 1, 0), 0.0), PT.port_ring(m, 0, (0, 1, 0), LEN / 4)]
    b = PT.port_rhs(a, ports, np.eye(2))
    x = S.solve(a, b)
    return m, a, ports, x


def _ohmic_loss(m, k0, j, sigma, omega):
    A = m.xyz[m.tri]
    rq = Q.points(A)
    wq = Q.weights(m.area)
    J = np.zeros(rq.shape, complex)
    for i in range(3):
        fi = (rq - A[:, i][:, None, :]) * (m.E.tri_sign[:, i] / (2 * m.area))[:, None, None]
        J += (j[m.E.tri_edge[:, i]] / (1j * k0))[:, None, None] * fi
    Rs = np.sqrt(omega * MU0 / (2 * sigma))
    return 0.5 * Rs * np.sum(wq[:, :, None] * np.abs(J) ** 2)


def test_input_power_is_radiated_plus_ohmic(dipole):
    m, a, ports, x = dipole
    I = PT.port_currents(a, x[:, :1], ports)[:, 0]
    Pin = PT.input_power(1.0, I[0])          # port 2 shorted: no power there
    Prad = PT.radiated_power(m, a.k0, S.j_delta(a, x[:, 0]))
    Ploss = _ohmic_loss(m, a.k0, x[:m.ne, 0], SIGMA, 2 * np.pi * F)
    assert Pin > 0 and Prad < Pin
    assert abs((Prad + Ploss) / Pin - 1) < 0.02, (Pin, Prad, Ploss)
    Zin = 1 / I[0]                           # the other port shorted: the plain dipole
    assert 50 < Zin.real < 200               # a half-wave dipole with some loss


def test_two_port_reciprocity(dipole):
    m, a, ports, x = dipole
    Y = PT.port_currents(a, x, ports)
    assert abs(Y[0, 1] - Y[1, 0]) < 1e-3 * abs(Y[0, 1])


def test_s_matrix_closed_forms():
    z0 = 50.0
    for Z in (50.0, 73.0 + 42.5j, 10.0 - 300.0j):
        Sm = PT.s_matrix(np.array([[1 / Z]]), z0)
        assert abs(Sm[0, 0] - (Z - z0) / (Z + z0)) < 1e-14
    # two uncoupled matched ports reflect nothing
    assert np.allclose(PT.s_matrix(np.diag([1 / z0, 1 / z0]), z0), 0.0)
    # a lossless reciprocal two-port (a series reactance) has a unitary S
    X = 37.0
    Y = np.array([[1, -1], [-1, 1]]) / (1j * X)
    Sm = PT.s_matrix(Y, z0)
    assert np.allclose(Sm.conj().T @ Sm, np.eye(2), atol=1e-12)
