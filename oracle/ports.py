"""Delta-gap edge ports, port currents and network parameters (Sec. IV-B: a
delta-gap edge port at the centre of the dipole, where S11 is measured; Sec.
IV-C: two such ports on the inductor).  Test infrastructure: only the tests, the
package's smoke check and the bench's CPU leg use this module.

The paper takes the delta-gap edge port from the method-of-moments literature
(Gibson) without restating it.  Reading used here (and by the CUDA library):

* A port on object o is the closed ring of mesh edges that lie in the plane
  s . r = c (s a unit vector along the feed), each edge having one triangle on
  each side of the plane.  Its edge n carries the sign sigma_n = +1 when T+ of
  the edge lies on the -s side (the RWG's unit flux crosses the plane along +s),
  -1 otherwise.
* The source is an impressed electric field V delta(s . r - c) s on the surface,
  an incident field confined to the gap.  Like the plane wave it enters the
  external EFIE only (row 1 of Eq. finalsystem): tested with the area-normalised
  RWG f_n (unit flux through its edge), <f_n, V delta s> = sigma_n V on the ring
  edges and 0 elsewhere (the other RWGs have no normal component on the ring
  edges), so b_n = sigma_n V / eta0 in the system's scaling (E / eta0).
* The port current is the electric surface current n x H through the ring along
  +s: with the unknown j = j k0 H (RWG coefficients of n x H, unit flux each),
  I = sum_n sigma_n j_n / (j k0).
* Network parameters: exciting port p with V_p = 1 and every other port with
  0 (shorted) gives the column Y[:, p] = I; Z = Y^-1 and, for a real reference
  impedance z0 at every port, S = (Z - z0)(Z + z0)^-1 = (I - z0 Y)(I + z0 Y)^-1.

Parity pinned by tests/test_oracle_ports.py: the ring right-hand side against a
brute-force surface integral of a finite gap field, the input power
Re(V I*) / 2 against the power radiated to infinity (a surface integral of the
far field) for a lossless dielectric bar, reciprocity Y12 = Y21 of two ports,
and S of a one-port against the reflection coefficient formula.
"""
from __future__ import annotations

import numpy as np

from .fill import ETA0


class Port:
    """A ring of edges (indices into the mesh's edge list) with their signs."""

    def __init__(self, edges, signs):
        self.edges = np.asarray(edges, dtype=np.int64)
        self.signs = np.asarray(signs, dtype=np.float64)


def port_ring(mesh, obj: int, s, c: float, tol: float = None) -> Port:
    """The edges of object ``obj`` in the plane s . r = c with one triangle on each side."""
    s = np.asarray(s, float)
    s = s / np.linalg.norm(s)
    e0, e1 = mesh.edge_range[obj]
    if tol is None:
        tol = 1e-9 * np.ptp(mesh.xyz, axis=0).max()
    d = mesh.xyz @ s - c
    cen = mesh.xyz[mesh.tri].mean(axis=1) @ s - c
    edges, signs = [], []
    for n in range(e0, e1):
        u, v = mesh.E.uv[n]
        if abs(d[u]) > tol or abs(d[v]) > tol:
            continue
        cp, cm = cen[mesh.E.tp[n]], cen[mesh.E.tm[n]]
        if cp * cm >= 0:
            continue  # both triangles on one side: an edge of the ring plane's outline, not a gap edge
        edges.append(n)
        signs.append(+1.0 if cp < 0 else -1.0)
    if not edges:
        raise ValueError("port: no edge of the object lies in the port plane")
    return Port(edges, signs)


def port_rhs(a, ports, V) -> np.ndarray:
    """Right-hand sides, one column per column of V (ports x columns)."""
    m = a.mesh
    V = np.asarray(V, dtype=complex).reshape(len(ports), -1)
    b = np.zeros((2 * m.ne + m.nt - m.nobj, V.shape[1]), dtype=complex)
    for p, port in enumerate(ports):
        b[port.edges, :] += port.signs[:, None] * V[p][None, :] / ETA0
    return b


def port_currents(a, x, ports) -> np.ndarray:
    """Currents through the ports (ports x columns) of solutions x (N x columns)."""
    x = np.asarray(x).reshape(x.shape[0], -1)
    out = np.zeros((len(ports), x.shape[1]), dtype=complex)
    for p, port in enumerate(ports):
        out[p] = (port.signs[:, None] * x[port.edges, :]).sum(axis=0) / (1j * a.k0)
    return out


def y_matrix(a, ports, solve) -> np.ndarray:
    """Admittance matrix: column p from unit voltage at port p, the others shorted."""
    b = port_rhs(a, ports, np.eye(len(ports)))
    x = solve(a, b)
    return port_currents(a, x, ports)


def s_matrix(Y, z0: float = 50.0) -> np.ndarray:
    Y = np.atleast_2d(np.asarray(Y, dtype=complex))
    n = Y.shape[0]
    return np.linalg.solve((np.eye(n) + z0 * Y).T, (np.eye(n) - z0 * Y).T).T


def input_power(V, I) -> float:
    """Time-average power delivered by a port source (exp(+j w t) phasors)."""
    return 0.5 * float(np.real(V * np.conj(I)))


def radiated_power(mesh, k0, jd, n_theta: int = 48, n_phi: int = 64) -> float:
    """Power radiated by j_Delta (free space): (1 / (2 eta0)) int |r E|^2 dOmega, with
    |r E|^2 = sigma / (4 pi) for |E0| = 1 (oracle.farfield.rcs); Gauss-Legendre in
    cos(theta), trapezoidal in phi."""
    from .farfield import rcs
    xg, wg = np.polynomial.legendre.leggauss(n_theta)
    th = np.arccos(xg)
    ph = 2 * np.pi * np.arange(n_phi) / n_phi
    T, P = np.meshgrid(th, ph, indexing='ij')
    W = np.outer(wg, np.full(n_phi, 2 * np.pi / n_phi))
    sig = rcs(mesh, k0, jd, T.ravel(), P.ravel()).reshape(T.shape)
    return float(np.sum(W * sig) / (4 * np.pi) / (2 * ETA0))
