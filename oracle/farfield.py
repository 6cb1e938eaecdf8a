"""Far field and radar cross section of the equivalent current J_Delta radiating
in free space (Sec. IV-A: RCS compared with the Mie series).

With j_Delta = j k0 J_Delta (RWG coefficients) and exp(+j w t), the scattered far
field is E_s = -eta0 exp(-j k0 r)/(4 pi r) (I - rr) . sum_n j_Delta,n N_n(rhat),
N_n = int f_n(r') exp(+j k0 rhat . r') dS' (6-point rule), so that the bistatic
RCS is sigma = eta0^2 |(I - rr) . F|^2 / (4 pi |E0|^2).
"""
import numpy as np

from . import quadrature as Q
from .fill import ETA0


def rcs(mesh, k0, jd, theta, phi=0.0, E0=1.0):
    theta = np.atleast_1d(np.asarray(theta, float))
    phi = np.broadcast_to(np.asarray(phi, float), theta.shape)
    rhat = np.stack([np.sin(theta) * np.cos(phi), np.sin(theta) * np.sin(phi), np.cos(theta)], axis=1)
    A = mesh.xyz[mesh.tri]
    rq = Q.points(A)
    wq = Q.weights(mesh.area)
    Fv = np.zeros((len(theta), 3), dtype=complex)
    ph = np.exp(1j * k0 * np.einsum('tqd,ad->atq', rq, rhat))            # (ang, nt, 6)
    for i in range(3):
        fi = (rq - A[:, i][:, None, :]) * (mesh.E.tri_sign[:, i] / (2 * mesh.area))[:, None, None]
        c = jd[mesh.E.tri_edge[:, i]]
        Fv += np.einsum('t,tq,atq,tqd->ad', c, wq, ph, fi)
    Fperp = Fv - rhat * np.einsum('ad,ad->a', rhat, Fv)[:, None]
    return ETA0 ** 2 * np.sum(np.abs(Fperp) ** 2, axis=1) / (4 * np.pi * abs(E0) ** 2)


def _rwg_radiation(P, area, tri_edge, tri_sign, coef, k0, rhat):
    """sum_n coef_n int f_n(r') exp(+j k0 rhat . r') dS' for the RWG functions of the
    triangles P (nt, 3, 3) (6-point rule), one row per direction rhat (n, 3)."""
    rq = Q.points(P)
    wq = Q.weights(area)
    out = np.zeros((len(rhat), 3), dtype=complex)
    ph = np.exp(1j * k0 * np.einsum('tqd,ad->atq', rq, rhat))
    for i in range(3):
        fi = (rq - P[:, i][:, None, :]) * (tri_sign[:, i] / (2 * area))[:, None, None]
        out += np.einsum('t,tq,atq,tqd->ad', coef[tri_edge[:, i]], wq, ph, fi)
    return out


def amplitude(mesh, k0, jd, rhat):
    """Complex far-field amplitude A(rhat) of J_Delta in free space, E_s ~ A exp(-j k0 r)/r:
    A = -eta0/(4 pi) (I - rr) . sum_n j_Delta,n N_n(rhat), one row per direction
    (rhat: (n, 3) unit vectors).  The RCS above is 4 pi |A|^2 / |E0|^2; the
    forward amplitude gives the extinction cross section by the optical theorem,
    sigma_ext = -(4 pi / k0) Im(p . A(khat)) / |E0|^2 for E_inc = p E0 exp(-j k0 khat . r)
    (the exp(+j w t) form of the theorem)."""
    rhat = np.atleast_2d(np.asarray(rhat, float))
    F = _rwg_radiation(mesh.xyz[mesh.tri], mesh.area, mesh.E.tri_edge, mesh.E.tri_sign, jd, k0, rhat)
    return -ETA0 / (4 * np.pi) * (F - rhat * np.einsum('ad,ad->a', rhat, F)[:, None])


def love_amplitude(mesh, k0, j, e, rhat):
    """Far-field amplitude of the total surface fields by Love's equivalence (the
    Stratton-Chu representation of the exterior field): the electric current
    J = n x H (RWG coefficients j / (j k0), j = the unknowns' first block) and the
    magnetic current M = -n x E (BC coefficients -eta0 e, e = the second block)
    radiating in free space, with E_J = -j w mu0 (I - rr) . int J exp(+j k0 rhat . r') / (4 pi)
    and E_M = j k0 rhat x int M exp(+j k0 rhat . r') / (4 pi):
        A = -eta0/(4 pi) [(I - rr) . sum_n j_n N_n + j k0 rhat x sum_n e_n N^BC_n],
    N^BC_n the same integral of the BC function, a combination of barycentric RWGs.
    The single-layer method radiates J_Delta = H - H_eq alone (amplitude above);
    both must give the scattered field outside."""
    rhat = np.atleast_2d(np.asarray(rhat, float))
    NJ = _rwg_radiation(mesh.xyz[mesh.tri], mesh.area, mesh.E.tri_edge, mesh.E.tri_sign, j, k0, rhat)
    NM = _rwg_radiation(mesh.bxyz[mesh.btri], mesh.barea, mesh.bE.tri_edge, mesh.bE.tri_sign, mesh.C @ e, k0, rhat)
    NJp = NJ - rhat * np.einsum('ad,ad->a', rhat, NJ)[:, None]
    return -ETA0 / (4 * np.pi) * (NJp + 1j * k0 * np.cross(rhat, NM))


def rcs_layered(mesh, stack, layer, omega, jd, theta, phi=0.0, E0=1.0):
    """Bistatic RCS above a stratified background (observation in the upper half-space).

    By reciprocity, the far-field component along p of the current radiating in
    layer `layer` of the stack is the current's reaction with the stack's total
    field of a plane wave arriving from the observation direction rhat with
    polarisation p (oracle.layered.incident_field with khat = -rhat): the
    free-space factor exp(+j k0 rhat . r') p becomes that field.  With
    F_p = sum_n j_Delta,n int f_n . E_(-rhat, p) dS' for p = theta-hat, phi-hat,
    sigma = eta0^2 (|F_theta|^2 + |F_phi|^2) / (4 pi |E0|^2).  theta < pi/2."""
    from . import layered as LY
    theta = np.atleast_1d(np.asarray(theta, float))
    phi = np.broadcast_to(np.asarray(phi, float), theta.shape)
    if np.any(theta >= np.pi / 2):
        raise ValueError("layered far field: observation directions in the upper half-space only")
    A = mesh.xyz[mesh.tri]
    rq = Q.points(A)
    wq = Q.weights(mesh.area)
    pts = rq.reshape(-1, 3)
    out = np.zeros(len(theta))
    for a, (th, ph) in enumerate(zip(theta, phi)):
        rhat = np.array([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)])
        that = np.array([np.cos(th) * np.cos(ph), np.cos(th) * np.sin(ph), -np.sin(th)])
        phat = np.array([-np.sin(ph), np.cos(ph), 0.0])
        s = 0.0
        for p in (that, phat):
            E = LY.incident_field(stack, layer, omega, -rhat, p, pts).reshape(rq.shape)   # (nt, 6, 3)
            F = 0j
            for i in range(3):
                fi = (rq - A[:, i][:, None, :]) * (mesh.E.tri_sign[:, i] / (2 * mesh.area))[:, None, None]
                c = jd[mesh.E.tri_edge[:, i]]
                F += np.einsum('t,tq,tqd,tqd->', c, wq, fi, E)
            s += abs(F) ** 2
        out[a] = ETA0 ** 2 * s / (4 * np.pi * abs(E0) ** 2)
    return out
