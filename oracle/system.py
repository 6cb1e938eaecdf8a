"""Assembly and dense solution of the single-layer dual-mesh system (Sec. II-B to II-E).

Unknowns, in this order (Eq. finalsystem):
    j  = j k0 H      RWG coefficients of n x H               (ne)
    e  = E / eta0    BC coefficients of n x E                (ne)
    u  = -c0 rho     pulse coefficients, each object's last triangle eliminated by B (nt - nobj)

Blocks (block-diagonal over objects where marked "o", Eq. Aobj):
    internal (object material, k):        mu_r L^A, eps_cr^-1 L^phi, K = Kbar + I_x / 2     (o)
    equivalent (background, k_l):         M_l = [[mu_l L^A_l, -eps_l^-1 D^T L^phi_l B], [F D, -k0^2 I]]
                                          [Y11; Y21] = M_l^-1 [[Kbar_l + I_x / 2], [0]]      (o)
    external (background, global):        L^A_m = mu_b L^A(k_b), L^phi_m = eps_b^-1 L^phi(k_b)

Final system (Eq. finalsystem, with C1, C2 of Eqs. C1, C2):
    [ L^A_m      C1   D^T L^phi_m B         ] [j]   [e_inc]
    [ mu_r L^A   -K   eps_cr^-1 D^T L^phi B ] [e] = [  0  ]
    [ F D        C2   k0^2 I                ] [u]   [  0  ]
    C1 = I_x - (L^A_m Y11 - D^T L^phi_m B Y21),   C2 = -(F D Y11 - k0^2 Y21).

Readings: row 2 carries -K (moving the right-hand side of Eq. AEFIEintdis to the
left gives -(Kbar + I_x/2); the printed +K is taken as a sign slip), and C1 uses
L^phi_m (it comes from row 1 of Eq. AEFIEextdisY; the printed L^phi_l coincides
with it in a homogeneous background).  The external operators here are those of
a homogeneous background (L^A_m = L^A_l); the tabulated layered kernel is not
part of this module.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.linalg as sla

from .fill import C0, EPS0, fill_L, fill_Kbar, fill_Ix, plane_wave


@dataclass
class Material:
    eps_r: float = 1.0
    mu_r: float = 1.0
    sigma: float = 0.0


def eps_c(m: Material, omega: float) -> complex:
    """Relative complex permittivity, Eq. epsrc."""
    return m.eps_r - 1j * m.sigma / (omega * EPS0)


def wavenumber(m: Material, k0: float) -> complex:
    """k = sqrt(eps_cr mu_r) k0 on the principal branch (Im k <= 0 for exp(-j k R) decay)."""
    return k0 * np.sqrt(complex(eps_c(m, k0 * C0)) * m.mu_r)


@dataclass
class Assembled:
    mesh: object
    k0: float
    LAm: np.ndarray
    LPm: np.ndarray
    Ix: np.ndarray
    blocks: list = field(default_factory=list)   # per object dict
    Z: np.ndarray = None


def assemble(mesh, materials, background, freq: float, build_Z: bool = True, layer: int = None,
             tables=None) -> Assembled:
    """background: a Material (homogeneous) or an oracle.layered.Stack with every object in
    ``layer``.  In a stack, the equivalent configuration (M_l, Eq. AEFIEeqvdis) uses the
    homogeneous kernels of layer l and L^A_m, L^phi_m add the reflected part of the
    multilayer kernel (images + tabulated remainder, see oracle.layered)."""
    omega = 2 * np.pi * freq
    k0 = omega / C0
    layered = not isinstance(background, Material)
    if layered:
        from . import layered as LY
        stack = background
        background = Material(stack.layers[layer][0], stack.layers[layer][1], stack.layers[layer][2])
    kb = wavenumber(background, k0)
    eb = eps_c(background, omega)
    all_tris = np.arange(mesh.nt)
    LA_b, LP_b = fill_L(mesh, kb, all_tris)
    LA_hom = background.mu_r * LA_b
    LP_hom = LP_b / eb
    LAm, LPm = LA_hom, LP_hom
    if layered:
        if tables is None:
            tables = default_tables(mesh, stack, layer, omega)
        LA_r, LP_r = LY.fill_reflected(mesh, stack, layer, omega, tables, all_tris)
        LAm, LPm = LA_hom + LA_r, LP_hom + LP_r
    Ix = fill_Ix(mesh)
    D, B, F = mesh.D(), mesh.B(), mesh.F()
    out = Assembled(mesh=mesh, k0=k0, LAm=LAm, LPm=LPm, Ix=Ix)
    for o in range(mesh.nobj):
        mat = materials[o]
        t0, t1 = mesh.tri_range[o]
        e0, e1 = mesh.edge_range[o]
        ko, eo = wavenumber(mat, k0), eps_c(mat, omega)
        tris = np.arange(t0, t1)
        LA_o, LP_o = fill_L(mesh, ko, tris)
        Kb_o, _ = fill_Kbar(mesh, ko, o)
        Ix_o = Ix[e0:e1, e0:e1]
        Do = D[t0:t1, e0:e1]
        Bo = B[t0:t1, t0 - o:t1 - o - 1]
        Fo = F[t0 - o:t1 - o - 1, t0:t1]
        # equivalent configuration: the object replaced by the background (Eq. AEFIEeqvdis),
        # homogeneous kernels of the background layer
        LA_l = LA_hom[e0:e1, e0:e1] / background.mu_r
        LP_l = LP_hom[t0:t1, t0:t1] * eb
        Kb_l, _ = fill_Kbar(mesh, kb, o)
        ne_o, nt_o = e1 - e0, t1 - t0
        Ml = np.block([[background.mu_r * LA_l, -(Do.T @ LP_l @ Bo) / eb],
                       [Fo @ Do, -k0 ** 2 * np.eye(nt_o - 1)]])
        Rl = np.vstack([Kb_l + 0.5 * Ix_o, np.zeros((nt_o - 1, ne_o))])
        Y = np.linalg.solve(Ml, Rl)                                   # Eq. Yeqdef
        out.blocks.append(dict(
            LA=mat.mu_r * LA_o, LP=LP_o / eo, K=Kb_o + 0.5 * Ix_o, Kbar=Kb_o,
            Kbar_l=Kb_l, Y11=Y[:ne_o], Y21=Y[ne_o:], Ml=Ml, k=ko, eps_c=eo,
            D=Do, B=Bo, F=Fo))
    out.layered = (stack, layer, tables) if layered else None
    if build_Z:
        out.Z = final_matrix(out)
    return out


def default_tables(mesh, stack, layer, omega):
    """Remainder tables over the objects' extent: 256 log-spaced rho x 128 (z + z') and 128 |z - z'|."""
    from . import layered as LY
    lo, hi = mesh.xyz.min(axis=0), mesh.xyz.max(axis=0)
    span = np.linalg.norm(hi - lo) * 1.01
    edge = np.min(np.linalg.norm(mesh.xyz[mesh.E.uv[:, 0]] - mesh.xyz[mesh.E.uv[:, 1]], axis=1))
    return LY.build_tables(stack, layer, omega, 1e-3 * edge, span, lo[2], hi[2])


def final_matrix(a: Assembled) -> np.ndarray:
    """Dense Z of Eq. finalsystem (rows: external EFIE, internal EFIE, external continuity)."""
    m = a.mesh
    ne, nt, no = m.ne, m.nt, m.nobj
    D, B, F = m.D(), m.B(), m.F()
    nq = nt - no
    Y11 = sla.block_diag(*[b['Y11'] for b in a.blocks])
    Y21 = sla.block_diag(*[b['Y21'] for b in a.blocks])
    LA = sla.block_diag(*[b['LA'] for b in a.blocks])
    LP = sla.block_diag(*[b['LP'] for b in a.blocks])
    K = sla.block_diag(*[b['K'] for b in a.blocks])
    DtLPmB = D.T @ a.LPm @ B
    C1 = a.Ix - (a.LAm @ Y11 - DtLPmB @ Y21)
    C2 = -(F @ D @ Y11 - a.k0 ** 2 * Y21)
    Z = np.block([
        [a.LAm, C1, DtLPmB],
        [LA, -K, D.T @ LP @ B],
        [F @ D, C2, a.k0 ** 2 * np.eye(nq)],
    ])
    return Z


def rhs(a: Assembled, khat=(0, 0, -1), pol=(1, 0, 0), E0=1.0):
    m = a.mesh
    b = np.zeros(2 * m.ne + m.nt - m.nobj, dtype=complex)
    if getattr(a, "layered", None):
        from . import layered as LY
        from .fill import ETA0
        from . import quadrature as Q
        stack, layer, _ = a.layered
        # the incident wave of the stack (oblique incidence from the upper half-space)
        A = m.xyz[m.tri]
        rq = Q.points(A)
        wq = Q.weights(m.area)
        Einc = LY.incident_field(stack, layer, a.k0 * C0, khat, pol, rq.reshape(-1, 3), E0)
        Einc = Einc.reshape(rq.shape) / ETA0
        for i in range(3):
            fi = (rq - A[:, i][:, None, :]) * (m.E.tri_sign[:, i] / (2 * m.area))[:, None, None]
            np.add.at(b, m.E.tri_edge[:, i], np.einsum('tq,tqd,tqd->t', wq, fi, Einc))
        return b
    b[:m.ne] = plane_wave(m, a.k0, khat, pol, E0)
    return b


def split(a: Assembled, x):
    m = a.mesh
    return x[:m.ne], x[m.ne:2 * m.ne], x[2 * m.ne:]


def j_delta(a: Assembled, x):
    """RWG coefficients of j k0 J_Delta = j k0 (H - H_eq) (Eqs. diffsourcesdis, invAEFIEeqvdis)."""
    j, e, _ = split(a, x)
    out = j.copy()
    for o, b in enumerate(a.blocks):
        e0, e1 = a.mesh.edge_range[o]
        out[e0:e1] -= b['Y11'] @ e[e0:e1]
    return out


def solve(a: Assembled, b):
    return sla.lu_solve(sla.lu_factor(a.Z), b)
