"""Layered-medium (stratified background) Green's function of the external
problem (Sec. II-C, "dyadic multilayer Green's function"; Sec. IV: quasistatic
part extracted and added back analytically, Sommerfeld integrals for the rest,
interpolation tables), restated from transmission-line theory for source and
observation points in the same layer l.  Plain numpy, FP64.  TEST INFRASTRUCTURE.

Spectral domain (k_rho), time convention exp(+j w t), k_z = sqrt(k^2 - k_rho^2)
with Im k_z <= 0.  TM (e) and TE (h) lines: Z^e = k_z/(w eps), Z^h = w mu/k_z.
In layer l (interfaces z_b < z_u, thickness d, voltage reflection Gu looking up,
Gd looking down, D = 1 - Gu Gd exp(-2 j k_z d)) with E0 = exp(-j k_z |z - z'|),
E1 = exp(-j k_z (2 z_u - z - z')), E2 = exp(-j k_z (z + z' - 2 z_b)),
E3 = exp(-j k_z (2d + z - z')), E4 = exp(-j k_z (2d - z + z')):

  V_i = Z/2 [E0 + (Gu E1 + Gd E2 + Gu Gd (E3 + E4))/D]         (shunt current source)
  I_v = 1/(2Z) [E0 + (-Gu E1 - Gd E2 + Gu Gd (E3 + E4))/D]      (series voltage source)
  I_i = 1/2 [sgn(z - z') E0 + (-Gu E1 + Gd E2 + Gu Gd (E3 - E4))/D]
  V_v = 1/2 [sgn(z - z') E0 + (Gu E1 - Gd E2 + Gu Gd (E3 - E4))/D]

Mixed-potential form E = -j w A - grad phi, A = G^A * J, phi = K^phi * rho, exact
for source and observer in one layer (matching the spectral TM/TE fields of
horizontal and vertical current elements):

  g_xx = V_i^h / (j w)                       (x x and y y)
  g_zu = j (mu / k_rho) (I_i^e - I_i^h)       (z component of A from the current along k_rho)
  g_uz = j (mu / k_rho) (V_v^e - V_v^h)       (component along k_rho of A from a z current)
  g_zz = [mu (k_rho^2 - k_z^2) / (eps k_rho^2) I_v^e + (w^2 mu^2 / k_rho^2) I_v^h] / (j w)
  k_phi = (j w / k_rho^2) (V_i^e - V_i^h)

and in space, with S_n[f](rho) = 1/(2 pi) int_0^inf f J_n(k_rho rho) k_rho dk_rho:
G_xx = S0[g_xx], G_z-rho = -j S1[g_zu], G_rho-z = -j S1[g_uz], G_zz = S0[g_zz],
K^phi = S0[k_phi];  G^A = G_xx (xx + yy) + z rhohat G_z-rho + rhohat z G_rho-z + z z G_zz,
rhohat = (rho_obs - rho_src)/|rho_obs - rho_src|.  Normalised as the operators of the
paper (L^A_m kernel G^A/mu0, L^phi_m kernel eps0 K^phi) every kernel reduces to mu_r G
and G/eps_r in a homogeneous medium.

Extraction: the direct term (first column) is the homogeneous kernel of layer l;
the quasistatic images of the two adjacent interfaces, with the k_rho -> infinity
limits of the reflection coefficients (Gu_inf, Gd_inf), are added analytically:
  xx: mu_r [Gu_h G(R1) + Gd_h G(R2)],  phi: [Gu_e G(R1) + Gd_e G(R2)] / eps_r,
  zz: mu_r [(Gu_h - 2 Gu_e) G(R1) + (Gd_h - 2 Gd_e) G(R2)],
with G(R) = exp(-j k_l R)/(4 pi R), R1 = |(rho, 2 z_u - z - z')|, R2 = |(rho, z + z' - 2 z_b)|.
The remainder is the sum of a part depending on (rho, z + z') (single reflections)
and a part depending on (rho, z - z') (double reflections), tabulated separately.
"""
from __future__ import annotations

import functools
from dataclasses import dataclass

import numpy as np
from scipy.special import jv

from .fill import C0, EPS0, MU0
from . import quadrature as Q

COMPONENTS = ("xx", "phi", "zz", "zr", "rz")   # zr = G_z-rho, rz = G_rho-z
ODD_IN_D = {"zr": True, "rz": True}


@dataclass
class Stack:
    """Layers top to bottom: (eps_r, mu_r, sigma, thickness); bottom 'halfspace' or 'pec'.

    Layer 0 is the upper half-space above z_top.  With bottom == 'halfspace' the last
    layer is a half-space, otherwise every layer below layer 0 is finite and a PEC
    lies under the last one.
    """
    layers: list
    z_top: float = 0.0
    bottom: str = "halfspace"

    def bounds(self, i):
        """(z_b, z_u) of layer i (+-inf for half-spaces)."""
        z = self.z_top
        if i == 0:
            return z, np.inf
        for j in range(1, i):
            z -= self.layers[j][3]
        last_half = self.bottom == "halfspace" and i == len(self.layers) - 1
        return (-np.inf if last_half else z - self.layers[i][3]), z

    def layer_of(self, z):
        for i in range(len(self.layers)):
            zb, zu = self.bounds(i)
            if zb < z < zu:
                return i
        raise ValueError("point on an interface or below the PEC")

    def eps(self, i, omega):
        e, m, s, _ = self.layers[i]
        return e - 1j * s / (omega * EPS0)

    def mu(self, i):
        return self.layers[i][1]


def kz_of(k, kr):
    kz = np.sqrt(k * k - kr * kr + 0j)
    return np.where(kz.imag > 0, -kz, kz)


def reflections(stack, l, omega, kr):
    """Generalised voltage reflection coefficients (Gu_e, Gu_h, Gd_e, Gd_h) seen from layer l."""
    k0 = omega / C0
    L = len(stack.layers)
    Ze, Zh, kz, d = [], [], [], []
    for i in range(L):
        eps, mu = stack.eps(i, omega), stack.mu(i)
        k = k0 * np.sqrt(eps * mu)
        q = kz_of(k, kr)
        kz.append(q)
        Ze.append(q / (omega * EPS0 * eps))
        Zh.append(omega * MU0 * mu / q)
        d.append(stack.layers[i][3])

    def fres(Z, i, j):  # wave in layer i hitting layer j
        return (Z[j] - Z[i]) / (Z[j] + Z[i])

    out = []
    for Z in (Ze, Zh):
        # looking up: up[i] at the top interface of layer i
        up = np.zeros_like(kr, dtype=complex)
        for i in range(1, l + 1):
            f = fres(Z, i, i - 1)
            if i - 1 == 0:
                up = f
            else:
                ph = up * np.exp(-2j * kz[i - 1] * d[i - 1])
                up = (f + ph) / (1 + f * ph)
        # looking down: down[i] at the bottom interface of layer i
        last = L - 1
        if stack.bottom == "pec":
            down = -np.ones_like(kr, dtype=complex)
        else:
            down = np.zeros_like(kr, dtype=complex)
        for i in range(last - 1, l - 1, -1):
            f = fres(Z, i, i + 1)
            if i + 1 == last and stack.bottom == "halfspace":
                down = f
            else:
                ph = down * np.exp(-2j * kz[i + 1] * d[i + 1])
                down = (f + ph) / (1 + f * ph)
        if l == L - 1:
            down = -np.ones_like(kr, dtype=complex) if stack.bottom == "pec" else np.zeros_like(kr, dtype=complex)
        if l == 0:
            up = np.zeros_like(kr, dtype=complex)
        out.append((up, down))
    (Gue, Gde), (Guh, Gdh) = out
    return Gue, Guh, Gde, Gdh


def static_reflections(stack, l, omega):
    """k_rho -> infinity limits (Gu_e, Gu_h, Gd_e, Gd_h): adjacent-interface Fresnel values."""
    L = len(stack.layers)
    el, ml = stack.eps(l, omega), stack.mu(l)

    def pair(j):
        ej, mj = stack.eps(j, omega), stack.mu(j)
        # Z^e ~ 1/eps, Z^h ~ mu at large k_rho
        return (el - ej) / (el + ej), (mj - ml) / (mj + ml)

    gue = guh = gde = gdh = 0.0
    if l > 0:
        gue, guh = pair(l - 1)
    if l < L - 1:
        gde, gdh = pair(l + 1)
    elif stack.bottom == "pec":
        gde = gdh = -1.0
    return complex(gue), complex(guh), complex(gde), complex(gdh)


def spectral(stack, l, omega, kr, s=None, dd=None, part="full", z=None, zp=None):
    """Normalised spectral kernels {component: array over kr}.

    part = 'full' (needs z, zp), 'A' (single reflections minus quasistatic images, needs
    s = z + z'), 'B' (double reflections, needs dd = z - z').
    """
    k0 = omega / C0
    eps_r, mu_r = stack.eps(l, omega), stack.mu(l)
    k = k0 * np.sqrt(eps_r * mu_r)
    kz = kz_of(k, kr)
    Ze = kz / (omega * EPS0 * eps_r)
    Zh = omega * MU0 * mu_r / kz
    zb, zu = stack.bounds(l)
    dl = zu - zb
    Gue, Guh, Gde, Gdh = reflections(stack, l, omega, kr)
    top, bot = np.isfinite(zu), np.isfinite(zb)
    D_e = 1 - Gue * Gde * (np.exp(-2j * kz * dl) if top and bot else 0)
    D_h = 1 - Guh * Gdh * (np.exp(-2j * kz * dl) if top and bot else 0)
    zero = np.zeros_like(kr, dtype=complex)
    if part == "full":
        s_, d_ = z + zp, z - zp
    elif part == "A":
        s_, d_ = s, None
    else:
        s_, d_ = None, dd
    E0 = np.exp(-1j * kz * abs(d_)) if part == "full" else zero
    sg = np.sign(d_) if part == "full" else 0.0
    E1 = np.exp(-1j * kz * (2 * zu - s_)) if (top and part in ("full", "A")) else zero
    E2 = np.exp(-1j * kz * (s_ - 2 * zb)) if (bot and part in ("full", "A")) else zero
    if top and bot and part in ("full", "B"):
        E3 = np.exp(-1j * kz * (2 * dl + d_))
        E4 = np.exp(-1j * kz * (2 * dl - d_))
    else:
        E3 = E4 = zero

    def lines(Z, Gu, Gd, D):
        Vi = Z / 2 * (E0 + (Gu * E1 + Gd * E2 + Gu * Gd * (E3 + E4)) / D)
        Iv = 1 / (2 * Z) * (E0 + (-Gu * E1 - Gd * E2 + Gu * Gd * (E3 + E4)) / D)
        Ii = 0.5 * (sg * E0 + (-Gu * E1 + Gd * E2 + Gu * Gd * (E3 - E4)) / D)
        Vv = 0.5 * (sg * E0 + (Gu * E1 - Gd * E2 + Gu * Gd * (E3 - E4)) / D)
        return Vi, Iv, Ii, Vv

    Vie, Ive, Iie, Vve = lines(Ze, Gue, Gde, D_e)
    Vih, Ivh, Iih, Vvh = lines(Zh, Guh, Gdh, D_h)
    jw = 1j * omega
    out = {
        "xx": Vih / (jw * MU0),
        "phi": EPS0 * jw / kr ** 2 * (Vie - Vih),
        "zz": (mu_r * (kr ** 2 - kz ** 2) / (EPS0 * eps_r * kr ** 2) * Ive
               + omega ** 2 * MU0 * mu_r ** 2 / kr ** 2 * Ivh) / jw,
        "zr": 1j * mu_r / kr * (Iie - Iih),
        "rz": 1j * mu_r / kr * (Vve - Vvh),
    }
    if part == "A":
        gue, guh, gde, gdh = static_reflections(stack, l, omega)
        g = 1 / (2j * kz)
        out["xx"] = out["xx"] - mu_r * (guh * E1 + gdh * E2) * g
        out["phi"] = out["phi"] - (gue * E1 + gde * E2) * g / eps_r
        out["zz"] = out["zz"] - mu_r * ((guh - 2 * gue) * E1 + (gdh - 2 * gde) * E2) * g
        # z-rho / rho-z: the static (k -> 0, k_rho -> infinity) single reflections, whose
        # S1 transform is closed-form (static_zr): exp(-k_rho zeta) in place of E1, E2
        X1 = np.exp(-kr * (2 * zu - s_)) if top else zero
        X2 = np.exp(-kr * (s_ - 2 * zb)) if bot else zero
        cu, cd = gue - guh, gde - gdh
        out["zr"] = out["zr"] - 0.5j * mu_r / kr * (-cu * X1 + cd * X2)
        out["rz"] = out["rz"] - 0.5j * mu_r / kr * (cu * X1 - cd * X2)
    return out


# ----------------------------------------------------------------------------- Sommerfeld integration
def sommerfeld_nodes(stack, l, omega, rho_max, zeta_min, n_ellipse=400, per_panel=16):
    """Nodes and weights (complex) of int_0^inf f(kr) dkr: an elliptic arc into the first
    quadrant over [0, a] (above every branch point and pole), then Gauss-Legendre panels on
    the real axis until exp(-kr zeta_min) < 1e-14."""
    k0 = omega / C0
    kmax = max(abs((k0 * np.sqrt(stack.eps(i, omega) * stack.mu(i))).real) for i in range(len(stack.layers)))
    a = max(1.5 * kmax, 2.0 * k0)
    b = min(0.5 * a, 2.0 / rho_max)
    x, w = np.polynomial.legendre.leggauss(n_ellipse)
    t = 0.5 * np.pi * (x + 1)
    wt = 0.5 * np.pi * w
    kr_e = 0.5 * a * (1 - np.cos(t)) + 1j * b * np.sin(t)
    dk_e = (0.5 * a * np.sin(t) + 1j * b * np.cos(t)) * wt
    kend = a + 32.0 / zeta_min
    width = min(np.pi / rho_max, (kend - a) / 4)
    npan = int(np.ceil((kend - a) / width))
    xp, wp = np.polynomial.legendre.leggauss(per_panel)
    edges = a + width * np.arange(npan + 1)
    mid = 0.5 * (edges[:-1] + edges[1:])
    kr_t = (mid[:, None] + 0.5 * width * xp[None, :]).ravel()
    dk_t = np.tile(0.5 * width * wp, npan).astype(complex)
    return np.concatenate([kr_e, kr_t]), np.concatenate([dk_e, dk_t])


def transform(values, nodes, weights, rho, order):
    """S_n[f](rho) for f sampled at the nodes: (len(rho), ...) ."""
    J = jv(order, np.outer(rho, nodes))                                  # (nrho, nnodes)
    return (J * (weights * nodes)[None, :]) @ values / (2 * np.pi)


ORDER = {"xx": 0, "phi": 0, "zz": 0, "zr": 1, "rz": 1}


def spatial_full(stack, l, omega, rho, z, zp, zeta_min=None):
    """Full spatial kernels by direct Sommerfeld integration (no extraction) at rho (array)."""
    zb, zu = stack.bounds(l)
    zmin = abs(z - zp) if zeta_min is None else zeta_min
    nodes, w = sommerfeld_nodes(stack, l, omega, max(np.max(rho), 1e-12), zmin)
    sp = spectral(stack, l, omega, nodes, part="full", z=z, zp=zp)
    out = {}
    for c in COMPONENTS:
        v = transform(sp[c][:, None], nodes, w, np.atleast_1d(rho), ORDER[c])[:, 0]
        out[c] = -1j * v if ORDER[c] == 1 else v
    return out


# ----------------------------------------------------------------------------- tables
@dataclass
class Tables:
    l: int
    omega: float
    rho: np.ndarray        # (nr,) log-spaced
    s: np.ndarray          # (ns,) z + z'
    d: np.ndarray          # (nd,) |z - z'| >= 0
    A: dict                # component -> (nr, ns)
    B: dict                # component -> (nr, nd)


def build_tables(stack, l, omega, rho_min, rho_max, zmin, zmax, nr=256, ns=128, nd=128):
    zb, zu = stack.bounds(l)
    rho = np.exp(np.linspace(np.log(rho_min), np.log(rho_max), nr))
    s = np.linspace(2 * zmin, 2 * zmax, ns)
    d = np.linspace(0.0, zmax - zmin, nd)
    zetas = []
    if np.isfinite(zu):
        zetas.append(2 * zu - 2 * zmax)
    if np.isfinite(zb):
        zetas.append(2 * zmin - 2 * zb)
    # Objects may rest on an interface (z + z' - 2 z_b = 0 there): the Sommerfeld tail
    # is then cut where exp(-k_rho zeta_floor) < 1e-14, zeta_floor = 1/16 of the
    # objects' height (the remainder decays algebraically once the static images,
    # z-rho / rho-z included, are out; the cut costs ~1e-4 of the remainder).
    zeta_floor = (zmax - zmin) / 16 if zmax > zmin else 1e-3 * rho_max
    zeta_a = max(min(zetas), zeta_floor) if zetas else 1.0
    A, B = {}, {}
    nodes, w = sommerfeld_nodes(stack, l, omega, rho_max, zeta_a)
    vals = {c: np.stack([spectral(stack, l, omega, nodes, s=si, part="A")[c] for si in s], axis=1) for c in COMPONENTS}
    for c in COMPONENTS:
        v = transform(vals[c], nodes, w, rho, ORDER[c])
        A[c] = -1j * v if ORDER[c] == 1 else v
    if np.isfinite(zu) and np.isfinite(zb):
        zeta_b = max(2 * (zu - zb) - (zmax - zmin), zeta_floor)
        nodes, w = sommerfeld_nodes(stack, l, omega, rho_max, zeta_b)
        vals = {c: np.stack([spectral(stack, l, omega, nodes, dd=di, part="B")[c] for di in d], axis=1)
                for c in COMPONENTS}
        for c in COMPONENTS:
            v = transform(vals[c], nodes, w, rho, ORDER[c])
            B[c] = -1j * v if ORDER[c] == 1 else v
    else:
        for c in COMPONENTS:
            B[c] = np.zeros((nr, nd), dtype=complex)
    return Tables(l, omega, rho, s, d, A, B)


def _bilinear(tab, xg, yg, x, y):
    """Bilinear interpolation on a uniform grid in x (here log rho) and y; clamped."""
    nx, ny = len(xg), len(yg)
    fx = np.clip((x - xg[0]) / (xg[-1] - xg[0]) * (nx - 1), 0, nx - 1 - 1e-12)
    fy = np.clip((y - yg[0]) / (yg[-1] - yg[0]) * (ny - 1), 0, ny - 1 - 1e-12) if ny > 1 else np.zeros_like(x)
    ix, iy = np.floor(fx).astype(int), np.floor(fy).astype(int)
    tx, ty = fx - ix, fy - iy
    iy1 = np.minimum(iy + 1, ny - 1)
    return ((1 - tx) * (1 - ty) * tab[ix, iy] + tx * (1 - ty) * tab[ix + 1, iy]
            + (1 - tx) * ty * tab[ix, iy1] + tx * ty * tab[ix + 1, iy1])


def remainder(T: Tables, rho, z, zp):
    """Interpolated remainder kernels {component: array} at (rho, z, z').

    Below the first table point the S0 kernels keep their value at rho_min, and the
    S1 kernels (z-rho, rho-z), which vanish linearly at rho = 0 (J1(0) = 0), are
    scaled by rho / rho_min."""
    lr = np.log(np.maximum(rho, T.rho[0]))
    lg = np.log(T.rho)
    s = z + zp
    dd = z - zp
    lin = np.minimum(rho / T.rho[0], 1.0)
    out = {}
    for c in COMPONENTS:
        a = _bilinear(T.A[c], lg, T.s, lr, s)
        b = _bilinear(T.B[c], lg, T.d, lr, np.abs(dd))
        out[c] = a + (np.sign(dd) * b if ODD_IN_D.get(c) else b)
        if ORDER[c] == 1:
            out[c] = out[c] * lin
    return out


def images(stack, l, omega, rho, z, zp, use_top=1.0, use_bot=1.0):
    """Quasistatic image kernels: {xx, phi, zz} spherical waves of layer l from the
    image points, {zr, rz} the static z-rho / rho-z images (static_zr).  use_top /
    use_bot (0 or 1, broadcastable) drop one interface's images where they are
    integrated apart (pairs touching through that interface); a coincident image
    point (R = 0) contributes 0 here."""
    k0 = omega / C0
    eps_r, mu_r = stack.eps(l, omega), stack.mu(l)
    k = k0 * np.sqrt(eps_r * mu_r)
    zb, zu = stack.bounds(l)
    gue, guh, gde, gdh = static_reflections(stack, l, omega)

    def G(zeta):
        R = np.sqrt(rho ** 2 + zeta ** 2)
        with np.errstate(invalid="ignore", divide="ignore"):
            return np.where(R > 0, np.exp(-1j * k * R) / (4 * np.pi * np.where(R > 0, R, 1.0)), 0.0)
    G1 = use_top * G(2 * zu - z - zp) if np.isfinite(zu) else 0.0
    G2 = use_bot * G(z + zp - 2 * zb) if np.isfinite(zb) else 0.0
    F1 = use_top * static_zr(rho, 2 * zu - z - zp) if np.isfinite(zu) else 0.0
    F2 = use_bot * static_zr(rho, z + zp - 2 * zb) if np.isfinite(zb) else 0.0
    cu, cd = gue - guh, gde - gdh
    return {"xx": mu_r * (guh * G1 + gdh * G2), "phi": (gue * G1 + gde * G2) / eps_r,
            "zz": mu_r * ((guh - 2 * gue) * G1 + (gdh - 2 * gde) * G2),
            "zr": mu_r * (-cu * F1 + cd * F2), "rz": mu_r * (cu * F1 - cd * F2)}


def static_zr(rho, zeta):
    """1/(4 pi) int_0^inf exp(-k zeta) J1(k rho) dk = (1 - zeta/R) / (4 pi rho) = rho / (4 pi R (R + zeta)),
    R = sqrt(rho^2 + zeta^2), zeta >= 0: the spatial form of the static z-rho image (0 at R = 0)."""
    rho = np.asarray(rho, float)
    zeta = np.asarray(zeta, float)
    R = np.sqrt(rho * rho + zeta * zeta)
    den = R * (R + zeta)
    with np.errstate(invalid="ignore", divide="ignore"):
        return np.where(den > 0, rho / np.where(den > 0, den, 1.0), 0.0) / (4 * np.pi)


# ----------------------------------------------------------------------------- fill of L^A_m, L^phi_m
def fill_reflected(mesh, stack, l, omega, T: Tables, tris):
    """Reflected part (images + tabulated remainder) of L^A_m and L^phi_m over ``tris``,
    by the 6 x 6 product rule, except the images of an interface for pairs of
    triangles that touch through it (touch_image): the remainder is smooth, and an
    image is singular only where a triangle meets the mirror of the other, i.e. at a
    shared vertex on that interface."""
    tris = np.asarray(tris)
    e_of = mesh.E.tri_edge
    edges = np.unique(e_of[tris])
    eidx = -np.ones(mesh.ne, dtype=np.int64)
    eidx[edges] = np.arange(len(edges))
    tidx = -np.ones(mesh.nt, dtype=np.int64)
    tidx[tris] = np.arange(len(tris))
    LA = np.zeros((len(edges), len(edges)), dtype=complex)
    LP = np.zeros((len(tris), len(tris)), dtype=complex)
    ta_all = np.repeat(tris, len(tris))
    tb_all = np.tile(tris, len(tris))
    for c0 in range(0, len(ta_all), 4096):
        ta, tb = ta_all[c0:c0 + 4096], tb_all[c0:c0 + 4096]
        A, B = mesh.xyz[mesh.tri[ta]], mesh.xyz[mesh.tri[tb]]
        rq, rs = Q.points(A), Q.points(B)
        wq, ws = Q.weights(mesh.area[ta]), Q.weights(mesh.area[tb])
        fa = (rq[:, :, None, :] - A[:, None, :, :]) * (mesh.E.tri_sign[ta] / (2 * mesh.area[ta][:, None]))[:, None, :, None]
        fb = (rs[:, :, None, :] - B[:, None, :, :]) * (mesh.E.tri_sign[tb] / (2 * mesh.area[tb][:, None]))[:, None, :, None]
        dv = rq[:, :, None, :] - rs[:, None, :, :]                      # (P, q, s, 3)
        rho = np.sqrt(dv[..., 0] ** 2 + dv[..., 1] ** 2)
        z = np.broadcast_to(rq[:, :, None, 2], rho.shape)
        zp = np.broadcast_to(rs[:, None, :, 2], rho.shape)
        t_top, t_bot = touch_masks(mesh, stack, l, ta, tb)
        im = images(stack, l, omega, rho, z, zp, use_top=(~t_top)[:, None, None], use_bot=(~t_bot)[:, None, None])
        rm = remainder(T, rho, z, zp)
        gxx = im["xx"] + rm["xx"]
        gzz = im["zz"] + rm["zz"]
        kphi = im["phi"] + rm["phi"]
        with np.errstate(invalid="ignore", divide="ignore"):
            rh = np.where(rho[..., None] > 0, dv[..., :2] / rho[..., None], 0.0)   # (P, q, s, 2)
        W = wq[:, :, None] * ws[:, None, :]
        # f_m . G . f_n = G_xx f_m,t . f_n,t + G_zz f_m,z f_n,z + G_zr f_m,z (rhohat . f_n) + G_rz (rhohat . f_m) f_n,z
        fa_t, fa_z = fa[..., :2], fa[..., 2]                              # (P, q, i, 2), (P, q, i)
        fb_t, fb_z = fb[..., :2], fb[..., 2]
        t_xx = np.einsum('pqs,pqia,psja->pij', W * gxx, fa_t, fb_t)
        t_zz = np.einsum('pqs,pqi,psj->pij', W * gzz, fa_z, fb_z)
        rhf_b = np.einsum('pqsa,psja->pqsj', rh, fb_t)                   # rhohat . f_n,t
        rhf_a = np.einsum('pqsa,pqia->pqsi', rh, fa_t)                   # rhohat . f_m,t
        t_zr = np.einsum('pqs,pqi,pqsj->pij', W * (im["zr"] + rm["zr"]), fa_z, rhf_b)
        t_rz = np.einsum('pqs,pqsi,psj->pij', W * (im["rz"] + rm["rz"]), rhf_a, fb_z)
        la = t_xx + t_zz + t_zr + t_rz
        lp = np.einsum('pqs->p', W * kphi) / (mesh.area[ta] * mesh.area[tb])
        for plane, tm in (("top", t_top), ("bottom", t_bot)):
            if tm.any():
                i = np.nonzero(tm)[0]
                la_t, lp_t = touch_image(mesh, stack, l, omega, ta[i], tb[i], plane)
                la[i] += la_t
                lp[i] += lp_t
        rows = eidx[e_of[ta]][:, :, None] * np.ones((1, 1, 3), dtype=np.int64)
        cols = eidx[e_of[tb]][:, None, :] * np.ones((1, 3, 1), dtype=np.int64)
        np.add.at(LA, (rows.ravel(), cols.ravel()), la.ravel())
        np.add.at(LP, (tidx[ta], tidx[tb]), lp)
    return LA, LP


def plane_wave_normal(stack, l, omega, E0=1.0):
    """Normal incidence from the upper half-space: incident E = x E0 exp(+j k0 z).

    In layer l the transverse field is a exp(+j k (z - z_ref)) + c exp(-j k (z - z_ref))
    (down- and up-going waves) with z_ref the top of the layer (z_top for layer 0);
    returns (a, c, k, z_ref).  Transfer through the stack: at the bottom of layer i
    the up/down ratio is the normal-incidence reflection coefficient looking down,
    and E_x is continuous across each interface."""
    k0 = omega / C0
    L = len(stack.layers)
    ks = [k0 * np.sqrt(stack.eps(i, omega) * stack.mu(i)) for i in range(L)]
    eta = [np.sqrt(stack.mu(i) / stack.eps(i, omega)) for i in range(L)]
    finite = [np.isfinite(stack.bounds(i)[0]) and i > 0 for i in range(L)]
    down = [0j] * L
    down[L - 1] = (-1.0 + 0j) if stack.bottom == "pec" else 0j
    for i in range(L - 2, -1, -1):
        f = (eta[i + 1] - eta[i]) / (eta[i + 1] + eta[i])
        ph = down[i + 1] * np.exp(-2j * ks[i + 1] * stack.layers[i + 1][3]) if finite[i + 1] else 0j
        down[i] = (f + ph) / (1 + f * ph)
    a = E0 * np.exp(1j * k0 * stack.z_top)                     # layer 0, referenced at z_top
    c = a * down[0]
    v = a + c                                                    # E_x at z_top
    for i in range(1, l + 1):
        d = stack.layers[i][3]
        gtop = down[i] * np.exp(-2j * ks[i] * d) if finite[i] else 0j
        a = v / (1 + gtop)
        c = a * gtop
        if finite[i]:
            v = a * np.exp(-1j * ks[i] * d) + c * np.exp(1j * ks[i] * d)
    zref = stack.z_top if l == 0 else stack.bounds(l)[1]
    return a, c, ks[l], zref


def _oblique_lines(stack, omega, kt_abs, pol_type):
    """Per layer: k_z, line impedance and the reflection coefficient looking down at
    the layer's bottom (a transmission line in z for the transverse E of one
    polarisation; pol_type 'TE': Z = w mu / k_z, 'TM': Z = k_z / (w eps))."""
    k0 = omega / C0
    L = len(stack.layers)
    kz, Z, d, finite = [], [], [], []
    for i in range(L):
        eps, mu = stack.eps(i, omega), stack.mu(i)
        q = complex(kz_of(k0 * np.sqrt(eps * mu), kt_abs))
        kz.append(q)
        Z.append(omega * MU0 * mu / q if pol_type == "TE" else q / (omega * EPS0 * eps))
        d.append(stack.layers[i][3])
        finite.append(i > 0 and (stack.bottom == "pec" or i < L - 1))
    down = [0j] * L
    down[L - 1] = -1.0 + 0j if stack.bottom == "pec" else 0j
    for i in range(L - 2, -1, -1):
        f = (Z[i + 1] - Z[i]) / (Z[i + 1] + Z[i])
        ph = down[i + 1] * np.exp(-2j * kz[i + 1] * d[i + 1]) if finite[i + 1] else 0j
        down[i] = (f + ph) / (1 + f * ph)
    return kz, Z, d, finite, down


def plane_wave_oblique(stack, omega, khat, pol, E0=1.0):
    """Plane wave incident from the upper half-space on the stack, in every layer.

    Incident field E_inc = pol E0 exp(-j k0 khat . r) (khat_z < 0, pol . khat = 0).
    The transverse wavevector kt = k0 (khat_x, khat_y) is the same in every layer;
    with rho = kt / |kt| (for normal incidence, the transverse direction of pol)
    and phi = z x rho, the field splits into a TE part (E along phi) and a TM
    part (H along phi).  For each, the transverse E component V(z) is a
    transmission line in z: in layer i, V = a exp(+j k_z (z - zref)) + c exp(-j k_z
    (z - zref)) (down- and up-going waves), zref the layer's top (z_top for the
    upper half-space), the ratio c / a at a layer's bottom the reflection
    coefficient looking down, and V continuous across each interface.  In layer i
    the field is
        E = exp(-j kt . r) [phi V_TE + rho V_TM + z (|kt| / k_z) (a_TM e^{+} - c_TM e^{-})],
    the z part from div E = 0 for each of the two TM waves.  Returns a list over
    the layers of dicts {a_te, c_te, a_tm, c_tm, kz, zref} and the common
    {kt (2,), krho, rho (3,), phi (3,)}."""
    khat = np.asarray(khat, float)
    pol = np.asarray(pol, complex)
    k0 = omega / C0
    kt = k0 * khat[:2]
    krho = float(np.hypot(kt[0], kt[1]))
    if krho > 1e-12 * k0:
        rho = np.array([kt[0] / krho, kt[1] / krho, 0.0])
    else:
        pt = np.array([pol[0], pol[1]])
        n = np.linalg.norm(pt)
        rho = np.array([pt[0].real, pt[1].real, 0.0]) / n if n > 0 else np.array([1.0, 0.0, 0.0])
        rho = rho / np.linalg.norm(rho)
    phi = np.cross([0.0, 0.0, 1.0], rho)
    L = len(stack.layers)
    out = [dict() for _ in range(L)]
    for ptype, key in (("TE", "te"), ("TM", "tm")):
        kz, Z, d, finite, down = _oblique_lines(stack, omega, krho, ptype)
        v0 = E0 * (pol @ phi if ptype == "TE" else pol @ rho)
        a = v0 * np.exp(1j * kz[0] * stack.z_top)      # down-going amplitude at z_top
        c = a * down[0]
        out[0]["a_" + key], out[0]["c_" + key], out[0]["kz"], out[0]["zref"] = a, c, kz[0], stack.z_top
        v = a + c                                        # V at z_top
        z = stack.z_top
        for i in range(1, L):
            gtop = down[i] * np.exp(-2j * kz[i] * d[i]) if finite[i] else 0j
            a = v / (1 + gtop)
            c = a * gtop
            out[i]["a_" + key], out[i]["c_" + key], out[i]["kz"], out[i]["zref"] = a, c, kz[i], z
            if finite[i]:
                v = a * np.exp(-1j * kz[i] * d[i]) + c * np.exp(1j * kz[i] * d[i])
                z -= d[i]
    return out, dict(kt=kt, krho=krho, rho=rho, phi=phi)


def incident_field(stack, l, omega, khat, pol, r, E0=1.0):
    """The field of plane_wave_oblique in layer l at points r (n, 3) -> (n, 3) complex."""
    layers, g = plane_wave_oblique(stack, omega, khat, pol, E0)
    c = layers[l]
    r = np.atleast_2d(r)
    zeta = r[:, 2] - c["zref"]
    ep, em = np.exp(1j * c["kz"] * zeta), np.exp(-1j * c["kz"] * zeta)
    vte = c["a_te"] * ep + c["c_te"] * em
    vtm = c["a_tm"] * ep + c["c_tm"] * em
    ez = (g["krho"] / c["kz"]) * (c["a_tm"] * ep - c["c_tm"] * em)
    lat = np.exp(-1j * (r[:, 0] * g["kt"][0] + r[:, 1] * g["kt"][1]))
    return lat[:, None] * (g["phi"][None, :] * vte[:, None] + g["rho"][None, :] * vtm[:, None]
                           + np.array([0.0, 0.0, 1.0])[None, :] * ez[:, None])


# ----------------------------------------------------------------------------- objects resting on an interface
DUFFY_N = 16     # Gauss-Legendre points per direction of the Duffy rule (touch_image)


def touch_masks(mesh, stack, l, ta, tb):
    """Pairs (ta[p], tb[p]) touching through the top / bottom interface of layer l:
    they share a vertex that lies on that interface (to 1e-9 of the mesh size)."""
    zb, zu = stack.bounds(l)
    z = mesh.xyz[:, 2]
    tol = 1e-9 * np.ptp(mesh.xyz, axis=0).max()
    out = []
    for zI in (zu, zb):
        if not np.isfinite(zI):
            out.append(np.zeros(len(ta), dtype=bool))
            continue
        on = np.abs(z - zI) <= tol
        va, vb = mesh.tri[ta], mesh.tri[tb]
        share = (va[:, :, None] == vb[:, None, :]) & on[va][:, :, None]
        out.append(share.any(axis=(1, 2)))
    return out[0], out[1]


def closest_point(r, T):
    """The point of triangle T (3, 3) nearest to r (3,)."""
    a, b, c = T
    n = np.cross(b - a, c - a)
    p = r - (r - a) @ n / (n @ n) * n                                  # projection on the plane
    # barycentric coordinates of p
    v0, v1, v2 = b - a, c - a, p - a
    d00, d01, d11, d20, d21 = v0 @ v0, v0 @ v1, v1 @ v1, v2 @ v0, v2 @ v1
    den = d00 * d11 - d01 * d01
    bv = (d11 * d20 - d01 * d21) / den
    bw = (d00 * d21 - d01 * d20) / den
    if bv >= 0 and bw >= 0 and bv + bw <= 1:
        return p
    best, bd = None, np.inf
    for u, v in ((a, b), (b, c), (c, a)):
        t = np.clip((r - u) @ (v - u) / ((v - u) @ (v - u)), 0.0, 1.0)
        q = u + t * (v - u)
        d = np.linalg.norm(r - q)
        if d < bd:
            best, bd = q, d
    return best


@functools.lru_cache(maxsize=8)
def _unit_square_rule(n):
    """n x n Gauss-Legendre points (u, v) and weights on the unit square."""
    x, w = np.polynomial.legendre.leggauss(n)
    x, w = 0.5 * (x + 1), 0.5 * w
    u, v = np.meshgrid(x, x, indexing="ij")
    return u, v, np.outer(w, w)


def duffy_rule(r, T, n=DUFFY_N):
    """Points (M, 3) and weights (M,) over triangle T for kernels singular at the point
    of T nearest to r: T is split at that point Q into (Q, T_i, T_i+1) and each part
    mapped from the unit square by p = Q + u (T_i - Q) + u v (T_i+1 - T_i), dS = 2 a u du dv
    (Duffy, SIAM J. Numer. Anal. 19, 1982), n x n Gauss-Legendre points; parts of
    zero area are dropped."""
    Qp = closest_point(r, T)
    u, v, wu = _unit_square_rule(n)
    full = np.linalg.norm(np.cross(T[1] - T[0], T[2] - T[0]))
    pts, wts = [], []
    for i in range(3):
        P1, P2 = T[i], T[(i + 1) % 3]
        a2 = np.linalg.norm(np.cross(P1 - Qp, P2 - P1))
        if a2 <= 1e-12 * full:
            continue
        p = Qp + u[..., None] * (P1 - Qp) + (u * v)[..., None] * (P2 - P1)
        pts.append(p.reshape(-1, 3))
        wts.append((a2 * u * wu).ravel())
    return np.concatenate(pts), np.concatenate(wts)


def touch_image(mesh, stack, l, omega, ta, tb, plane):
    """The images of one interface ('top' or 'bottom') of layer l for pairs touching
    through it: (la (P, 3, 3), lp (P,)) added to the product-rule terms without them.

    The image of source point r' in the interface z_I is r'' = (x', y', 2 z_I - z'),
    so an image term integrates over the mirrored source triangle, where the RWG
    keeps its transverse part and flips its z part.  xx, phi, zz: the spherical wave
    G = exp(-j k_l R)/(4 pi R) from r'', with 1/R and R integrated in closed form
    over the mirrored triangle and the rest by its 6 points (the direct term's
    touching rule).  z-rho, rho-z: the static kernel rhohat (1 - zeta/R)/(4 pi rho) =
    (r - r'')_t / (4 pi R (R + zeta)), zeta = |z - z''|, inner integral by duffy_rule
    on the mirrored triangle.  The outer integral is the 6-point rule."""
    from .fill import green_smooth
    from .singular import integrals
    k0 = omega / C0
    eps_r, mu_r = stack.eps(l, omega), stack.mu(l)
    k = k0 * np.sqrt(eps_r * mu_r)
    zb, zu = stack.bounds(l)
    gue, guh, gde, gdh = static_reflections(stack, l, omega)
    if plane == "bottom":
        zI, ge, gh = zb, gde, gdh
        czr = mu_r * (gde - gdh)
    else:
        zI, ge, gh = zu, gue, guh
        czr = -mu_r * (gue - guh)
    crz = -czr
    cxx, czz, cphi = mu_r * gh, mu_r * (gh - 2 * ge), ge / eps_r
    xyz, tri = mesh.xyz, mesh.tri
    A = xyz[tri[ta]]
    Bm = xyz[tri[tb]].copy()
    Bm[..., 2] = 2 * zI - Bm[..., 2]
    P = len(ta)
    rq, rs = Q.points(A), Q.points(Bm)
    wq, ws = Q.weights(mesh.area[ta]), Q.weights(mesh.area[tb])
    sa = mesh.E.tri_sign[ta] / (2 * mesh.area[ta])[:, None]             # (P, 3)
    sb = mesh.E.tri_sign[tb] / (2 * mesh.area[tb])[:, None]
    fa = (rq[:, :, None, :] - A[:, None, :, :]) * sa[:, None, :, None]   # (P, 6, 3i, 3)
    # spherical-wave images: int G and int p G over the mirrored triangle
    R = np.linalg.norm(rq[:, :, None, :] - rs[:, None, :, :], axis=-1)
    Gs = green_smooth(k, R) * ws[:, None, :]
    I0 = Gs.sum(axis=2)                                                  # (P, 6)
    Ip = np.einsum('pqs,psd->pqd', Gs, rs)                               # (P, 6, 3)
    I = integrals(rq.reshape(-1, 3), np.repeat(Bm, 6, axis=0))
    rho = I['rho'].reshape(P, 6, 3)
    inv_r, rr = I['inv_r'].reshape(P, 6), I['r'].reshape(P, 6)
    I0 = I0 + inv_r / (4 * np.pi) - k * k * rr / (8 * np.pi)
    Ip = Ip + (I['p_over_r'].reshape(P, 6, 3) + rho * inv_r[..., None]) / (4 * np.pi) \
        - k * k * (I['p_r'].reshape(P, 6, 3) + rho * rr[..., None]) / (8 * np.pi)
    inner = Ip[:, :, None, :] - Bm[:, None, :, :] * I0[:, :, None, None]   # int (p'' - v''_j) G: (P, 6, 3j, 3)
    la = cxx * np.einsum('pq,pqid,pqjd->pij', wq, fa[..., :2], inner[..., :2]) * sb[:, None, :]
    la = la - czz * np.einsum('pq,pqi,pqj->pij', wq, fa[..., 2], inner[..., 2]) * sb[:, None, :]
    lp = cphi * np.einsum('pq,pq->p', wq, I0) / (mesh.area[ta] * mesh.area[tb])
    # static z-rho / rho-z images by the Duffy rule
    la = la.astype(complex)
    for p in range(P):
        for q in range(6):
            r = rq[p, q]
            pts, wts = duffy_rule(r, Bm[p], DUFFY_N)
            d = r - pts
            Rr = np.linalg.norm(d, axis=1)
            zeta = np.abs(r[2] - pts[:, 2])
            den = Rr * (Rr + zeta)
            Wk = np.where(den[:, None] > 0, d[:, :2] / np.where(den > 0, den, 1.0)[:, None], 0.0) \
                * (wts / (4 * np.pi))[:, None]                              # (M, 2)
            J0 = Wk.sum(axis=0)                                           # (2,)
            J1 = Wk.T @ pts                                               # (2, 3)
            for j in range(3):
                vj = Bm[p, j]
                tj = (J1[0, 0] - vj[0] * J0[0]) + (J1[1, 1] - vj[1] * J0[1])   # int W . (p'' - v''_j)_t
                zj = J1[:, 2] - vj[2] * J0                                      # int W (p'' - v''_j)_z
                for i in range(3):
                    f = fa[p, q, i]
                    la[p, i, j] += wq[p, q] * sb[p, j] * (czr * f[2] * tj - crz * (f[:2] @ zj))
    return la, lp
