"""Closed-form integrals over a flat triangle used by singularity extraction on
self and touching pairs (Sec. II-B; extraction rule: subtract 1/(4 pi R) and
-k^2 R/(8 pi) from G for L, and the static gradient for K-bar).

For an observation point r and a triangle T' with unit normal n (from its vertex
order), write d = n.(r - p1), rho = r - d n (projection) and P = rho' - rho for a
source point r' in T'.  Reducing each surface integral to a contour integral with
the surface divergence theorem in the plane of T' gives, with per edge i (from
p_i to p_i+1): unit vector s_i, outward in-plane normal m_i = s_i x n, end
abscissae s-, s+, distance t0 = (p_i - rho).m_i, R0^2 = t0^2 + d^2, end distances R-, R+,

    f_i   = ln((R+ + s+) / (R- + s-)),
    beta_i = atan(t0 s+ / (R0^2 + |d| R+)) - atan(t0 s- / (R0^2 + |d| R-)),
    Omega = sum beta_i  (solid angle of T' seen from r),

    int 1/R        = sum t0 f - |d| Omega
    int R          = 1/6 sum t0 (s+R+ - s-R- + R0^2 f) + d^2/3 int 1/R
    int P / R      = 1/2 sum m (s+R+ - s-R- + R0^2 f)
    int P R        = 1/3 sum m [(s+R+^3 - s-R-^3)/4 + 3 R0^2 (s+R+ - s-R-)/8 + 3 R0^4 f/8]
    int grad_r 1/R = -sum m f - sign(d) n Omega.

All functions are vectorised over a leading axis: ``r`` (n, 3), ``tri`` (n, 3, 3).
"""
import numpy as np


def _edge_terms(r, tri):
    p1, p2, p3 = tri[:, 0], tri[:, 1], tri[:, 2]
    cr = np.cross(p2 - p1, p3 - p1)
    n = cr / np.linalg.norm(cr, axis=1, keepdims=True)
    d = np.einsum('nd,nd->n', n, r - p1)
    rho = r - d[:, None] * n
    out = []
    for a, b in ((p1, p2), (p2, p3), (p3, p1)):
        L = np.linalg.norm(b - a, axis=1, keepdims=True)
        s = (b - a) / L
        m = np.cross(s, n)
        sm = np.einsum('nd,nd->n', a - rho, s)
        spl = np.einsum('nd,nd->n', b - rho, s)
        t0 = np.einsum('nd,nd->n', a - rho, m)
        R02 = t0 ** 2 + d ** 2
        Rm = np.sqrt(sm ** 2 + R02)
        Rp = np.sqrt(spl ** 2 + R02)
        # ln((R+ + s+)/(R- + s-)) written without cancellation: R + s = R0^2/(R - s) for s < 0
        with np.errstate(divide='ignore', invalid='ignore'):
            num = np.where(spl > 0, Rp + spl, R02 / (Rp - spl))
            den = np.where(sm > 0, Rm + sm, R02 / (Rm - sm))
            both_neg = (spl <= 0) & (sm <= 0)
            f = np.where(both_neg, np.log((Rm - sm) / (Rp - spl)), np.log(num / den))
            ad = np.abs(d)
            q1 = R02 + ad * Rp
            q2 = R02 + ad * Rm
            beta = np.where(q1 > 0, np.arctan(t0 * spl / np.where(q1 > 0, q1, 1.0)), 0.0) \
                - np.where(q2 > 0, np.arctan(t0 * sm / np.where(q2 > 0, q2, 1.0)), 0.0)
        out.append((m, sm, spl, t0, R02, Rm, Rp, f, beta))
    return n, d, rho, out


def integrals(r, tri):
    """Returns dict with 'inv_r', 'r' (scalars), 'p_over_r', 'p_r', 'grad_inv_r' (vectors), 'rho', 'n', 'd'."""
    n, d, rho, E = _edge_terms(r, tri)
    omega = sum(e[8] for e in E)
    inv_r = sum(e[3] * e[7] for e in E) - np.abs(d) * omega
    rr = sum(e[3] * (e[2] * e[6] - e[1] * e[5] + e[4] * e[7]) for e in E) / 6.0 + d ** 2 / 3.0 * inv_r
    p_over_r = sum(e[0] * (0.5 * (e[2] * e[6] - e[1] * e[5] + e[4] * e[7]))[:, None] for e in E)
    p_r = sum(e[0] * ((e[2] * e[6] ** 3 - e[1] * e[5] ** 3) / 4.0
                      + 3.0 * e[4] * (e[2] * e[6] - e[1] * e[5]) / 8.0
                      + 3.0 * e[4] ** 2 * e[7] / 8.0)[:, None] for e in E) / 3.0
    grad = -sum(e[0] * e[7][:, None] for e in E) - (np.sign(d) * omega)[:, None] * n
    return dict(inv_r=inv_r, r=rr, p_over_r=p_over_r, p_r=p_r, grad_inv_r=grad, rho=rho, n=n, d=d)
