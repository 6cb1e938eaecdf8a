"""Galerkin fill of the operators of Sec. II-B and II-C, plainly, in FP64.

Readings of the discretisation (Eqs. opLAhgf, opLphihgf, opKhgf, AEFIEintdis):

    L^A[m, n]   = int_T f_m(r) . int_T' f_n(r') G(r, r') dS' dS          (RWG x RWG)
    L^phi[p, q] = int int h_p(r) h_q(r') G(r, r') dS' dS                (pulse x pulse)
    Kbar[m, n]  = int f_m(r) . PV int grad_r G(r, r') x b_n(r') dS' dS    (RWG x BC)
    I_x[m, n]   = int (n x f_m) . b_n dS                                 (Gram, BC tested with n x RWG)
    e_inc[m]    = int f_m . E_inc / eta0 dS

with G = exp(-j k R) / (4 pi R) (Eq. hgf), time convention exp(+j w t).

Quadrature: the 6-point Dunavant rule on the test and on the source triangle.
Touching pairs (sharing at least one point) use singularity extraction: for L the
inner integral of 1/(4 pi R) - k^2 R/(8 pi) is done in closed form and the
remainder G - 1/(4 pi R) + k^2 R/(8 pi) by the same 6-point rule; for Kbar the
static gradient grad 1/(4 pi R) is done in closed form.  A barycentric source
triangle lying inside the test triangle contributes zero to Kbar (coplanar: the
integrand is normal to the plane while f_m is tangential).  BC functions enter as
sums of barycentric RWG functions (``mesh.C``), see ``oracle.topology``.

Good conductors (Sec. II-B: the entries of highly conductive objects need
integration that follows the fast decay of G over a skin depth).  Reading: a
source triangle T' (primal for L, barycentric for Kbar) with an edge longer than
1/|Im k| is bisected through the midpoint of its longest edge, recursively,
until no child has an edge longer than 1/|Im k| (``source_rule``), and the
6-point rule is applied on each child.  Bisection refines only across the long
direction, so the thin triangles of a graded conductor mesh are not split
across their short side.  A split touching pair extracts only the static
1/(4 pi R) term: the k^2 R/(8 pi) term is no longer small against G once
|k| d > 1.  When any source of a fill is split, that fill also drops the
non-touching pairs whose bounding spheres are farther apart than 40 / |Im k|
(G has decayed below exp(-40) there).
"""
from __future__ import annotations

import numpy as np

from . import quadrature as Q
from .singular import integrals

C0 = 299792458.0
MU0 = 4e-7 * np.pi
EPS0 = 1.0 / (MU0 * C0 ** 2)
ETA0 = MU0 * C0

CHUNK = 4096
SUB_MAX_CHILDREN = 4096  # most children of one split source triangle
SPLIT_TIE = 1e-9         # edges within this relative distance of the longest count as longest
R8_CUTOFF = 40.0   # |Im k| x (distance of the bounding spheres) beyond which a pair is dropped


def green(k, R):
    return np.exp(-1j * k * R) / (4 * np.pi * R)


def green_smooth(k, R):
    """G - 1/(4 pi R) + k^2 R / (8 pi); a Taylor series where |k R| is small."""
    x = k * R
    with np.errstate(invalid='ignore', divide='ignore'):
        full = (np.exp(-1j * x) - 1.0) / (4 * np.pi * R) + k * k * R / (8 * np.pi)
    ser = np.zeros_like(full)
    for n in range(1, 12):
        if n == 2:
            continue
        ser = ser + (-1j * k) ** n * R ** (n - 1) / np.prod(np.arange(1, n + 1), dtype=float)
    ser = ser / (4 * np.pi)
    return np.where(np.abs(x) < 0.05, ser, full)


def green_smooth1(k, R):
    """G - 1/(4 pi R) = (exp(-j k R) - 1)/(4 pi R); a Taylor series where |k R| is small."""
    x = k * R
    with np.errstate(invalid='ignore', divide='ignore'):
        full = (np.exp(-1j * x) - 1.0) / (4 * np.pi * R)
    ser = np.zeros_like(full)
    for n in range(1, 12):
        ser = ser + (-1j * k) ** n * R ** (n - 1) / np.prod(np.arange(1, n + 1), dtype=float)
    ser = ser / (4 * np.pi)
    return np.where(np.abs(x) < 0.05, ser, full)


def split_children(P, h):
    """Children of the triangle with vertices P (3, 3) under longest-edge bisection
    until no child has an edge longer than h: barycentric vertex triples with
    respect to P (nc, 3, 3) and area fractions (nc,).  Edge i joins vertices i and
    i + 1; the edge split is the first within SPLIT_TIE of the longest; the child
    holding the edge's first vertex comes first."""
    todo = [(np.eye(3), 1.0)]
    out_b, out_f = [], []
    while todo:
        B, f = todo.pop()
        X = B @ P
        L = np.linalg.norm(X - np.roll(X, -1, axis=0), axis=1)
        Lmax = L.max()
        if not (Lmax > h):
            out_b.append(B)
            out_f.append(f)
            continue
        i = int(np.nonzero(L >= (1.0 - SPLIT_TIE) * Lmax)[0][0])
        a, b, c = B[i], B[(i + 1) % 3], B[(i + 2) % 3]
        m = 0.5 * (a + b)
        todo.append((np.array([m, b, c]), 0.5 * f))
        todo.append((np.array([a, m, c]), 0.5 * f))
        if len(out_b) + len(todo) > SUB_MAX_CHILDREN:
            raise ValueError(f"source triangle too large for the skin depth: more than {SUB_MAX_CHILDREN} children")
    return np.array(out_b), np.array(out_f)


def source_rule(P, k):
    """Quadrature of one source triangle (vertices P) for wavenumber k: barycentric
    points (ns, 3) and weights (ns,) summing to 1; the 6-point rule when no edge
    exceeds 1/|Im k|, else the 6-point rule on each child of ``split_children``."""
    aki = abs(np.imag(k))
    h = 1.0 / aki if aki > 0 else np.inf
    Bc, fr = split_children(np.asarray(P, dtype=float), h)
    pts = np.einsum('qk,ckd->cqd', Q.BARY, Bc).reshape(-1, 3)
    return pts, (fr[:, None] * Q.W[None, :]).reshape(-1)


def needs_split(k, P):
    """Per triangle (P: (n, 3, 3)): has an edge longer than 1/|Im k|."""
    return abs(np.imag(k)) * _diam(P) > 1.0


def _diam(P):
    """Longest edge of triangles P (n, 3, 3)."""
    return np.max(np.linalg.norm(P - np.roll(P, 1, axis=1), axis=2), axis=1)


def _sphere(P):
    """Bounding sphere of triangles P: centroid and largest vertex distance."""
    c = P.mean(axis=1)
    return c, np.max(np.linalg.norm(P - c[:, None, :], axis=2), axis=1)


def _kept(k, Pa, Pb, touch):
    """Pairs kept by the far-pair rule: touching, or |Im k| (|c - c'| - r - r') <= 40."""
    ca, ra = _sphere(Pa)
    cb, rb = _sphere(Pb)
    gap = np.linalg.norm(ca - cb, axis=1) - ra - rb
    return touch | (abs(np.imag(k)) * gap <= R8_CUTOFF)


def grad_green_factor(k, R):
    """g1 with grad_r G = (r - r') g1: g1 = -(1 + j k R) exp(-j k R) / (4 pi R^3)."""
    return -(1 + 1j * k * R) * np.exp(-1j * k * R) / (4 * np.pi * R ** 3)


def grad_green_smooth_factor(k, R):
    """g1 of G - 1/(4 pi R): (1 - (1 + j k R) exp(-j k R)) / (4 pi R^3), series for small |k R|."""
    x = 1j * k * R
    full = (1.0 - (1 + x) * np.exp(-x)) / (4 * np.pi * R ** 3)
    ser = np.zeros_like(full)
    for n in range(2, 14):
        ser = ser + (-1) ** n * (n - 1) * x ** n / np.prod(np.arange(1, n + 1), dtype=float)
    ser = ser / (4 * np.pi * R ** 3)
    return np.where(np.abs(x) < 0.05, ser, full)


# ----------------------------------------------------------------------------- L^A and L^phi

def _touch_primal(tri, a, b):
    ta, tb = tri[a], tri[b]
    return (ta[:, :, None] == tb[:, None, :]).any(axis=(1, 2))


def _L_pairs(mesh, k, ta, tb, rule=None):
    """Local RWG x RWG (P, 3, 3) and pulse x pulse (P,) integrals of triangle pairs.
    rule: per-pair source quadrature (barycentric points (P, ns, 3), weights (P, ns)),
    the same ns for every pair; None = the 6-point rule.  ns > 6 means split."""
    xyz, tri = mesh.xyz, mesh.tri
    A, B = xyz[tri[ta]], xyz[tri[tb]]
    if rule is None:
        rule = (np.broadcast_to(Q.BARY, (len(tb), 6, 3)), np.broadcast_to(Q.W, (len(tb), 6)))
    bs, wsub = rule
    rq, rs = Q.points(A), np.einsum('pqk,pkd->pqd', bs, B)
    wq, ws = Q.weights(mesh.area[ta]), mesh.area[tb][:, None] * wsub
    fa = rq[:, :, None, :] - A[:, None, :, :]          # r - v_i   (P, 6, 3, 3)
    fb = rs[:, :, None, :] - B[:, None, :, :]          # r' - w_j
    scale = (mesh.E.tri_sign[ta][:, :, None] * mesh.E.tri_sign[tb][:, None, :]
             / (4 * mesh.area[ta] * mesh.area[tb])[:, None, None])
    la = np.zeros((len(ta), 3, 3), dtype=complex)
    lp = np.zeros(len(ta), dtype=complex)
    touch = _touch_primal(tri, ta, tb)
    far = ~touch
    if far.any():
        R = np.linalg.norm(rq[far][:, :, None, :] - rs[far][:, None, :, :], axis=-1)
        G = green(k, R) * wq[far][:, :, None] * ws[far][:, None, :]
        la[far] = np.einsum('pqs,pqid,psjd->pij', G, fa[far], fb[far], optimize='greedy')
        lp[far] = G.sum(axis=(1, 2))
    if touch.any():
        idx = np.nonzero(touch)[0]
        P = len(idx)
        R = np.linalg.norm(rq[idx][:, :, None, :] - rs[idx][:, None, :, :], axis=-1)
        two = bs.shape[1] == 6                                               # unsplit: extract 1/R and R, else 1/R only
        Gs = (green_smooth(k, R) if two else green_smooth1(k, R)) * ws[idx][:, None, :]   # (P, 6q, ns)
        inner_a = np.einsum('pqs,psjd->pqjd', Gs, fb[idx])                   # (P, 6, 3, 3)
        inner_p = Gs.sum(axis=2)                                             # (P, 6)
        kk = k * k if two else 0.0
        r = rq[idx].reshape(-1, 3)
        T = np.repeat(B[idx], 6, axis=0)
        I = integrals(r, T)
        rho = I['rho'].reshape(P, 6, 1, 3)
        w = B[idx][:, None, :, :]                                            # (P, 1, 3j, 3)
        por = I['p_over_r'].reshape(P, 6, 1, 3)
        pr = I['p_r'].reshape(P, 6, 1, 3)
        inv_r = I['inv_r'].reshape(P, 6, 1, 1)
        rr = I['r'].reshape(P, 6, 1, 1)
        inner_a = inner_a + (por + (rho - w) * inv_r) / (4 * np.pi) \
            - kk * (pr + (rho - w) * rr) / (8 * np.pi)
        inner_p = inner_p + I['inv_r'].reshape(P, 6) / (4 * np.pi) - kk * I['r'].reshape(P, 6) / (8 * np.pi)
        la[idx] = np.einsum('pq,pqid,pqjd->pij', wq[idx], fa[idx], inner_a)
        lp[idx] = np.einsum('pq,pq->p', wq[idx], inner_p)
    return la * scale, lp / (mesh.area[ta] * mesh.area[tb])


def _rule_groups(k, P, srcs):
    """Sources grouped by the size of their quadrature, with the rules stacked:
    [(sources, (points (S, ns, 3), weights (S, ns)) or None for the plain 6-point
    rule when no source of the fill is split)]."""
    srcs = np.asarray(srcs)
    if not needs_split(k, P[srcs]).any():
        return [(srcs, None)]
    rules = [source_rule(P[s], k) for s in srcs]
    ns = np.array([len(r[1]) for r in rules])
    out = []
    for n in np.unique(ns):
        sel = np.nonzero(ns == n)[0]
        out.append((srcs[sel], (np.stack([rules[i][0] for i in sel]), np.stack([rules[i][1] for i in sel]))))
    return out


def fill_L(mesh, k, tris):
    """L^A over the edges of triangles ``tris`` and L^phi over ``tris`` (whole objects)."""
    tris = np.asarray(tris)
    e_of = mesh.E.tri_edge
    edges = np.unique(e_of[tris])
    eidx = -np.ones(mesh.ne, dtype=np.int64)
    eidx[edges] = np.arange(len(edges))
    tidx = -np.ones(mesh.nt, dtype=np.int64)
    tidx[tris] = np.arange(len(tris))
    LA = np.zeros((len(edges), len(edges)), dtype=complex)
    LP = np.zeros((len(tris), len(tris)), dtype=complex)
    P = mesh.xyz[mesh.tri]
    for srcs, rules in _rule_groups(k, P, tris):
        ta_all = np.repeat(tris, len(srcs))
        tb_all = np.tile(srcs, len(tris))
        ri_all = np.tile(np.arange(len(srcs)), len(tris))
        if rules is not None:
            keep = _kept(k, P[ta_all], P[tb_all], _touch_primal(mesh.tri, ta_all, tb_all))
            ta_all, tb_all, ri_all = ta_all[keep], tb_all[keep], ri_all[keep]
        step = max(1, CHUNK * 6 // (rules[0].shape[1] if rules is not None else 6))
        for c in range(0, len(ta_all), step):
            ta, tb, ri = ta_all[c:c + step], tb_all[c:c + step], ri_all[c:c + step]
            la, lp = _L_pairs(mesh, k, ta, tb, None if rules is None else (rules[0][ri], rules[1][ri]))
            rows = eidx[e_of[ta]][:, :, None] * np.ones((1, 1, 3), dtype=np.int64)
            cols = eidx[e_of[tb]][:, None, :] * np.ones((1, 3, 1), dtype=np.int64)
            np.add.at(LA, (rows.ravel(), cols.ravel()), la.ravel())
            np.add.at(LP, (tidx[ta], tidx[tb]), lp)
    return LA, LP


# ----------------------------------------------------------------------------- Kbar

def _touch_bary(mesh, ta, cb):
    """0 = far, 1 = touching (extraction), 2 = child of the test triangle (zero)."""
    nv = mesh.nv
    parent = mesh.bparent[cb]
    bv = mesh.btri[cb]                                               # (P, 3)
    tv = mesh.tri[ta]                                                # (P, 3)
    tm = nv + mesh.E.tri_edge[ta]                                    # midpoint ids of the test edges
    keys = np.concatenate([tv, tm], axis=1)                          # (P, 6)
    touch = (bv[:, :, None] == keys[:, None, :]).any(axis=(1, 2))
    out = np.where(touch, 1, 0)
    return np.where(parent == ta, 2, out)


def _K_pairs(mesh, k, ta, cb, rule=None):
    """Local RWG (test, primal) x barycentric RWG (source) integrals of Kbar, (P, 3, 3).
    rule: per-pair source quadrature as for _L_pairs (None = the 6-point rule)."""
    A = mesh.xyz[mesh.tri[ta]]
    Bt = mesh.bxyz[mesh.btri[cb]]
    if rule is None:
        rule = (np.broadcast_to(Q.BARY, (len(cb), 6, 3)), np.broadcast_to(Q.W, (len(cb), 6)))
    bs, wsub = rule
    rq, rs = Q.points(A), np.einsum('pqk,pkd->pqd', bs, Bt)
    wq, ws = Q.weights(mesh.area[ta]), mesh.barea[cb][:, None] * wsub
    ns = rs.shape[1]
    fa = (rq[:, :, None, :] - A[:, None, :, :]) * \
        (mesh.E.tri_sign[ta] / (2 * mesh.area[ta][:, None]))[:, None, :, None]          # f_i(r_q)
    sb = mesh.bE.tri_sign[cb] / (2 * mesh.barea[cb][:, None])                            # (P, 3)
    gb = (rs[:, :, None, :] - Bt[:, None, :, :]) * sb[:, None, :, None]                  # g_j(r_s)
    kind = _touch_bary(mesh, ta, cb)
    out = np.zeros((len(ta), 3, 3), dtype=complex)
    far = np.nonzero(kind == 0)[0]
    if len(far):
        d = rq[far][:, :, None, :] - rs[far][:, None, :, :]                               # r - r'
        R = np.linalg.norm(d, axis=-1)
        g1 = grad_green_factor(k, R) * wq[far][:, :, None] * ws[far][:, None, :]
        # inner[p, q, j] = sum_s g1 (r_q - r'_s) x g_j(r'_s);  out = sum_q f_i(r_q) . inner
        X = np.cross(d[:, :, :, None, :], gb[far][:, None, :, :, :])                     # (P, q, s, j, 3)
        inner = np.matmul(g1[:, :, None, :], X.reshape(len(far), 6, ns, 9)).reshape(len(far), 6, 3, 3)
        out[far] = np.einsum('pqia,pqja->pij', fa[far], inner)
    near = np.nonzero(kind == 1)[0]
    if len(near):
        P = len(near)
        d = rq[near][:, :, None, :] - rs[near][:, None, :, :]
        R = np.linalg.norm(d, axis=-1)
        g1 = grad_green_smooth_factor(k, R) * ws[near][:, None, :]
        X = np.cross(d[:, :, :, None, :], gb[near][:, None, :, :, :])
        inner = np.matmul(g1[:, :, None, :], X.reshape(P, 6, ns, 9)).reshape(P, 6, 3, 3)
        I = integrals(rq[near].reshape(-1, 3), np.repeat(Bt[near], 6, axis=0))
        gs = I['grad_inv_r'].reshape(P, 6, 1, 3) / (4 * np.pi)
        # static part: [int grad 1/(4 pi R) dS'] x g_j evaluated through (r - r') x (r' - w) = (r - r') x (r - w)
        rw = (rq[near][:, :, None, :] - Bt[near][:, None, :, :]) * sb[near][:, None, :, None]
        inner = inner + np.cross(np.broadcast_to(gs, rw.shape), rw)
        out[near] = np.einsum('pq,pqid,pqjd->pij', wq[near], fa[near], inner)
    return out


def fill_Kbar(mesh, k, obj):
    """Kbar (RWG test x BC source) of object ``obj``: (ne_o x ne_o), plus its barycentric form."""
    t0, t1 = mesh.tri_range[obj]
    e0, e1 = mesh.edge_range[obj]
    bidx = np.nonzero(mesh.bE.obj == obj)[0]
    b0 = bidx[0]
    tris = np.arange(t0, t1)
    kids = np.arange(6 * t0, 6 * t1)
    Kb = np.zeros((e1 - e0, len(bidx)), dtype=complex)
    P = mesh.xyz[mesh.tri]
    Pb = mesh.bxyz[mesh.btri]
    for srcs, rules in _rule_groups(k, Pb, kids):
        ta_all = np.repeat(tris, len(srcs))
        cb_all = np.tile(srcs, len(tris))
        ri_all = np.tile(np.arange(len(srcs)), len(tris))
        if rules is not None:
            keep = _kept(k, P[ta_all], Pb[cb_all], _touch_bary(mesh, ta_all, cb_all) > 0)
            ta_all, cb_all, ri_all = ta_all[keep], cb_all[keep], ri_all[keep]
        step = max(1, CHUNK * 6 // (rules[0].shape[1] if rules is not None else 6))
        for c in range(0, len(ta_all), step):
            ta, cb, ri = ta_all[c:c + step], cb_all[c:c + step], ri_all[c:c + step]
            loc = _K_pairs(mesh, k, ta, cb, None if rules is None else (rules[0][ri], rules[1][ri]))
            rows = (mesh.E.tri_edge[ta] - e0)[:, :, None] * np.ones((1, 1, 3), dtype=np.int64)
            cols = (mesh.bE.tri_edge[cb] - b0)[:, None, :] * np.ones((1, 3, 1), dtype=np.int64)
            np.add.at(Kb, (rows.ravel(), cols.ravel()), loc.ravel())
    Cobj = mesh.C[b0:b0 + len(bidx), e0:e1].toarray()
    return Kb @ Cobj, Kb


# ----------------------------------------------------------------------------- Gram I_x

def fill_Ix(mesh):
    """I_x[m, n] = int (n x f_m) . b_n over the whole mesh (block diagonal by object)."""
    Ixb = np.zeros((mesh.ne, mesh.bE.ne))
    for t in range(mesh.nt):
        A = mesh.xyz[mesh.tri[t]]
        n = mesh.normal[t]
        for c in range(6 * t, 6 * t + 6):
            Bt = mesh.bxyz[mesh.btri[c]]
            rs = Q.points(Bt[None])[0]
            ws = Q.weights(mesh.barea[c:c + 1])[0]
            for i in range(3):
                fi = mesh.E.tri_sign[t, i] * (rs - A[i]) / (2 * mesh.area[t])
                nf = np.cross(n, fi)
                for j in range(3):
                    gj = mesh.bE.tri_sign[c, j] * (rs - Bt[j]) / (2 * mesh.barea[c])
                    Ixb[mesh.E.tri_edge[t, i], mesh.bE.tri_edge[c, j]] += np.sum(ws * np.einsum('qd,qd->q', nf, gj))
    return Ixb @ mesh.C.toarray()


# ----------------------------------------------------------------------------- excitation

def plane_wave(mesh, k0, khat, pol, E0=1.0):
    """e_inc[m] = int f_m . E_inc / eta0 with E_inc = pol E0 exp(-j k0 khat . r)."""
    khat = np.asarray(khat, float)
    pol = np.asarray(pol, complex)
    A = mesh.xyz[mesh.tri]
    rq = Q.points(A)
    wq = Q.weights(mesh.area)
    Einc = E0 * pol[None, None, :] * np.exp(-1j * k0 * rq @ khat)[..., None] / ETA0   # (nt, 6, 3)
    b = np.zeros(mesh.ne, dtype=complex)
    for i in range(3):
        fi = (rq - A[:, i][:, None, :]) * (mesh.E.tri_sign[:, i] / (2 * mesh.area))[:, None, None]
        np.add.at(b, mesh.E.tri_edge[:, i], np.einsum('tq,tqd,tqd->t', wq, fi, Einc))
    return b
