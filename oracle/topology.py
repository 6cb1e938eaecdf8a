"""Discretisation of the surface (Sec. II-B): RWG edges, pulses, the incidence
matrix D, the charge-neutrality matrices B and F, the barycentric refinement and the
Buffa-Christiansen (BC) functions on it.

Conventions fixed here (the paper defers D, B, F and BC to the cited works; the
reading below is the one the CUDA library documents in ``include/sldm.h``):

* Edge ``n`` joins vertices ``u < v``.  ``T+`` is the triangle whose
  counter-clockwise boundary runs ``u -> v``; ``T-`` runs ``v -> u``.  Edges are
  ordered by ``(object, u, v)``.
* Area-normalised RWG: ``f_n = (r - p+)/(2 A+)`` on ``T+`` and
  ``-(r - p-)/(2 A-)`` on ``T-`` (``p`` = vertex opposite the edge).  Unit flux
  from ``T+`` to ``T-`` through the edge; ``div f_n = +1/A+ , -1/A-``.
* Area-normalised pulse ``h_p = 1/A_p`` on triangle ``p``; hence
  ``div f_n = sum_p D[p, n] h_p`` with ``D[T+, n] = +1``, ``D[T-, n] = -1``.
* Charge neutrality per object: the last triangle (in input order) of each object
  carries minus the sum of the other charges: ``B_o = [I; -1^T]``; the continuity
  row of that triangle is dropped: ``F_o = [I 0]``.
* Barycentric refinement: triangle (a, b, c) with centroid g and edge midpoints is
  split into (a, m_ab, g), (m_ab, b, g), (b, m_bc, g), (m_bc, c, g), (c, m_ca, g),
  (m_ca, a, g).
* BC function of edge n = (u, v): a combination of barycentric RWGs (unit flux
  each) carrying unit flux from the dual cell of ``u`` into the dual cell of
  ``v`` through the dual edge g+ - m_n - g- (1/2 through each half), zero flux
  through every other part of the two cells' boundaries, and equal integrated
  divergence +1/(2 N_u) on each of the 2 N_u barycentric triangles of the cell of
  ``u`` (and -1/(2 N_v) in the cell of ``v``).  The circulation left free by those
  conditions is fixed by zero flux through the half edge u - m_n (and v - m_n).
  With this orientation ``b_n`` is close to ``n x f_n`` and diag(I_x) > 0.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


class Edges:
    """Undirected edges of an oriented closed triangle mesh with RWG data."""

    def __init__(self, tri, obj=None, sort_obj=True):
        tri = np.asarray(tri, dtype=np.int64)
        nt = len(tri)
        if obj is None:
            obj = np.zeros(nt, dtype=np.int64)
        obj = np.asarray(obj, dtype=np.int64)
        directed = {}
        for t in range(nt):
            for i in range(3):
                a, b = tri[t, (i + 1) % 3], tri[t, (i + 2) % 3]  # edge opposite local vertex i
                if (a, b) in directed:
                    raise ValueError("mesh is not an oriented 2-manifold")
                directed[(a, b)] = (t, i)
        keys = []
        for (a, b) in directed:
            if a < b:
                if (b, a) not in directed:
                    raise ValueError("mesh is not closed")
                keys.append((obj[directed[(a, b)][0]] if sort_obj else 0, a, b))
        keys.sort()
        ne = len(keys)
        self.uv = np.array([[k[1], k[2]] for k in keys], dtype=np.int64).reshape(ne, 2)
        self.tp = np.empty(ne, dtype=np.int64)
        self.tm = np.empty(ne, dtype=np.int64)
        self.ip = np.empty(ne, dtype=np.int64)   # local index (opposite vertex) in T+
        self.im = np.empty(ne, dtype=np.int64)
        self.tri_edge = np.empty((nt, 3), dtype=np.int64)
        self.tri_sign = np.empty((nt, 3), dtype=np.float64)
        for n, (_, a, b) in enumerate(keys):
            tp, ip = directed[(a, b)]
            tm, im = directed[(b, a)]
            self.tp[n], self.ip[n], self.tm[n], self.im[n] = tp, ip, tm, im
            self.tri_edge[tp, ip], self.tri_sign[tp, ip] = n, +1.0
            self.tri_edge[tm, im], self.tri_sign[tm, im] = n, -1.0
        self.obj = obj[self.tp]
        self.ne = ne
        self.directed = directed


class Mesh:
    """Primal mesh, its barycentric refinement and the BC functions."""

    def __init__(self, xyz, tri, obj=None):
        self.xyz = np.asarray(xyz, dtype=np.float64)
        self.tri = np.asarray(tri, dtype=np.int64)
        nt = len(self.tri)
        self.nt = nt
        self.nv = len(self.xyz)
        self.obj = np.zeros(nt, dtype=np.int64) if obj is None else np.asarray(obj, dtype=np.int64)
        if np.any(np.diff(self.obj) < 0):
            raise ValueError("objects must be contiguous triangle ranges")
        self.nobj = int(self.obj.max()) + 1
        self.E = Edges(self.tri, self.obj)
        self.ne = self.E.ne
        p = self.xyz[self.tri]                                  # (nt, 3, 3)
        cr = np.cross(p[:, 1] - p[:, 0], p[:, 2] - p[:, 0])
        self.area = 0.5 * np.linalg.norm(cr, axis=1)
        self.normal = cr / (2.0 * self.area[:, None])
        self.centroid = p.mean(axis=1)
        self.tri_range = np.array([[np.searchsorted(self.obj, o), np.searchsorted(self.obj, o, 'right')]
                                   for o in range(self.nobj)])
        self.edge_range = np.array([[np.searchsorted(self.E.obj, o), np.searchsorted(self.E.obj, o, 'right')]
                                    for o in range(self.nobj)])
        self._barycentric()
        self._bc()

    # ---- D, B, F (Sec. II-B; definitions per the reading in the module docstring)
    def D(self):
        D = np.zeros((self.nt, self.ne))
        D[self.E.tp, np.arange(self.ne)] = 1.0
        D[self.E.tm, np.arange(self.ne)] = -1.0
        return D

    def B(self):
        """Block-diagonal (nt x (nt - nobj)): charge of each object's last triangle = -sum of the rest."""
        B = np.zeros((self.nt, self.nt - self.nobj))
        col = 0
        for o in range(self.nobj):
            t0, t1 = self.tri_range[o]
            k = t1 - t0 - 1
            B[t0:t0 + k, col:col + k] = np.eye(k)
            B[t1 - 1, col:col + k] = -1.0
            col += k
        return B

    def F(self):
        """Block-diagonal ((nt - nobj) x nt): drops the continuity row of each object's last triangle."""
        F = np.zeros((self.nt - self.nobj, self.nt))
        row = 0
        for o in range(self.nobj):
            t0, t1 = self.tri_range[o]
            k = t1 - t0 - 1
            F[row:row + k, t0:t0 + k] = np.eye(k)
            row += k
        return F

    # ---- barycentric refinement
    def _barycentric(self):
        nv, ne, nt = self.nv, self.ne, self.nt
        E = self.E
        mid = 0.5 * (self.xyz[E.uv[:, 0]] + self.xyz[E.uv[:, 1]])
        self.bxyz = np.concatenate([self.xyz, mid, self.centroid])
        btri = np.empty((6 * nt, 3), dtype=np.int64)
        for t in range(nt):
            a, b, c = self.tri[t]
            mab = nv + E.tri_edge[t, 2]
            mbc = nv + E.tri_edge[t, 0]
            mca = nv + E.tri_edge[t, 1]
            g = nv + ne + t
            btri[6 * t:6 * t + 6] = [[a, mab, g], [mab, b, g], [b, mbc, g],
                                     [mbc, c, g], [c, mca, g], [mca, a, g]]
        self.btri = btri
        self.bparent = np.repeat(np.arange(nt), 6)
        self.bobj = self.obj[self.bparent]
        self.bE = Edges(btri, self.bobj)
        q = self.bxyz[btri]
        cr = np.cross(q[:, 1] - q[:, 0], q[:, 2] - q[:, 0])
        self.barea = 0.5 * np.linalg.norm(cr, axis=1)
        self.bcentroid = q.mean(axis=1)

    def _ring(self, x, y0):
        """Counter-clockwise ring of triangles around vertex x, starting with edge (x, y0)."""
        out = []
        y = y0
        for _ in range(64):
            t, i = self.E.directed[(x, y)]
            loc = list(self.tri[t])
            p = loc.index(x)
            ynext = loc[(p + 2) % 3]
            out.append((t, p, y, ynext))
            y = ynext
            if y == y0:
                return out
        raise ValueError("vertex ring did not close")

    def _bc(self):
        """Sparse coefficients C (n_bary_edges x ne) with BC_n = sum_k C[k, n] g_k."""
        E, bE = self.E, self.bE
        rows, cols, vals = [], [], []

        def add_flux(t_from, t_to, flux, n):
            # barycentric edge shared by children t_from and t_to
            k = None
            for i in range(3):
                kk = bE.tri_edge[t_from, i]
                if bE.tp[kk] == t_to or bE.tm[kk] == t_to:
                    k = kk
                    break
            if k is None:
                raise RuntimeError("children are not adjacent")
            s = 1.0 if bE.tp[k] == t_from else -1.0
            rows.append(k); cols.append(n); vals.append(s * flux)

        for n in range(self.ne):
            u, v = E.uv[n]
            for x, y0, sgn in ((u, v, +1.0), (v, u, -1.0)):
                ring = self._ring(x, y0)
                N = len(ring)
                children = []
                for (t, p, _, _) in ring:
                    children.append(6 * t + 2 * p)           # (x, m(x, y_k), g)
                    children.append(6 * t + (2 * p + 5) % 6)  # (m(x, y_k+1), x, g)
                # Child i (0-based) must have net outflow sgn/(2N); children 0 and 2N-1
                # also pass sgn/2 through the dual edge.  Summing the balance from
                # child 0 with zero flux through the half edge (x, m_n) gives the flux
                # from child i to child i+1: sgn * (i + 1 - N) / (2N).
                for i in range(2 * N - 1):
                    F = sgn * (i + 1 - N) / (2.0 * N)
                    if F != 0.0:
                        add_flux(children[i], children[i + 1], F, n)
            # dual edge halves: from the cell of u into the cell of v, 1/2 each
            tp, ip, tm, im = E.tp[n], E.ip[n], E.tm[n], E.im[n]
            pu = list(self.tri[tp]).index(u)
            add_flux(6 * tp + 2 * pu, 6 * tp + (2 * ((pu + 1) % 3) + 5) % 6, 0.5, n)
            pu_m = list(self.tri[tm]).index(u)
            pv_m = list(self.tri[tm]).index(v)
            add_flux(6 * tm + (2 * pu_m + 5) % 6, 6 * tm + 2 * pv_m, 0.5, n)
        self.C = sp.csc_matrix((vals, (rows, cols)), shape=(self.bE.ne, self.ne))
