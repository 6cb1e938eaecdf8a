"""Seeded synthetic surface meshes (geometry only).

These generators produce closed, outward-oriented triangle meshes shaped like the
workloads of the single-layer dual-mesh BEM (a dielectric sphere, ellipsoids, a
copper wire, dielectric cylinders).  They contain no part of the method's
arithmetic: no basis functions, Green's functions or quadrature.  Both the CPU
oracle tests and the CUDA path consume their output.

Every mesh is returned as ``(xyz, tri)``: ``xyz`` float64 (nv, 3), ``tri`` int32
(nt, 3) with counter-clockwise vertex order seen from outside (outward normal).
"""
from __future__ import annotations

import numpy as np


def _icosahedron():
    t = (1.0 + 5.0 ** 0.5) / 2.0
    v = np.array([
        [-1, t, 0], [1, t, 0], [-1, -t, 0], [1, -t, 0],
        [0, -1, t], [0, 1, t], [0, -1, -t], [0, 1, -t],
        [t, 0, -1], [t, 0, 1], [-t, 0, -1], [-t, 0, 1],
    ], dtype=np.float64)
    f = np.array([
        [0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11],
        [1, 5, 9], [5, 11, 4], [11, 10, 2], [10, 7, 6], [7, 1, 8],
        [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8], [3, 8, 9],
        [4, 9, 5], [2, 4, 11], [6, 2, 10], [8, 6, 7], [9, 8, 1],
    ], dtype=np.int64)
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    return v, f


def _subdivide(v, f):
    """Split every triangle into four through its edge midpoints (unit sphere)."""
    verts = [tuple(p) for p in v]
    index = {}

    def mid(a, b):
        key = (a, b) if a < b else (b, a)
        if key not in index:
            p = (np.asarray(verts[a]) + np.asarray(verts[b])) * 0.5
            p /= np.linalg.norm(p)
            index[key] = len(verts)
            verts.append(tuple(p))
        return index[key]

    out = []
    for a, b, c in f:
        ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
        out += [[a, ab, ca], [b, bc, ab], [c, ca, bc], [ab, bc, ca]]
    return np.array(verts, dtype=np.float64), np.array(out, dtype=np.int64)


def icosphere(sub: int, radius: float = 1.0, center=(0.0, 0.0, 0.0)):
    """Geodesic sphere: 20 * 4**sub triangles, vertices on the sphere of ``radius``."""
    v, f = _icosahedron()
    for _ in range(sub):
        v, f = _subdivide(v, f)
    v = v * radius + np.asarray(center, dtype=np.float64)
    return v, f.astype(np.int32)


def ellipsoid(sub: int, semi_axes, center=(0.0, 0.0, 0.0)):
    """Icosphere scaled along x, y, z by ``semi_axes`` (orientation is preserved)."""
    v, f = icosphere(sub, 1.0)
    v = v * np.asarray(semi_axes, dtype=np.float64) + np.asarray(center, dtype=np.float64)
    return v, f


def box(lx: float, ly: float, lz: float, nx: int, ny: int, nz: int, center=(0.0, 0.0, 0.0),
        grade: float = 1.0, jitter: float = 0.0, seed: int = 0):
    """Closed rectangular box meshed with a structured grid on each face.

    ``grade`` > 1 grades the grid geometrically toward the box edges (ratio between
    the largest and the smallest cell along one axis; a 3-tuple grades x, y, z
    separately); ``jitter`` moves each
    face-interior vertex in the face plane by a seeded uniform amount of that
    fraction of the local cell size.
    """
    rng = np.random.default_rng(seed)

    grades = tuple(grade) if np.ndim(grade) else (grade, grade, grade)

    def axis(n, L, grade):
        if grade == 1.0 or n < 2:
            s = np.linspace(0.0, 1.0, n + 1)
        else:
            half = (n + 1) // 2
            r = grade ** (1.0 / max(half - 1, 1))
            w = r ** np.arange(half)
            w = np.concatenate([w, w[::-1][(n % 2):]]) if n > 1 else w
            w = w[:n]
            s = np.concatenate([[0.0], np.cumsum(w)]) / np.sum(w)
        return (s - 0.5) * L

    xs, ys, zs = axis(nx, lx, grades[0]), axis(ny, ly, grades[1]), axis(nz, lz, grades[2])
    vid = {}
    verts = []

    def vert(i, j, k):
        key = (i, j, k)
        if key not in vid:
            vid[key] = len(verts)
            verts.append([xs[i], ys[j], zs[k]])
        return vid[key]

    tris = []

    def face(fixed_axis, fixed_idx, outward_sign):
        a1, a2 = [a for a in range(3) if a != fixed_axis]
        n1 = (nx, ny, nz)[a1]
        n2 = (nx, ny, nz)[a2]
        for i in range(n1):
            for j in range(n2):
                corners = []
                for (di, dj) in ((0, 0), (1, 0), (1, 1), (0, 1)):
                    idx = [0, 0, 0]
                    idx[fixed_axis] = fixed_idx
                    idx[a1] = i + di
                    idx[a2] = j + dj
                    corners.append(vert(*idx))
                p0, p1, p2, p3 = corners
                # (a1, a2, fixed) right-handed when fixed_axis follows a2 cyclically
                right_handed = (a1, a2, fixed_axis) in ((0, 1, 2), (1, 2, 0), (2, 0, 1))
                ccw = right_handed == (outward_sign > 0)
                if (i + j) % 2 == 0:
                    quad = [(p0, p1, p2), (p0, p2, p3)]
                else:
                    quad = [(p0, p1, p3), (p1, p2, p3)]
                for t in quad:
                    tris.append(t if ccw else (t[0], t[2], t[1]))

    face(0, 0, -1); face(0, nx, +1)
    face(1, 0, -1); face(1, ny, +1)
    face(2, 0, -1); face(2, nz, +1)
    v = np.array(verts, dtype=np.float64)
    if jitter > 0.0:
        keys = list(vid.keys())
        for (i, j, k), n in zip(keys, range(len(keys))):
            idx = vid[(i, j, k)]
            on = [(i in (0, nx)), (j in (0, ny)), (k in (0, nz))]
            if sum(on) != 1:
                continue  # box edges and corners stay put
            ax = on.index(True)
            for a, (c, arr, nn) in enumerate(((i, xs, nx), (j, ys, ny), (k, zs, nz))):
                if a == ax:
                    continue
                h = min(arr[c] - arr[c - 1], arr[c + 1] - arr[c])
                v[idx, a] += jitter * h * rng.uniform(-1.0, 1.0)
    v = v + np.asarray(center, dtype=np.float64)
    return v, np.array(tris, dtype=np.int32)


def cylinder(radius: float, height: float, n_around: int = 20, n_side: int = 4,
             n_rings: int = 2, center=(0.0, 0.0, 0.0)):
    """Closed circular cylinder along z, base at ``center[2]``.

    Side: ``n_around`` x ``n_side`` quads split in two.  Each cap: a fan of
    ``n_around // 2`` triangles around the axis point from an inner ring of
    ``n_around // 2`` vertices, then ``n_rings - 1`` annuli stitching the inner ring
    to the rim.  With the defaults (20, 4, 2): 160 side + 2 x (10 + 30) = 240
    triangles.
    """
    cx, cy, cz = center
    verts = []
    tris = []

    def add(p):
        verts.append(p)
        return len(verts) - 1

    ang = 2 * np.pi * np.arange(n_around) / n_around
    rim = []
    for k in range(n_side + 1):
        z = cz + height * k / n_side
        rim.append([add([cx + radius * np.cos(a), cy + radius * np.sin(a), z]) for a in ang])
    for k in range(n_side):
        for i in range(n_around):
            i2 = (i + 1) % n_around
            a, b = rim[k][i], rim[k][i2]
            c, d = rim[k + 1][i2], rim[k + 1][i]
            tris += [(a, b, c), (a, c, d)]

    def cap(z, ring_outer, up):
        m = n_around // 2
        inner_r = radius * 0.5
        ang_in = 2 * np.pi * (np.arange(m) + 0.5) / m
        inner = [add([cx + inner_r * np.cos(a), cy + inner_r * np.sin(a), z]) for a in ang_in]
        centre = add([cx, cy, z])
        loc = []
        for i in range(m):
            loc.append((centre, inner[i], inner[(i + 1) % m]))
        # annulus between the inner ring (m vertices) and the rim (n_around = 2m vertices)
        for i in range(m):
            o0, o1, o2 = ring_outer[2 * i], ring_outer[2 * i + 1], ring_outer[(2 * i + 2) % n_around]
            i0, i1 = inner[i - 1] if i > 0 else inner[m - 1], inner[i]
            loc += [(i0, o0, o1), (i0, o1, i1), (i1, o1, o2)]
        for t in loc:
            tris.append(t if up else (t[0], t[2], t[1]))

    cap(cz + height, rim[n_side], True)
    cap(cz, rim[0], False)
    return np.array(verts, dtype=np.float64), np.array(tris, dtype=np.int32)


def merge(*meshes):
    """Concatenate meshes; returns (xyz, tri, obj_id) with one object per input mesh."""
    xyz, tri, obj = [], [], []
    off = 0
    for o, (v, f) in enumerate(meshes):
        xyz.append(v)
        tri.append(f + off)
        obj.append(np.full(len(f), o, dtype=np.int32))
        off += len(v)
    return np.concatenate(xyz), np.concatenate(tri).astype(np.int32), np.concatenate(obj)


def cylinder_array(nx: int, ny: int, radius: float, height: float, period: float, z0: float = 0.0):
    """nx x ny capped cylinders (240 triangles each) on a square lattice, bases at z0.

    Returns (xyz, tri, obj) with one object per cylinder, row by row.
    """
    ox = -(nx - 1) * period / 2
    oy = -(ny - 1) * period / 2
    return merge(*[cylinder(radius, height, center=(ox + i * period, oy + j * period, z0))
                   for j in range(ny) for i in range(nx)])


def copper_wire(seed: int = 2106_06184 + 1):
    """The multiscale conductor: a 100 x 2 x 1 um bar along x centred at
    (0, 0, -5 um), 40 x 8 x 4 cells graded along x from 0.50 um at the ends to
    6.88 um in the middle (0.25 um across), face-interior vertices jittered by 1%
    of the local cell (seeded): 2,048 triangles, 3,072 edges."""
    return box(100e-6, 2e-6, 1e-6, 40, 8, 4, center=(0.0, 0.0, -5e-6), grade=(13.760248682707653, 1.0, 1.0),
               jitter=0.01, seed=seed)
