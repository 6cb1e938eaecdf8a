"""Six-point, degree-4 symmetric Gauss rule on a triangle (Dunavant, 1985), the
quadrature used on both triangles of every pair of the fill (Sec. II-B).

``BARY`` holds barycentric coordinates, ``W`` the weights normalised to sum 1 (the
integral over a triangle of area A is ``A * sum(W * f(points))``).
"""
import numpy as np

_a1, _b1, _w1 = 0.445948490915965, 0.108103018168070, 0.223381589678011
_a2, _b2, _w2 = 0.091576213509771, 0.816847572980459, 0.109951743655322

BARY = np.array([
    [_b1, _a1, _a1], [_a1, _b1, _a1], [_a1, _a1, _b1],
    [_b2, _a2, _a2], [_a2, _b2, _a2], [_a2, _a2, _b2],
])
W = np.array([_w1, _w1, _w1, _w2, _w2, _w2])


def points(tri_xyz):
    """Quadrature points of triangles ``tri_xyz`` (n, 3, 3) -> (n, 6, 3)."""
    return np.einsum('qk,nkd->nqd', BARY, tri_xyz)


def weights(area):
    """Quadrature weights (area Jacobian included) of triangles of ``area`` (n,) -> (n, 6)."""
    return np.outer(area, W)
