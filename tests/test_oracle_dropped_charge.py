"""The charge-neutrality reading of B and F (Sec. II-B; D, B, F are defined by
reference only): per object the charge of one triangle is eliminated as minus
the sum of the others, B = [I; -1^T], and its continuity row is dropped,
F = [I 0].  Which triangle is eliminated is a numbering choice (the last of each
object), so reordering an object's triangles must leave the solution unchanged:
the edge unknowns j and e (edges are numbered by their vertices, not by the
triangle order), the full charge vector B u (up to the reordering) and the RCS.
A B that does not conserve charge (+1^T in place of -1^T, planted in the oracle
here) makes the solution depend on which triangle was eliminated.
"""
import numpy as np
import pytest

from oracle import farfield
from oracle import system as S
from oracle.topology import Mesh
from workloads.meshes import icosphere, merge

THETA = np.radians([0.0, 60.0, 120.0, 180.0])


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _solve(xyz, tri, obj, mats, freq):
    m = Mesh(xyz, tri, obj)
    A = S.assemble(m, mats, S.Material(), freq)
    x = S.solve(A, S.rhs(A))
    j, e, u = S.split(A, x)
    return m, j, e, m.B() @ u, farfield.rcs(m, A.k0, S.j_delta(A, x), THETA)


def _cases():
    v, f = icosphere(1, 0.1)
    yield "sphere", (v, f, None), [S.Material(4.0)], 300e6, np.roll(np.arange(len(f)), 17)
    xyz, tri, obj = merge(icosphere(1, 0.06), icosphere(1, 0.05, (0.15, 0.02, 0.0)))
    n0 = int(np.sum(obj == 0))
    perm = np.arange(len(tri))
    perm[n0:] = n0 + np.roll(np.arange(len(tri) - n0), 31)       # reorder the second object only
    yield "two_objects", (xyz, tri, obj), [S.Material(6.0, 1.0, 0.05), S.Material(2.5)], 500e6, perm


@pytest.mark.parametrize("case", list(_cases()), ids=lambda c: c[0])
def test_eliminated_triangle_does_not_matter(case):
    _, (xyz, tri, obj), mats, freq, perm = case
    m1, j1, e1, q1, s1 = _solve(xyz, tri, obj, mats, freq)
    m2, j2, e2, q2, s2 = _solve(xyz, tri[perm], None if obj is None else obj[perm], mats, freq)
    assert np.array_equal(m1.E.uv, m2.E.uv)
    assert _rel(j2, j1) < 1e-11 and _rel(e2, e1) < 1e-11
    assert _rel(q2, q1[perm]) < 1e-11
    assert np.max(np.abs(s2 / s1 - 1)) < 1e-10


def test_charge_not_conserved_depends_on_eliminated_triangle(monkeypatch):
    v, f = icosphere(1, 0.1)
    perm = np.roll(np.arange(len(f)), 17)
    right = Mesh.B

    def wrong_B(self):
        B = right(self)
        B[B == -1.0] = 1.0
        return B

    monkeypatch.setattr(Mesh, "B", wrong_B)
    _, j1, _, _, s1 = _solve(v, f, None, [S.Material(4.0)], 300e6)
    _, j2, _, _, s2 = _solve(v, f[perm], None, [S.Material(4.0)], 300e6)
    assert _rel(j2, j1) > 1e-2 and np.max(np.abs(s2 / s1 - 1)) > 1e-2
