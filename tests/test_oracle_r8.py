"""Pins of the oracle's good-conductor integration (source triangles bisected
through their longest edge until no edge exceeds 1/|Im k|, one-term extraction
on split touching pairs, far pairs dropped beyond |Im k| R = 40), against facts
fixed outside it:
polynomial exactness of the composite rule, closed-form integrals of a smooth
function, brute-force integration of strongly decaying kernels, and the size of
the dropped entries."""
import math

import numpy as np
import pytest

from oracle import fill, quadrature as Q
from oracle.topology import Mesh
from workloads.meshes import icosphere

from test_oracle_pins import _duffy

MU0 = 4e-7 * np.pi
EPS0 = 1.0 / (MU0 * 299792458.0 ** 2)


def copper_k(freq, sigma=5.8e7):
    w = 2 * np.pi * freq
    k0 = w / 299792458.0
    return k0 * np.sqrt(complex(1.0, -sigma / (w * EPS0)))


REF = np.array([[0.0, 0, 0], [1.0, 0, 0], [0.0, 1, 0]])   # reference triangle (0,0), (1,0), (0,1)


@pytest.mark.parametrize("h", [2.0, 0.9, 0.4, 0.2])
def test_split_rule_exact_to_degree_4(h):
    pts, w = fill.source_rule(REF, 1j / h)
    assert abs(w.sum() - 1.0) < 1e-14 and np.allclose(pts.sum(axis=1), 1.0) and pts.min() > 0.0
    # int x^a y^b = a! b! / (a + b + 2)!
    x, y = pts[:, 1], pts[:, 2]
    for a in range(5):
        for b in range(5 - a):
            exact = math.factorial(a) * math.factorial(b) / math.factorial(a + b + 2)
            assert abs(0.5 * np.sum(w * x ** a * y ** b) - exact) < 1e-14, (h, a, b)


def test_split_children_geometry():
    """Every child's longest edge is at most h, the area fractions are powers of 1/2
    summing to 1, an unsplit triangle is its own child, and a thin triangle is cut
    across its long direction only."""
    for P, h in ((REF, 0.3), (np.array([[0.0, 0, 0], [10.0, 0, 0], [3.0, 0.5, 0]]), 1.0)):
        B, f = fill.split_children(P, h)
        X = np.einsum('cvk,kd->cvd', B, P)
        assert np.max(np.linalg.norm(X - np.roll(X, -1, axis=1), axis=2)) <= h
        assert abs(f.sum() - 1.0) < 1e-15 and np.allclose(np.log2(f), np.round(np.log2(f)))
        area = 0.5 * np.linalg.norm(np.cross(X[:, 1] - X[:, 0], X[:, 2] - X[:, 0]), axis=1)
        assert np.allclose(area / (0.5 * np.linalg.norm(np.cross(P[1] - P[0], P[2] - P[0]))), f)
    B, f = fill.split_children(REF, 2.0)
    assert len(f) == 1 and np.array_equal(B[0], np.eye(3))
    thin = np.array([[0.0, 0, 0], [10.0, 0, 0], [3.0, 0.5, 0]])
    _, f = fill.split_children(thin, 1.0)
    assert len(f) <= 48            # edge-midpoint quartering to the same edge bound needs 4^4 = 256


def test_split_rule_converges_on_a_smooth_function():
    """int exp(a x + b y) over the reference triangle = [(e^a - e^b)/(a - b) - (e^a - 1)/a] / b."""
    a, b = 2.0, -3.0
    exact = ((np.exp(a) - np.exp(b)) / (a - b) - (np.exp(a) - 1) / a) / b
    err = []
    for h in (2.0, 1.0, 0.5, 0.25):
        pts, w = fill.source_rule(REF, 1j / h)
        err.append(abs(0.5 * np.sum(w * np.exp(a * pts[:, 1] + b * pts[:, 2])) - exact))
    for e0, e1 in zip(err, err[1:]):
        assert e1 < e0 / 10.0, err


def test_needs_split_rule():
    k = 1.0 - 1.0j
    P = np.array([d * REF / np.sqrt(2) for d in (0.5, 1.0, 1.5)])   # longest edge d
    assert list(fill.needs_split(k, P)) == [False, False, True]
    assert not fill.needs_split(3.0 + 0j, P).any()                   # lossless: never split
    with pytest.raises(ValueError):
        fill.source_rule(REF * 1e3, k)                               # too many children


def _lp_brute(k, A, B, n=160):
    """(1/(A A')) int_T int_T' G by the 6-point outer rule and Duffy/Gauss-Legendre inner integrals."""
    rq = Q.points(A[None])[0]
    aA = 0.5 * np.linalg.norm(np.cross(A[1] - A[0], A[2] - A[0]))
    aB = 0.5 * np.linalg.norm(np.cross(B[1] - B[0], B[2] - B[0]))
    wq = Q.weights(np.array([aA]))[0]
    inner = np.array([_duffy(r, B, lambda q: np.exp(-1j * k * np.linalg.norm(r - q, axis=-1))
                             / (4 * np.pi * np.linalg.norm(r - q, axis=-1)), n=n) for r in rq])
    return np.sum(wq * inner) / (aA * aB)


@pytest.mark.parametrize("case", ["self", "edge"])
def test_split_touching_pair_vs_brute_force(case):
    """Copper at 50 GHz (skin depth 0.30 um) on a 3.6 um triangle: the split rule
    matches brute force; the unsplit 6-point rule is off by tens of per cent."""
    k = copper_k(50e9)
    A = np.array([[0, 0, 0], [3.6e-6, 0, 0], [0.9e-6, 3.0e-6, 0]])
    if case == "self":
        B = A.copy()
        xyz = A
        tri = np.array([[0, 1, 2]])
        ta = tb = np.array([0])
    else:
        B = np.array([[3.6e-6, 0, 0], [0, 0, 0], [2.1e-6, -2.7e-6, 0.6e-6]])
        xyz = np.array([A[0], A[1], A[2], B[2]])
        tri = np.array([[0, 1, 2], [1, 0, 3]])
        ta, tb = np.array([0]), np.array([1])
    m = _Pair(xyz, tri)
    pts, w = fill.source_rule(B, k)
    assert len(w) >= 6 * 16
    ref = _lp_brute(k, A, B, n=200)
    _, lp = fill._L_pairs(m, k, ta, tb, (pts[None], w[None]))
    _, lp0 = fill._L_pairs(m, k, ta, tb)
    assert abs(lp[0] - ref) < 3e-4 * abs(ref), (lp[0], ref)
    assert abs(lp0[0] - ref) > 0.5 * abs(ref)


class _Pair:
    """The attributes of oracle.topology.Mesh that _L_pairs reads, for loose triangles."""

    def __init__(self, xyz, tri):
        self.xyz, self.tri = xyz, tri
        P = xyz[tri]
        self.area = 0.5 * np.linalg.norm(np.cross(P[:, 1] - P[:, 0], P[:, 2] - P[:, 0]), axis=1)

        class E:
            tri_sign = np.ones((len(tri), 3))
        self.E = E


def test_dropped_pairs_are_negligible():
    """Pairs beyond |Im k| R = 40 hold less than 1e-15 of the self term."""
    k = copper_k(50e9)
    v, f = icosphere(1, 15e-6)
    m = Mesh(v, f)
    P = m.xyz[m.tri]
    ta = np.repeat(np.arange(m.nt), m.nt)
    tb = np.tile(np.arange(m.nt), m.nt)
    keep = fill._kept(k, P[ta], P[tb], fill._touch_primal(m.tri, ta, tb))
    assert 0 < np.sum(~keep) < len(ta)
    drop = np.nonzero(~keep)[0][:40]

    def lp_of(a, b):
        pts, w = fill.source_rule(P[b], k)
        return fill._L_pairs(m, k, np.array([a]), np.array([b]), (pts[None], w[None]))[1][0]
    lp = np.array([lp_of(ta[i], tb[i]) for i in drop])
    assert np.max(np.abs(lp)) < 1e-15 * abs(lp_of(0, 0))


def _copper_sphere(split=True):
    """Copper sphere (icosphere sub 1, radius 6 um, edges 3.8 um) at 50 GHz: skin
    depth 0.30 um, source triangles split 4 times (barycentric ones 3 times)."""
    from oracle import system as S
    v, f = icosphere(1, 6e-6)
    m = Mesh(v, f)
    mat = S.Material(1.0, 1.0, 5.8e7)
    A = S.assemble(m, [mat], S.Material(), 50e9)
    b = S.rhs(A)
    x = S.solve(A, b)
    vol = abs(np.einsum('td,td->t', v[f[:, 0]], np.cross(v[f[:, 1]], v[f[:, 2]])).sum()) / 6
    return m, A, x, (3 * vol / (4 * np.pi)) ** (1 / 3), S.eps_c(mat, 2 * np.pi * 50e9)


def _absorbed(A, x):
    """Power into the object, 1/2 Re int (n x H)* . E_t, from the total surface fields:
    n x H = j / (j k0) in RWG, n x E = eta0 e in BC, int f_m . (b_n x n) = I_x[m, n]."""
    from oracle import system as S
    eta0 = MU0 * 299792458.0
    j, e, _ = S.split(A, x)
    return 0.5 * eta0 * np.real(np.conj(j / (1j * A.k0)) @ (A.Ix @ e))


def _mie_absorbed(k0, a, eps):
    from oracle import mie
    x = k0 * a
    n, an, bn = mie.coefficients(x, np.sqrt(np.conj(complex(eps))))
    qext = 2 / x ** 2 * np.sum((2 * n + 1) * np.real(an + bn))
    qsca = 2 / x ** 2 * np.sum((2 * n + 1) * (np.abs(an) ** 2 + np.abs(bn) ** 2))
    return (qext - qsca) * np.pi * a ** 2 / (2 * MU0 * 299792458.0)


@pytest.mark.slow
def test_copper_sphere_vs_mie(monkeypatch):
    """Skin-effect loss and scattering of a copper sphere against the Mie series of the
    equal-volume sphere; the same system without splitting loses 3/4 of the loss."""
    from oracle import farfield, mie, system as S
    m, A, x, a_eq, eps = _copper_sphere()
    p = _absorbed(A, x) / _mie_absorbed(A.k0, a_eq, eps)
    assert abs(p - 1) < 0.05, p
    th = np.radians(np.array([0, 45, 90, 135, 180.0]))
    s = farfield.rcs(m, A.k0, S.j_delta(A, x), th)
    assert np.max(np.abs(10 * np.log10(s / mie.rcs_eplane(A.k0, a_eq, eps, np.pi - th)))) < 0.15
    # planted mistake: no splitting
    monkeypatch.setattr(fill, "needs_split", lambda k, P: np.zeros(len(P), dtype=bool))
    m, A, x, a_eq, eps = _copper_sphere()
    assert _absorbed(A, x) / _mie_absorbed(A.k0, a_eq, eps) < 0.5
