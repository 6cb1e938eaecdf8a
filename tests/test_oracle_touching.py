"""Pair-level pins of the oracle's touching-pair branches (Sec. II-B, singularity
extraction on self and adjacent pairs) against brute-force quadrature.

For a touching pair the oracle integrates the inner (source) integral of the
static terms in closed form and the remainder with the 6-point rule.  Here the
inner integral is instead computed by brute force (the triangle split at the
projection of the observation point, Duffy map, 120 x 120 Gauss-Legendre) at
the same 6 outer points, straight from the definitions

    L^A[i, j]   = int f_i(r) . int f_j(r') G(R) dS' dS,      f = s (r - p) / (2 A)
    L^phi       = int int G(R) dS' dS / (A A')
    Kbar[i, j]  = int f_i(r) . int grad_r G(R) x g_j(r') dS' dS,
                  grad_r G = -(1 + j k R) exp(-j k R) (r - r') / (4 pi R^3),

so the comparison checks the closed-form combination of every vector term (the
(rho - w) shift of L^A, the (r - w) form of the static Kbar cross product) and
the remainder rule together.  At small |k| h the remainder's quadrature error is
negligible (the pins are at 1e-10); at |k| h ~ 1 it is the 6-point rule's
O((k h)^4) error.  Planted mistakes in the closed forms fail these pins.
"""
import numpy as np
import pytest

from oracle import fill, quadrature as Q, singular
from oracle.topology import Mesh
from workloads.meshes import icosphere

from test_oracle_pins import _duffy


@pytest.fixture(scope="module")
def m1():
    v, f = icosphere(1, 1.0)
    return Mesh(v, f)


def _shared(m, a, b):
    return len(set(m.tri[a]) & set(m.tri[b]))


def _la_brute(m, k, a, b, n=120):
    A, B = m.xyz[m.tri[a]], m.xyz[m.tri[b]]
    rq = Q.points(A[None])[0]
    wq = Q.weights(m.area[[a]])[0]
    sa, sb = m.E.tri_sign[a], m.E.tri_sign[b]
    la = np.zeros((3, 3), complex)
    lp = 0.0
    for q in range(6):
        r = rq[q]

        def G(p):
            R = np.linalg.norm(r - p, axis=-1)
            return np.exp(-1j * k * R) / (4 * np.pi * R)

        lp += wq[q] * _duffy(r, B, G, n=n)
        for j in range(3):
            inner = _duffy(r, B, lambda p: sb[j] * (p - B[j]) / (2 * m.area[b]) * G(p)[..., None], n=n)
            for i in range(3):
                la[i, j] += wq[q] * (sa[i] * (r - A[i]) / (2 * m.area[a])) @ inner
    return la, lp / (m.area[a] * m.area[b])


def _kbar_brute(m, k, a, c, n=120):
    A, Bt = m.xyz[m.tri[a]], m.bxyz[m.btri[c]]
    rq = Q.points(A[None])[0]
    wq = Q.weights(m.area[[a]])[0]
    sa, sb = m.E.tri_sign[a], m.bE.tri_sign[c]
    out = np.zeros((3, 3), complex)
    for q in range(6):
        r = rq[q]

        def grad_g(p):
            d = r - p
            R = np.linalg.norm(d, axis=-1)
            return (-(1 + 1j * k * R) * np.exp(-1j * k * R) / (4 * np.pi * R ** 3))[..., None] * d

        for j in range(3):
            inner = _duffy(r, Bt, lambda p: np.cross(grad_g(p), sb[j] * (p - Bt[j]) / (2 * m.barea[c])), n=n)
            for i in range(3):
                out[i, j] += wq[q] * (sa[i] * (r - A[i]) / (2 * m.area[a])) @ inner
    return out


def _pairs_L(m):
    """Triangle 0 with itself, an edge-adjacent and a vertex-adjacent triangle."""
    edge = next(t for t in range(m.nt) if t != 0 and _shared(m, 0, t) == 2)
    vert = next(t for t in range(m.nt) if _shared(m, 0, t) == 1)
    return [0, edge, vert]


@pytest.mark.parametrize("k,tol", [(0.05, 1e-10), (2.0, 3e-5)])
def test_LA_touching_block_vs_brute_force(m1, k, tol):
    for b in _pairs_L(m1):
        la, lp = fill._L_pairs(m1, k, np.array([0]), np.array([b]))
        bf, bp = _la_brute(m1, k, 0, b)
        assert np.max(np.abs(la[0] - bf)) <= tol * np.max(np.abs(bf)), b
        assert abs(lp[0] - bp) <= tol * abs(bp), b


def _touching_children(m):
    kind = fill._touch_bary(m, np.zeros(6 * m.nt, np.int64), np.arange(6 * m.nt))
    near = np.nonzero(kind == 1)[0]
    # children of non-coplanar neighbours touching at a vertex or at a test-edge midpoint
    return near[::5]


@pytest.mark.parametrize("k,tol", [(1e-3, 2e-10), (0.5, 3e-5)])
def test_Kbar_touching_noncoplanar_vs_brute_force(m1, k, tol):
    kids = _touching_children(m1)
    assert len(kids) >= 5 and np.all(m1.bparent[kids] != 0)
    for c in kids:
        got = fill._K_pairs(m1, k, np.array([0]), np.array([c]))[0]
        bf = _kbar_brute(m1, k, 0, c)
        assert np.max(np.abs(got - bf)) <= tol * np.max(np.abs(bf)), c


@pytest.mark.parametrize("term", ["p_over_r", "rho", "grad_inv_r"])
def test_planted_closed_form_mistakes_are_caught(m1, monkeypatch, term):
    """A sign slip in a closed-form vector term of the oracle breaks the pins above."""
    real = singular.integrals

    def broken(r, tri):
        out = dict(real(r, tri))
        out[term] = -out[term]
        return out

    monkeypatch.setattr(fill, "integrals", broken)
    if term == "grad_inv_r":
        c = _touching_children(m1)[0]
        got = fill._K_pairs(m1, 1e-3, np.array([0]), np.array([c]))[0]
        bf = _kbar_brute(m1, 1e-3, 0, c, n=60)
    else:
        b = _pairs_L(m1)[1]
        got = fill._L_pairs(m1, 0.05, np.array([0]), np.array([b]))[0][0]
        bf = _la_brute(m1, 0.05, 0, b, n=60)[0]
    assert np.max(np.abs(got - bf)) > 1e-3 * np.max(np.abs(bf))


def test_LA_galerkin_symmetry_far_entries(m1):
    """Entries between edges none of whose triangles touch use the same product
    rule both ways, so L^A is complex symmetric there to rounding."""
    m = m1
    k = 2 * np.pi * 600e6 / fill.C0 * 10.0  # |k| h ~ 1 on the unit sphere
    LA, LP = fill.fill_L(m, k, np.arange(m.nt))
    touch_t = fill._touch_primal(m.tri, np.repeat(np.arange(m.nt), m.nt),
                                 np.tile(np.arange(m.nt), m.nt)).reshape(m.nt, m.nt)
    sup = np.stack([m.E.tp, m.E.tm], axis=1)                     # (ne, 2) triangles of each edge
    far_e = ~(touch_t[sup[:, 0]][:, sup[:, 0]] | touch_t[sup[:, 0]][:, sup[:, 1]]
              | touch_t[sup[:, 1]][:, sup[:, 0]] | touch_t[sup[:, 1]][:, sup[:, 1]])
    assert far_e.sum() > 0.5 * m.ne ** 2
    assert np.max(np.abs((LA - LA.T)[far_e])) <= 1e-13 * np.max(np.abs(LA))
    assert np.max(np.abs((LP - LP.T)[~touch_t])) <= 1e-13 * np.max(np.abs(LP))
