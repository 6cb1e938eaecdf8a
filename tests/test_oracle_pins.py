"""Pins of the CPU oracle against facts fixed outside it: polynomial exactness of
the quadrature, brute-force integration, closed forms (Mie series, Rayleigh limit,
a published Mie sample), invariants of D/B/F and of the BC functions, Galerkin
symmetry and the transparent-object invariant of Sec. II (no scattering when an
object's material equals its background's)."""
import math
import os

import numpy as np
import pytest

from oracle import quadrature as Q
from oracle import singular, fill, system as S, farfield, mie
from oracle.topology import Mesh
from workloads.meshes import icosphere, ellipsoid, box, cylinder

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- quadrature
def test_dunavant_exact_to_degree_4():
    # reference triangle (0,0), (1,0), (0,1): int x^a y^b = a! b! / (a + b + 2)!
    tri = np.array([[[0.0, 0, 0], [1.0, 0, 0], [0.0, 1, 0]]])
    p = Q.points(tri)[0]
    w = Q.weights(np.array([0.5]))[0]
    for a in range(5):
        for b in range(5 - a):
            exact = math.factorial(a) * math.factorial(b) / math.factorial(a + b + 2)
            got = np.sum(w * p[:, 0] ** a * p[:, 1] ** b)
            assert abs(got - exact) < 1e-14, (a, b)
    # and not exact at degree 6 (the rule is the degree-4 one)
    got = np.sum(w * p[:, 0] ** 6)
    assert abs(got - math.factorial(6) / math.factorial(8)) > 1e-6


# ---------------------------------------------------------------- closed forms vs brute force
def _duffy(r, tri, fn, n=48):
    """Brute-force integral over a triangle: split at the projection of r, Duffy map, Gauss-Legendre."""
    nrm = np.cross(tri[1] - tri[0], tri[2] - tri[0])
    nrm /= np.linalg.norm(nrm)
    d = nrm @ (r - tri[0])
    rho = r - d * nrm
    x, w = np.polynomial.legendre.leggauss(n)
    x, w = 0.5 * (x + 1), 0.5 * w
    U, V = np.meshgrid(x, x, indexing="ij")
    WW = np.outer(w, w)
    tot = 0.0
    for a, b in ((tri[0], tri[1]), (tri[1], tri[2]), (tri[2], tri[0])):
        sa = 0.5 * np.cross(a - rho, b - rho) @ nrm
        q = rho + U[..., None] * ((1 - V)[..., None] * (a - rho) + V[..., None] * (b - rho))
        vals = fn(q)
        tot = tot + np.tensordot(WW * 2 * sa * U, vals, axes=([0, 1], [0, 1]))
    return tot


@pytest.mark.parametrize("r", [
    [0.3, 0.3, 0.5], [0.4, 0.3, 0.0], [2.0, -1.0, 0.3], [0.2, 0.25, 0.02], [-0.5, 0.4, -0.2]])
def test_closed_form_integrals_vs_brute_force(r):
    r = np.array(r, float)
    tri = np.array([[0, 0, 0], [1, 0.1, 0], [0.3, 0.9, 0.2]], float)
    I = singular.integrals(r[None], tri[None])
    R = lambda q: np.linalg.norm(r - q, axis=-1)
    nrm = I["n"][0]
    rho = I["rho"][0]
    chk = [
        (I["inv_r"][0], _duffy(r, tri, lambda q: 1 / R(q))),
        (I["r"][0], _duffy(r, tri, lambda q: R(q))),
        (I["p_over_r"][0], _duffy(r, tri, lambda q: (q - rho) / R(q)[..., None])),
        (I["p_r"][0], _duffy(r, tri, lambda q: (q - rho) * R(q)[..., None])),
    ]
    if abs(I["d"][0]) > 0.05:
        chk.append((I["grad_inv_r"][0], _duffy(r, tri, lambda q: -(r - q) / R(q)[..., None] ** 3, n=96)))
    for got, ref in chk:
        assert np.linalg.norm(np.atleast_1d(got - ref)) <= 1e-9 * np.linalg.norm(np.atleast_1d(ref))


def test_green_smooth_series_matches_direct():
    k = 3.0 - 0.2j
    R = np.array([0.011, 0.014, 0.016])  # |kR| on both sides of the series switch at 0.05
    direct = (np.exp(-1j * k * R) - 1) / (4 * np.pi * R) + k * k * R / (8 * np.pi)
    assert np.allclose(fill.green_smooth(k, R), direct, rtol=1e-9, atol=0)
    g = (1 - (1 + 1j * k * R) * np.exp(-1j * k * R)) / (4 * np.pi * R ** 3)
    assert np.allclose(fill.grad_green_smooth_factor(k, R), g, rtol=1e-7, atol=0)


@pytest.mark.parametrize("k,tol", [(0.05, 1e-10), (2.0, 1e-5), (1.0 - 0.5j, 1e-5)])
def test_touching_pair_inner_integral_vs_brute_force(k, tol):
    """L^phi self term of one triangle: the extracted inner integral agrees with brute
    force; what is left is the 6-point rule on the remainder, O((k h)^3)."""
    v, f = icosphere(1, 1.0)
    m = Mesh(v, f)
    la, lp = fill._L_pairs(m, k, np.array([0]), np.array([0]))
    tri = m.xyz[m.tri[0]]
    rq = Q.points(tri[None])[0]
    wq = Q.weights(m.area[:1])[0]
    inner = np.array([_duffy(r, tri, lambda q: np.exp(-1j * k * np.linalg.norm(r - q, axis=-1))
                             / (4 * np.pi * np.linalg.norm(r - q, axis=-1)), n=120) for r in rq])
    ref = np.sum(wq * inner) / m.area[0] ** 2
    assert abs(lp[0] - ref) < tol * abs(ref)


# ---------------------------------------------------------------- topology
@pytest.fixture(scope="module")
def mesh1():
    v, f = icosphere(1, 0.1)
    return Mesh(v, f)


def test_edges_and_incidence(mesh1):
    m = mesh1
    assert m.ne == 3 * m.nt // 2
    D = m.D()
    assert np.all(D.sum(axis=0) == 0)                       # 1^T D = 0 (charge neutrality)
    F, B = m.F(), m.B()
    assert np.linalg.matrix_rank(F @ D) == m.nt - 1
    assert np.allclose(F @ B, np.eye(m.nt - 1))
    assert np.allclose(np.ones(m.nt) @ B, 0)
    # divergence of RWG: +1/A+ on T+, -1/A- on T-  <=> unit flux
    for n in range(0, m.ne, 17):
        tp, ip = m.E.tp[n], m.E.ip[n]
        p = m.xyz[m.tri[tp]]
        a, b = p[(ip + 1) % 3], p[(ip + 2) % 3]
        mid = 0.5 * (a + b)
        fval = (mid - p[ip]) / (2 * m.area[tp])
        nu = np.cross(b - a, m.normal[tp])
        nu /= np.linalg.norm(nu)
        assert abs(fval @ nu * np.linalg.norm(b - a) - 1) < 1e-12


def test_bc_functions(mesh1):
    m = mesh1
    C = m.C.toarray()
    div = np.zeros((6 * m.nt, m.ne))
    for k in range(m.bE.ne):
        div[m.bE.tp[k]] += C[k]
        div[m.bE.tm[k]] -= C[k]
    deg = np.bincount(m.tri.ravel(), minlength=m.nv) // 1
    for n in range(m.ne):
        u, v = m.E.uv[n]
        kids_u = [c for c in range(6 * m.nt) if u in m.btri[c]]
        kids_v = [c for c in range(6 * m.nt) if v in m.btri[c]]
        assert np.allclose(div[kids_u, n], 1 / (2 * deg[u]))
        assert np.allclose(div[kids_v, n], -1 / (2 * deg[v]))
        rest = np.setdiff1d(np.arange(6 * m.nt), kids_u + kids_v)
        assert np.allclose(div[rest, n], 0)
    Ix = fill.fill_Ix(m)
    assert Ix.diagonal().min() > 0
    assert np.linalg.cond(Ix) < 10


def test_gram_bounded_under_refinement():
    conds = []
    for sub in (1, 2):
        v, f = icosphere(sub, 1.0)
        conds.append(np.linalg.cond(fill.fill_Ix(Mesh(v, f))))
    assert max(conds) < 10 and conds[1] < 2 * conds[0]


# ---------------------------------------------------------------- operator invariants
def test_galerkin_symmetry(mesh1):
    m = mesh1
    k = 2 * np.pi * 600e6 / fill.C0
    LA, LP = fill.fill_L(m, k, np.arange(m.nt))
    # entries between edges whose triangles do not touch use the same product rule both ways
    far_t = ~fill._touch_primal(m.tri, np.repeat(np.arange(m.nt), m.nt), np.tile(np.arange(m.nt), m.nt)).reshape(m.nt, m.nt)
    assert np.max(np.abs((LP - LP.T)[far_t])) <= 1e-13 * np.max(np.abs(LP))
    assert np.linalg.norm(LA - LA.T) <= 2e-3 * np.linalg.norm(LA)
    assert np.linalg.norm(LP - LP.T) <= 2e-3 * np.linalg.norm(LP)


def test_kbar_zero_for_coplanar_children(mesh1):
    m = mesh1
    loc = fill._K_pairs(m, 3.0, np.array([5] * 6), np.arange(30, 36))
    assert np.all(loc == 0)


def test_kbar_flat_touching_pair_vanishes():
    """On a flat face of a box, touching coplanar pairs give (numerically) zero Kbar."""
    v, f = box(1.0, 1.0, 1.0, 3, 3, 3)
    m = Mesh(v, f)
    t = 0
    same_plane = [s for s in range(m.nt) if abs(m.normal[s] @ m.normal[t] - 1) < 1e-12 and s != t]
    kids = np.array([6 * s + c for s in same_plane for c in range(6)])
    loc = fill._K_pairs(m, 1.5, np.full(len(kids), t), kids)
    assert np.max(np.abs(loc)) < 1e-15


# ---------------------------------------------------------------- Mie
def test_mie_published_sample():
    vals = {}
    for line in open(os.path.join(GOLDEN, "bhmie_sample.txt")):
        if line.strip() and not line.startswith("#"):
            k, v = line.split()
            vals[k] = float(v)
    x = 2 * np.pi * vals["radius"] / vals["wavelength"]
    n, a, b = mie.coefficients(x, complex(vals["m_re"], vals["m_im"]))
    qext = 2 / x ** 2 * np.sum((2 * n + 1) * np.real(a + b))
    qsca = 2 / x ** 2 * np.sum((2 * n + 1) * (np.abs(a) ** 2 + np.abs(b) ** 2))
    qback = abs(np.sum((2 * n + 1) * (-1.0) ** n * (a - b))) ** 2 / x ** 2
    assert abs(qext - vals["qext"]) < 1e-4 and abs(qsca - vals["qsca"]) < 1e-4 and abs(qback - vals["qback"]) < 1e-4
    qe, qs = mie.efficiencies(x, complex(vals["m_re"], vals["m_im"]))
    assert abs(qe - vals["qext"]) < 1e-4 and abs(qs - vals["qsca"]) < 1e-4


def test_mie_rayleigh_limit():
    k0, a, eps = 1.0, 1e-3, 4.0
    th = np.array([0.0, np.pi / 3])
    s = mie.rcs_eplane(k0, a, eps, th)
    ray = 4 * np.pi * k0 ** 4 * a ** 6 * abs((eps - 1) / (eps + 2)) ** 2 * np.cos(th) ** 2
    assert np.allclose(s, ray, rtol=1e-5)


@pytest.fixture(scope="module")
def sphere_cfg1():
    """Dielectric sphere, radius 0.1 m, eps_r 4, icosphere sub 2, 300 MHz (Sec. IV-A type)."""
    v, f = icosphere(2, 0.1)
    m = Mesh(v, f)
    A = S.assemble(m, [S.Material(4.0)], S.Material(), 300e6)
    b = S.rhs(A)
    x = S.solve(A, b)
    return m, A, b, x, v, f


@pytest.mark.slow
def test_sphere_rcs_vs_mie(sphere_cfg1):
    m, A, b, x, v, f = sphere_cfg1
    assert np.linalg.norm(A.Z @ x - b) <= 1e-12 * np.linalg.norm(b)
    th = np.radians(np.array([0, 20, 40, 60, 120, 140, 160, 180.0]))
    s = farfield.rcs(m, A.k0, S.j_delta(A, x), th)
    # faceted sphere: compare with the Mie sphere of equal volume (faceting at sub 2
    # removes 3.4 % of the volume, about -0.3 dB against the circumscribed sphere)
    vol = abs(np.einsum('td,td->t', v[f[:, 0]], np.cross(v[f[:, 1]], v[f[:, 2]])).sum()) / 6
    a_eq = (3 * vol / (4 * np.pi)) ** (1 / 3)
    s_eq = mie.rcs_eplane(A.k0, a_eq, 4.0, np.pi - th)
    s_true = mie.rcs_eplane(A.k0, 0.1, 4.0, np.pi - th)
    assert np.max(np.abs(10 * np.log10(s / s_eq))) < 0.06
    assert np.all(np.abs(10 * np.log10(s / s_true)) < 0.45)


@pytest.mark.slow
def test_continuity_row_holds(sphere_cfg1):
    """The computed charges satisfy F D (j - Y11 e) - k0^2 (q - Y21 e) = 0 (Eq. AEFIEextdis, row 2)."""
    m, A, b, x, *_ = sphere_cfg1
    j, e, u = S.split(A, x)
    r = m.F() @ m.D() @ (j - A.blocks[0]['Y11'] @ e) + A.k0 ** 2 * (u + A.blocks[0]['Y21'] @ e)
    assert np.linalg.norm(r) <= 1e-10 * np.linalg.norm(m.F() @ m.D() @ j)


def test_transparent_object_scatters_nothing():
    v, f = icosphere(1, 0.1)
    m = Mesh(v, f)
    bg = S.Material(2.0, 1.0, 0.0)
    A = S.assemble(m, [S.Material(2.0, 1.0, 0.0)], bg, 400e6)
    b = S.rhs(A)
    x = S.solve(A, b)
    j, e, _ = S.split(A, x)
    jd = S.j_delta(A, x)
    assert np.linalg.norm(jd) <= 1e-12 * np.linalg.norm(j)
    assert np.linalg.norm(A.Ix @ e - b[:m.ne]) <= 1e-12 * np.linalg.norm(b[:m.ne])


def test_multi_object_block_structure():
    """Two disjoint spheres: interior blocks are per object; only L_m couples them (Eq. Aobj)."""
    from workloads.meshes import merge
    xyz, tri, obj = merge(icosphere(1, 0.05, (0, 0, 0)), icosphere(1, 0.05, (0.2, 0, 0)))
    m = Mesh(xyz, tri, obj)
    A = S.assemble(m, [S.Material(3.0), S.Material(5.0)], S.Material(), 300e6)
    assert A.Z.shape[0] == 2 * m.ne + m.nt - 2
    b = S.rhs(A)
    x = S.solve(A, b)
    assert np.linalg.norm(A.Z @ x - b) <= 1e-12 * np.linalg.norm(b)
    # swapping the objects' order leaves the far field unchanged
    xyz2, tri2, obj2 = merge(icosphere(1, 0.05, (0.2, 0, 0)), icosphere(1, 0.05, (0, 0, 0)))
    m2 = Mesh(xyz2, tri2, obj2)
    A2 = S.assemble(m2, [S.Material(5.0), S.Material(3.0)], S.Material(), 300e6)
    x2 = S.solve(A2, S.rhs(A2))
    th = np.radians([0.0, 45.0, 135.0])
    s1 = farfield.rcs(m, A.k0, S.j_delta(A, x), th)
    s2 = farfield.rcs(m2, A2.k0, S.j_delta(A2, x2), th)
    assert np.allclose(s1, s2, rtol=1e-9)
