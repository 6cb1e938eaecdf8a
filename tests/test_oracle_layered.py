"""Pins of the layered-medium oracle (external problem in a stratified background):
exact images over a PEC ground, reduction to the homogeneous kernel for identical
layers, the electrostatic image limit over a dielectric half-space, the tabulated
remainder against direct Sommerfeld integration, plane-wave transfer through a
stack, and the full system over a PEC ground against the sphere + image-sphere
pair in free space."""
import numpy as np
import pytest

from oracle import layered as LY
from oracle import system as S
from oracle.fill import C0
from oracle.topology import Mesh
from workloads.meshes import icosphere, merge

F = 1e9
W = 2 * np.pi * F
K0 = W / C0
LAM = C0 / F


def G(k, R):
    return np.exp(-1j * k * R) / (4 * np.pi * R)


def test_pec_ground_gives_exact_images():
    st = LY.Stack([(1.0, 1.0, 0.0, np.inf)], z_top=0.0, bottom="pec")
    z, zp = 0.3 * LAM, 0.1 * LAM
    rho = np.array([0.05, 0.3, 1.0]) * LAM
    full = LY.spatial_full(st, 0, W, rho, z, zp)
    R0, R2 = np.sqrt(rho ** 2 + (z - zp) ** 2), np.sqrt(rho ** 2 + (z + zp) ** 2)
    ref = {"xx": G(K0, R0) - G(K0, R2), "phi": G(K0, R0) - G(K0, R2), "zz": G(K0, R0) + G(K0, R2),
           "zr": 0 * rho, "rz": 0 * rho}
    scale = np.abs(G(K0, R0)).max()
    for c in LY.COMPONENTS:
        assert np.abs(full[c] - ref[c]).max() < 1e-12 * scale, c


def test_identical_layers_reduce_to_homogeneous():
    eps = 2.5
    st = LY.Stack([(eps, 1.0, 0.0, np.inf), (eps, 1.0, 0.0, 0.2 * LAM), (eps, 1.0, 0.0, np.inf)], z_top=0.0)
    z, zp = -0.05 * LAM, -0.15 * LAM
    rho = np.array([0.05, 0.5]) * LAM
    full = LY.spatial_full(st, 1, W, rho, z, zp)
    k = K0 * np.sqrt(eps)
    R0 = np.sqrt(rho ** 2 + (z - zp) ** 2)
    assert np.allclose(full["xx"], G(k, R0), rtol=1e-10, atol=0)
    assert np.allclose(full["zz"], G(k, R0), rtol=1e-10, atol=0)
    assert np.allclose(full["phi"], G(k, R0) / eps, rtol=1e-10, atol=0)
    assert np.abs(full["zr"]).max() < 1e-12 * np.abs(G(k, R0)).max()
    Gue, Guh, Gde, Gdh = LY.reflections(st, 1, W, np.array([0.3 * k, 2 * k + 0.1j]))
    assert np.all(np.abs(np.concatenate([Gue, Guh, Gde, Gdh])) < 1e-14)


def test_static_image_over_dielectric_halfspace():
    """As k -> 0 the scalar-potential kernel tends to the electrostatic image (e1-e2)/(e1+e2)."""
    f = 1e3
    w = 2 * np.pi * f
    e1, e2 = 1.0, 6.0
    st = LY.Stack([(e1, 1.0, 0.0, np.inf), (e2, 1.0, 0.0, np.inf)], z_top=0.0)
    z, zp = 0.3, 0.1
    rho = np.array([0.05, 0.4, 1.5])
    full = LY.spatial_full(st, 0, w, rho, z, zp)
    R0, R2 = np.sqrt(rho ** 2 + (z - zp) ** 2), np.sqrt(rho ** 2 + (z + zp) ** 2)
    stat = (1 / R0 + (e1 - e2) / (e1 + e2) / R2) / (4 * np.pi * e1)
    # dynamic corrections are O(k0 R) ~ 1e-5 at 1 kHz; a wrong image coefficient misses by O(1)
    assert np.allclose(full["phi"].real, stat, rtol=1e-4)


def test_tabulated_remainder_against_direct_sommerfeld():
    st = LY.Stack([(1.0, 1.0, 0.0, np.inf), (4.0, 1.0, 0.0, 0.1 * LAM), (11.9, 1.0, 0.1, np.inf)], z_top=0.0)
    layer = 1
    zmin, zmax = -0.07 * LAM, -0.03 * LAM
    T = LY.build_tables(st, layer, W, 1e-3 * LAM, 0.6 * LAM, zmin, zmax)
    k = K0 * 2.0
    for z, zp in [(-0.04 * LAM, -0.06 * LAM), (-0.065 * LAM, -0.035 * LAM)]:
        rho = np.array([0.03, 0.15, 0.5]) * LAM
        full = LY.spatial_full(st, layer, W, rho, z, zp)
        R0 = np.sqrt(rho ** 2 + (z - zp) ** 2)
        im = LY.images(st, layer, W, rho, z, zp)
        rm = LY.remainder(T, rho, z, zp)
        direct = {"xx": G(k, R0), "phi": G(k, R0) / 4.0, "zz": G(k, R0), "zr": 0, "rz": 0}
        for c in LY.COMPONENTS:
            tot = direct[c] + im.get(c, 0) + rm[c]
            # the default 256 x 128 bilinear tables reproduce the kernels to a few 1e-4
            assert np.abs(tot - full[c]).max() <= 2e-3 * np.abs(full[c]).max(), c


def test_plane_wave_through_stack():
    # PEC ground: standing wave exp(+j k z) - exp(-j k z)
    st = LY.Stack([(1.0, 1.0, 0.0, np.inf)], z_top=0.0, bottom="pec")
    a, c, k, zref = LY.plane_wave_normal(st, 0, W)
    assert abs(a - 1) < 1e-14 and abs(c + 1) < 1e-14
    # dielectric half-space: Fresnel reflection and power balance
    n = 2.0
    st = LY.Stack([(1.0, 1.0, 0.0, np.inf), (n * n, 1.0, 0.0, np.inf)], z_top=0.0)
    a, c, k, zref = LY.plane_wave_normal(st, 0, W)
    r = (1 / n - 1) / (1 / n + 1)
    assert abs(c / a - r) < 1e-14
    a1, c1, k1, _ = LY.plane_wave_normal(st, 1, W)
    assert abs(c1) < 1e-14 and abs(abs(r) ** 2 + n * abs(a1) ** 2 - 1) < 1e-12
    # lossless slab over PEC: total reflection, unit magnitude
    st = LY.Stack([(1.0, 1.0, 0.0, np.inf), (3.0, 1.0, 0.0, 0.13 * LAM)], z_top=0.0, bottom="pec")
    a, c, k, zref = LY.plane_wave_normal(st, 0, W)
    assert abs(abs(c / a) - 1) < 1e-12


def test_sphere_over_pec_equals_image_pair_in_free_space():
    f, h, rad = 300e6, 0.15, 0.1
    v, fc = icosphere(1, rad, (0.0, 0.0, h))
    m = Mesh(v, fc)
    st = LY.Stack([(1.0, 1.0, 0.0, np.inf)], z_top=0.0, bottom="pec")
    A = S.assemble(m, [S.Material(4.0)], st, f, layer=0)
    x = S.solve(A, S.rhs(A))
    vi = v.copy()
    vi[:, 2] *= -1
    xyz, tri, obj = merge((v, fc), (vi, fc[:, ::-1].copy()))
    m2 = Mesh(xyz, tri, obj)
    A2 = S.assemble(m2, [S.Material(4.0)] * 2, S.Material(), f)
    x2 = S.solve(A2, S.rhs(A2, khat=(0, 0, -1)) - S.rhs(A2, khat=(0, 0, 1)))
    ne, nt = m.ne, m.nt
    for a_, b_ in ((x[:ne], x2[:ne]), (x[ne:2 * ne], x2[m2.ne:m2.ne + ne]), (x[2 * ne:], x2[2 * m2.ne:2 * m2.ne + nt - 1])):
        assert np.linalg.norm(a_ - b_) <= 1e-11 * np.linalg.norm(b_)


def _curl(fun, r, h=1e-6):
    """curl of a vector field by central differences (fun: (n,3) -> (n,3))."""
    J = np.zeros((3, 3), complex)   # J[i, j] = d E_i / d x_j
    for j in range(3):
        e = np.zeros(3)
        e[j] = h
        J[:, j] = (fun(np.array([r + e]))[0] - fun(np.array([r - e]))[0]) / (2 * h)
    return np.array([J[2, 1] - J[1, 2], J[0, 2] - J[2, 0], J[1, 0] - J[0, 1]])


OBLIQUE_STACK = LY.Stack([(1.0, 1.0, 0.0, np.inf), (4.0, 1.0, 0.0, 0.2 * LAM),
                          (2.5, 2.0, 0.0, 0.07 * LAM), (11.9, 1.0, 0.05, np.inf)], z_top=0.1 * LAM)


def _oblique(theta, phi):
    th, ph = np.radians(theta), np.radians(phi)
    khat = np.array([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), -np.cos(th)])
    e_te = np.array([-np.sin(ph), np.cos(ph), 0.0])
    e_tm = np.cross(e_te, khat)
    return khat, e_te, e_tm


@pytest.mark.parametrize("bottom", ["halfspace", "pec"])
def test_oblique_wave_meets_interface_conditions(bottom):
    """Oblique incidence through a lossy, magnetic stack: across every interface
    the tangential E, the normal eps E and the tangential H = curl E / (-j w mu)
    are continuous; on a PEC ground the tangential E vanishes; inside each
    layer E is divergence-free (so the z part of the TM wave is right)."""
    layers = list(OBLIQUE_STACK.layers)
    if bottom == "pec":  # every layer below the upper half-space finite, a PEC under the last
        layers[-1] = (11.9, 1.0, 0.05, 0.11 * LAM)
    st = LY.Stack(layers, OBLIQUE_STACK.z_top, bottom)
    khat, e_te, e_tm = _oblique(40.0, 25.0)
    pol = (0.6 * e_te + 0.8j * e_tm)
    L = len(st.layers)
    zs = [st.bounds(i)[0] for i in range(L - 1)] if bottom == "halfspace" else [st.bounds(i)[0] for i in range(L)]
    xy = np.array([0.11, -0.07]) * LAM
    for i, z in enumerate(zs):
        r = np.array([xy[0], xy[1], z])
        fa = lambda p, i=i: LY.incident_field(st, i, W, khat, pol, p)
        Ea = fa(np.array([r]))[0]
        Ha = _curl(fa, r) / (-1j * W * LY.MU0 * st.mu(i))
        if i == L - 1:  # PEC under the last layer
            assert np.abs(Ea[:2]).max() < 1e-12
            continue
        fb = lambda p, i=i: LY.incident_field(st, i + 1, W, khat, pol, p)
        Eb = fb(np.array([r]))[0]
        Hb = _curl(fb, r) / (-1j * W * LY.MU0 * st.mu(i + 1))
        assert np.abs(Ea[:2] - Eb[:2]).max() < 1e-12
        assert abs(st.eps(i, W) * Ea[2] - st.eps(i + 1, W) * Eb[2]) < 1e-12 * abs(st.eps(i + 1, W))
        assert np.abs(Ha[:2] - Hb[:2]).max() < 1e-7 * np.abs(Ha).max()
    for i in range(L):
        zb, zu = st.bounds(i)
        z = zu - 0.03 * LAM if np.isfinite(zu) else zb + 0.05 * LAM
        r = np.array([0.02 * LAM, 0.05 * LAM, z])
        div = 0j
        for j in range(3):
            e = np.zeros(3)
            e[j] = 1e-6
            div += (LY.incident_field(st, i, W, khat, pol, np.array([r + e]))[0][j]
                    - LY.incident_field(st, i, W, khat, pol, np.array([r - e]))[0][j]) / 2e-6
        assert abs(div) < 1e-6 * K0


def test_oblique_reduces_to_normal_and_free_space():
    st = OBLIQUE_STACK
    pts = lambda i: np.array([[0.1, 0.2, st.bounds(i)[1] - 0.01 * LAM if i else st.z_top + 0.3 * LAM]])
    # theta = 0: the normal-incidence transfer of the x polarisation
    for i in range(len(st.layers)):
        E = LY.incident_field(st, i, W, [0, 0, -1.0], [1.0, 0, 0], pts(i))[0]
        a, c, k, zref = LY.plane_wave_normal(st, i, W)
        z = pts(i)[0, 2]
        assert abs(E[0] - (a * np.exp(1j * k * (z - zref)) + c * np.exp(-1j * k * (z - zref)))) < 1e-13
        assert abs(E[1]) < 1e-14 and abs(E[2]) < 1e-14
    # identical layers: the free-space wave itself
    same = LY.Stack([(1.0, 1.0, 0.0, np.inf), (1.0, 1.0, 0.0, 0.2 * LAM), (1.0, 1.0, 0.0, np.inf)], z_top=0.0)
    khat, e_te, e_tm = _oblique(63.0, -110.0)
    pol = 0.3 * e_te - 0.4j * e_tm
    r = np.array([[0.3, -0.2, 0.4], [0.1, 0.1, -0.1], [-0.2, 0.5, -0.9]]) * LAM
    for i, p in zip((0, 1, 2), r):
        E = LY.incident_field(same, i, W, khat, pol, p[None])[0]
        assert np.abs(E - pol * np.exp(-1j * K0 * khat @ p)).max() < 1e-13


def test_oblique_fresnel_and_brewster():
    """Air over glass: the reflected TE / TM amplitudes are the Fresnel
    coefficients (transverse E convention), zero for TM at Brewster's angle
    tan theta_B = n, and the power balance |r|^2 + Re(k_z2 / k_z1 ...) |t|^2 = 1."""
    n = 1.5
    st = LY.Stack([(1.0, 1.0, 0.0, np.inf), (n * n, 1.0, 0.0, np.inf)], z_top=0.0)
    for theta in (0.0, 30.0, np.degrees(np.arctan(n)), 75.0):
        khat, e_te, e_tm = _oblique(theta, 10.0)
        ct = np.cos(np.radians(theta))
        ct2 = np.sqrt(1 - (np.sin(np.radians(theta)) / n) ** 2)
        lay, _ = LY.plane_wave_oblique(st, W, khat, e_te)
        r_te = (ct - n * ct2) / (ct + n * ct2)
        assert abs(lay[0]["c_te"] / lay[0]["a_te"] - r_te) < 1e-14
        t = lay[1]["a_te"] / lay[0]["a_te"]
        assert abs(abs(r_te) ** 2 + n * ct2 / ct * abs(t) ** 2 - 1) < 1e-13
        lay, _ = LY.plane_wave_oblique(st, W, khat, e_tm)
        r_tm = (ct2 / n - ct) / (ct2 / n + ct)  # Z = k_z / (w eps): (Z2 - Z1) / (Z2 + Z1)
        assert abs(lay[0]["c_tm"] / lay[0]["a_tm"] - r_tm) < 1e-14
        if abs(theta - np.degrees(np.arctan(n))) < 1e-9:
            assert abs(lay[0]["c_tm"]) < 1e-14


def test_oblique_sphere_over_pec_equals_image_pair():
    """A sphere over a PEC ground lit at 35 degrees (TE + TM mixed) solves like the
    sphere and its mirror image in free space lit by the incident wave plus its
    mirror wave (k_z and the tangential E reversed, the normal E kept)."""
    f, h, rad = 300e6, 0.15, 0.1
    v, fc = icosphere(1, rad, (0.0, 0.0, h))
    m = Mesh(v, fc)
    st = LY.Stack([(1.0, 1.0, 0.0, np.inf)], z_top=0.0, bottom="pec")
    khat, e_te, e_tm = _oblique(35.0, 20.0)
    pol = 0.8 * e_te + 0.6j * e_tm
    A = S.assemble(m, [S.Material(4.0)], st, f, layer=0)
    x = S.solve(A, S.rhs(A, khat=khat, pol=pol))
    vi = v.copy()
    vi[:, 2] *= -1
    xyz, tri, obj = merge((v, fc), (vi, fc[:, ::-1].copy()))
    m2 = Mesh(xyz, tri, obj)
    A2 = S.assemble(m2, [S.Material(4.0)] * 2, S.Material(), f)
    mirror = np.array([1.0, 1.0, -1.0])
    x2 = S.solve(A2, S.rhs(A2, khat=khat, pol=pol) + S.rhs(A2, khat=khat * mirror, pol=-pol * mirror))
    ne, nt = m.ne, m.nt
    for a_, b_ in ((x[:ne], x2[:ne]), (x[ne:2 * ne], x2[m2.ne:m2.ne + ne]), (x[2 * ne:], x2[2 * m2.ne:2 * m2.ne + nt - 1])):
        assert np.linalg.norm(a_ - b_) <= 1e-11 * np.linalg.norm(b_)


# ----------------------------------------------------------------------------- objects resting on an interface
def _resting_cylinder(zI, up=True):
    """A 240-triangle cylinder (r = 0.1 lam, h = 0.15 lam) whose base (up) or top
    (not up) lies on the plane z = zI."""
    from workloads.meshes import cylinder
    h = 0.15 * LAM
    v, f = cylinder(0.1 * LAM, h, center=(0.0, 0.0, zI if up else zI - h))
    return Mesh(v, f)


def _brute_image_pair(m, st, l, a, b, plane, n=40):
    """One interface's image terms of pair (a, b) straight from images() on the
    original source triangle: inner integrals by a 40 x 40 Duffy rule centred at the
    point of b nearest to the mirror of each outer point."""
    from oracle import quadrature as Q
    zb, zu = st.bounds(l)
    zI = zb if plane == "bottom" else zu
    A, B = m.xyz[m.tri[a]], m.xyz[m.tri[b]]
    rq, wq = Q.points(A[None])[0], Q.weights(m.area[[a]])[0]
    sa, sb = m.E.tri_sign[a] / (2 * m.area[a]), m.E.tri_sign[b] / (2 * m.area[b])
    la = np.zeros((3, 3), complex)
    lp = 0j
    for q in range(6):
        r = rq[q]
        rm = np.array([r[0], r[1], 2 * zI - r[2]])
        pts, wts = LY.duffy_rule(rm, B, n)
        dv = r - pts
        rho = np.hypot(dv[:, 0], dv[:, 1])
        im = LY.images(st, l, W, rho, r[2], pts[:, 2], use_top=float(plane == "top"), use_bot=float(plane == "bottom"))
        with np.errstate(invalid="ignore", divide="ignore"):
            rh = np.where(rho[:, None] > 0, dv[:, :2] / rho[:, None], 0.0)
        fa = sa[:, None] * (r - A)                                          # (3i, 3)
        for j in range(3):
            fb = sb[j] * (pts - B[j])                                       # (M, 3)
            Vx = im["xx"][:, None] * fb[:, :2] + im["rz"][:, None] * rh * fb[:, 2:3]
            Vz = im["zz"] * fb[:, 2] + im["zr"] * np.einsum('md,md->m', rh, fb[:, :2])
            V = np.concatenate([(wts[:, None] * Vx).sum(0), [(wts * Vz).sum()]])
            la[:, j] += wq[q] * fa @ V
        lp += wq[q] * (wts * im["phi"]).sum()
    return la, lp / (m.area[a] * m.area[b])


def _touch_classes(m, zI):
    """Triangles with all three / two / one vertices on z = zI."""
    tol = 1e-9 * LAM
    on = np.abs(m.xyz[:, 2] - zI) <= tol
    cnt = on[m.tri].sum(axis=1)
    return [np.nonzero(cnt == c)[0] for c in (3, 2, 1)]


@pytest.mark.parametrize("plane", ["bottom", "top"])
def test_touch_image_against_brute_force(plane):
    """The images of a pair touching through an interface (closed forms over the
    mirrored triangle, Duffy rule for the static z-rho terms) against the same
    kernels from images() integrated over the original source triangle by a fine
    Duffy rule, for every kind of touch: coincident cap triangles on the interface,
    caps sharing an edge or a vertex, a side triangle meeting a cap at an edge on
    the interface, side triangles meeting at a vertex on it.  The slab is magnetic
    so that both the TE and TM statics enter."""
    st = LY.Stack([(1.0, 1.0, 0.0, np.inf), (4.0, 1.5, 0.0, 0.4 * LAM), (11.9, 1.0, 0.0, np.inf)], z_top=0.0)
    l = 1
    zI = -0.4 * LAM if plane == "bottom" else 0.0
    m = _resting_cylinder(zI, up=(plane == "bottom"))
    cap, side2, side1 = _touch_classes(m, zI)
    tri = m.tri
    share = lambda a, b: len(set(tri[a]) & set(tri[b]))
    pairs = [(cap[0], cap[0])]
    pairs.append((cap[0], next(b for b in cap if b != cap[0] and share(cap[0], b) == 2)))
    pairs.append((cap[0], next(b for b in cap if share(cap[0], b) == 1)))
    s2 = next(a for a in side2 if any(share(a, c) == 2 for c in cap))
    c2 = next(c for c in cap if share(s2, c) == 2)
    pairs += [(s2, c2), (c2, s2), (s2, s2)]
    s1 = next(a for a in side1 if share(a, s2) >= 1)
    pairs += [(s1, s1), (s2, s1), (s1, s2)]
    ta = np.array([p[0] for p in pairs])
    tb = np.array([p[1] for p in pairs])
    t_top, t_bot = LY.touch_masks(m, st, l, ta, tb)
    assert (t_bot if plane == "bottom" else t_top).all() and not (t_top if plane == "bottom" else t_bot).any()
    la, lp = LY.touch_image(m, st, l, W, ta, tb, plane)
    for p, (a, b) in enumerate(pairs):
        bl, bp = _brute_image_pair(m, st, l, a, b, plane)
        scale = np.abs(bl).max()
        assert np.abs(la[p] - bl).max() <= 2e-6 * scale, (a, b, np.abs(la[p] - bl).max() / scale)
        assert abs(lp[p] - bp) <= 2e-6 * abs(bp), (a, b, abs(lp[p] - bp) / abs(bp))


def test_table_on_the_interface_against_fine_sommerfeld():
    """An object resting on glass: the remainder table's row on the interface
    (z + z' = 2 z_b, where nothing decays exponentially), at its rho nodes, against
    the same spectral remainder integrated with a tail 20 times longer; and off the
    interface the images + interpolated remainder still reproduce the full
    Sommerfeld kernel."""
    st = LY.Stack([(1.0, 1.0, 0.0, np.inf), (2.25, 1.0, 0.0, np.inf)], z_top=0.0)
    h = 0.3 * LAM
    T = LY.build_tables(st, 0, W, 1e-3 * LAM, 2 * LAM, 0.0, h)
    ir = np.array([0, 60, 120, 180, 255])      # table nodes: the tail cut alone, no interpolation
    rho = T.rho[ir]
    nodes, w = LY.sommerfeld_nodes(st, 0, W, 2 * LAM, h / 16 / 20)
    sp = LY.spectral(st, 0, W, nodes, s=0.0, part="A")
    rm = {c: T.A[c][ir, 0] for c in LY.COMPONENTS}
    for c in LY.COMPONENTS:
        v = LY.transform(sp[c][:, None], nodes, w, rho, LY.ORDER[c])[:, 0]
        ref = -1j * v if LY.ORDER[c] == 1 else v
        scale = np.abs(T.A[c]).max()
        assert np.abs(rm[c] - ref).max() <= 1e-3 * scale, (c, np.abs(rm[c] - ref).max() / scale)
    z, zp = 0.1 * LAM, 0.02 * LAM
    rho = np.array([0.03, 0.2, 0.8]) * LAM
    full = LY.spatial_full(st, 0, W, rho, z, zp)
    im = LY.images(st, 0, W, rho, z, zp)
    rm = LY.remainder(T, rho, z, zp)
    R0 = np.sqrt(rho ** 2 + (z - zp) ** 2)
    direct = {"xx": G(K0, R0), "phi": G(K0, R0), "zz": G(K0, R0), "zr": 0, "rz": 0}
    for c in LY.COMPONENTS:
        tot = direct[c] + im[c] + rm[c]
        assert np.abs(tot - full[c]).max() <= 2e-3 * np.abs(full[c]).max(), c


def test_resting_cylinder_blocks_are_reciprocal():
    """A cylinder resting on glass: the reflected L^A_m and L^phi_m are complex
    symmetric (reciprocity; the z-rho and rho-z images pair up): to rounding where
    no pair touches through the interface (the product rule is the same both ways),
    and in norm to the accuracy of the touching-pair rule (closed-form inner, 6-point
    outer integral, as for the direct term).  The transparent object (eps = air)
    leaves the incident field unscattered (J_Delta = 0)."""
    st = LY.Stack([(1.0, 1.0, 0.0, np.inf), (2.25, 1.0, 0.0, np.inf)], z_top=0.0)
    m = _resting_cylinder(0.0)
    T = S.default_tables(m, st, 0, W)
    LA, LP = LY.fill_reflected(m, st, 0, W, T, np.arange(m.nt))
    ta, tb = np.repeat(np.arange(m.nt), m.nt), np.tile(np.arange(m.nt), m.nt)
    touch = LY.touch_masks(m, st, 0, ta, tb)[1].reshape(m.nt, m.nt)
    assert touch.any()
    assert np.max(np.abs((LP - LP.T)[~touch])) <= 1e-13 * np.max(np.abs(LP))
    e_touch = np.zeros((m.ne, m.ne), dtype=bool)
    for a, b in zip(*np.nonzero(touch)):
        e_touch[np.ix_(m.E.tri_edge[a], m.E.tri_edge[b])] = True
    assert np.max(np.abs((LA - LA.T)[~(e_touch | e_touch.T)])) <= 1e-13 * np.max(np.abs(LA))
    assert np.linalg.norm(LA - LA.T) <= 2e-3 * np.linalg.norm(LA)
    assert np.linalg.norm(LP - LP.T) <= 2e-3 * np.linalg.norm(LP)
    A = S.assemble(m, [S.Material(1.0)], st, F, layer=0, tables=T)
    x = S.solve(A, S.rhs(A, khat=[np.sin(0.3), 0, -np.cos(0.3)], pol=[0, 1.0, 0]))
    assert np.linalg.norm(S.j_delta(A, x)) <= 1e-9 * np.linalg.norm(x[:m.ne])


def test_layered_rcs_reductions():
    """The far field above a stack: identical layers give the free-space RCS, and
    a sphere over a PEC ground radiates in the upper half-space like the sphere and
    its mirror image in free space (same solutions as the image-pair pin above)."""
    from oracle import farfield
    f, h, rad = 300e6, 0.15, 0.1
    w = 2 * np.pi * f
    th = np.radians([0.0, 20.0, 45.0, 70.0, 85.0])
    v, fc = icosphere(1, rad, (0.0, 0.0, h))
    m = Mesh(v, fc)
    same = LY.Stack([(1.0, 1.0, 0.0, np.inf), (1.0, 1.0, 0.0, 0.1), (1.0, 1.0, 0.0, np.inf)], z_top=0.0)
    A = S.assemble(m, [S.Material(4.0)], S.Material(), f)
    jd = S.j_delta(A, S.solve(A, S.rhs(A)))
    ref = farfield.rcs(m, A.k0, jd, th)
    got = farfield.rcs_layered(m, same, 0, w, jd, th)
    assert np.max(np.abs(got - ref) / ref) < 1e-12
    got = farfield.rcs_layered(m, same, 0, w, jd, th, phi=np.pi / 3)
    assert np.max(np.abs(got - farfield.rcs(m, A.k0, jd, th, phi=np.pi / 3)) / ref.max()) < 1e-12
    # sphere over PEC vs the image pair in free space
    st = LY.Stack([(1.0, 1.0, 0.0, np.inf)], z_top=0.0, bottom="pec")
    A = S.assemble(m, [S.Material(4.0)], st, f, layer=0)
    x = S.solve(A, S.rhs(A))
    vi = v.copy()
    vi[:, 2] *= -1
    xyz, tri, obj = merge((v, fc), (vi, fc[:, ::-1].copy()))
    m2 = Mesh(xyz, tri, obj)
    A2 = S.assemble(m2, [S.Material(4.0)] * 2, S.Material(), f)
    x2 = S.solve(A2, S.rhs(A2, khat=(0, 0, -1)) - S.rhs(A2, khat=(0, 0, 1)))
    for ph in (0.0, 1.1):
        ref = farfield.rcs(m2, A2.k0, S.j_delta(A2, x2), th, phi=ph)
        got = farfield.rcs_layered(m, st, 0, w, S.j_delta(A, x), th, phi=ph)
        assert np.max(np.abs(got - ref) / ref.max()) < 1e-9, (ph, got, ref)
