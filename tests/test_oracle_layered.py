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
