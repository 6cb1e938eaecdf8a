"""Energy balance of the oracle's full system against the Mie series (Sec. IV-A).

A sphere (icosphere sub 1, faceted volume matched by the equal-volume Mie
sphere) at k0 a = 1.47, where the forward amplitude is not small against the
scattered field: the extinction cross section from the forward amplitude (the
optical theorem), the scattering cross section from the far field integrated
over all directions, and their difference, the absorption, each against the
Mie series, for a lossless and a lossy dielectric.  A lossless object must
scatter what it removes from the incident wave; a lossy one absorbs the
difference.  This pins the lossy-material path and the far field's
normalisation against the incident power, which the RCS alone leaves free up
to a common factor in |A|^2.

The Mie efficiencies are pinned first by their own identities: Q_ext = Q_sca
for a real index, Q_ext = (4/x^2) Re S(0), and the Rayleigh limits.
"""
import numpy as np
import pytest

from oracle import farfield, mie
from oracle import system as S
from oracle.topology import Mesh
from workloads.meshes import icosphere

F = 700e6


def _sphere_directions(nt=24, nphi=48):
    x, w = np.polynomial.legendre.leggauss(nt)
    th, ph = np.arccos(x), 2 * np.pi * np.arange(nphi) / nphi
    T, P = np.meshgrid(th, ph, indexing="ij")
    rhat = np.stack([np.sin(T) * np.cos(P), np.sin(T) * np.sin(P), np.cos(T)], -1).reshape(-1, 3)
    return rhat, np.outer(w, np.full(nphi, 2 * np.pi / nphi)).ravel()


def _cross_sections(mesh, A, jd, khat, pol):
    fwd = farfield.amplitude(mesh, A.k0, jd, khat)[0]
    ext = -(4 * np.pi / A.k0) * np.imag(pol @ fwd)
    rhat, w = _sphere_directions()
    sca = np.sum(w * np.sum(np.abs(farfield.amplitude(mesh, A.k0, jd, rhat)) ** 2, axis=1))
    return ext, sca


def test_mie_efficiency_identities():
    for x in (0.3, 1.5, 4.0):
        qe, qs = mie.efficiencies(x, 2.0)
        assert abs(qe - qs) <= 1e-12 * qe                     # no absorption for a real index
        m = 2.0 + 0.3j
        qe, qs = mie.efficiencies(x, m)
        S1, S2 = mie.amplitudes(x, m, 0.0)
        assert abs(qe - 4 / x ** 2 * np.real(S1[0])) <= 1e-12 * qe   # forward amplitude
        assert abs(S1[0] - S2[0]) <= 1e-12 * abs(S1[0])
        assert qs < qe
    x, m = 1e-2, 2.0 + 0.3j
    al = (m ** 2 - 1) / (m ** 2 + 2)
    qe, qs = mie.efficiencies(x, m)
    assert abs(qs / (8 / 3 * x ** 4 * abs(al) ** 2) - 1) < 1e-3      # Rayleigh scattering
    assert abs((qe - qs) / (4 * x * np.imag(al)) - 1) < 1e-3          # Rayleigh absorption


@pytest.fixture(scope="module")
def sphere():
    v, f = icosphere(1, 0.1)
    vol = abs(np.einsum("td,td->t", v[f[:, 0]], np.cross(v[f[:, 1]], v[f[:, 2]])).sum()) / 6
    return Mesh(v, f), (3 * vol / (4 * np.pi)) ** (1 / 3)


def _mie(A, a_eq, mat):
    m = np.sqrt(np.conj(S.eps_c(mat, 2 * np.pi * F)))
    qe, qs = mie.efficiencies(A.k0 * a_eq, m)
    g = np.pi * a_eq ** 2
    return qe * g, qs * g


@pytest.mark.parametrize("sigma", [0.0, 0.02])
def test_extinction_scattering_absorption_vs_mie(sphere, sigma):
    mesh, a_eq = sphere
    mat = S.Material(4.0, 1.0, sigma)
    A = S.assemble(mesh, [mat], S.Material(), F)
    khat, pol = np.array([0.0, 0.0, -1.0]), np.array([1.0, 0.0, 0.0])
    x = S.solve(A, S.rhs(A, khat, pol))
    ext, sca = _cross_sections(mesh, A, S.j_delta(A, x), khat, pol)
    m_ext, m_sca = _mie(A, a_eq, mat)
    assert abs(ext / m_ext - 1) < 0.02, (ext, m_ext)
    assert abs(sca / m_sca - 1) < 0.01, (sca, m_sca)
    if sigma == 0:
        assert abs(ext / sca - 1) < 0.015                     # what is removed is scattered
    else:
        assert abs((ext - sca) / (m_ext - m_sca) - 1) < 0.02  # the difference is absorbed
    # planted mistake: radiating j (H alone) instead of J_Delta = j - Y11 e
    j, _, _ = S.split(A, x)
    ext_w, sca_w = _cross_sections(mesh, A, j, khat, pol)
    assert abs(ext_w / m_ext - 1) > 0.1 or abs(sca_w / m_sca - 1) > 0.1
