"""Mie series for a homogeneous sphere (Bohren & Huffman, ch. 4): an independent,
closed-form pin for the dielectric-sphere case of Sec. IV-A.

Bistatic RCS in the plane of the incident polarisation (E-plane):
sigma(theta_s) = 4 pi |S2(theta_s)|^2 / k^2, and in the perpendicular plane
(H-plane) with S1; theta_s is the scattering angle from the forward direction.
The series is written for exp(-i w t); a material given as eps_c with
exp(+j w t) enters as its complex conjugate.
"""
import numpy as np
from scipy.special import spherical_jn, spherical_yn


def _psi(n, z):
    return z * spherical_jn(n, z)


def _dpsi(n, z):
    return spherical_jn(n, z) + z * spherical_jn(n, z, derivative=True)


def coefficients(x, m, nmax=None):
    if nmax is None:
        nmax = int(np.ceil(abs(x) + 4 * abs(x) ** (1 / 3) + 8))
    n = np.arange(1, nmax + 1)
    mx = m * x
    psi_x, dpsi_x = _psi(n, x), _dpsi(n, x)
    xi_x = x * (spherical_jn(n, x) + 1j * spherical_yn(n, x))
    dxi_x = (spherical_jn(n, x) + 1j * spherical_yn(n, x)) + x * (
        spherical_jn(n, x, derivative=True) + 1j * spherical_yn(n, x, derivative=True))
    psi_mx, dpsi_mx = _psi(n, mx), _dpsi(n, mx)
    a = (m * psi_mx * dpsi_x - psi_x * dpsi_mx) / (m * psi_mx * dxi_x - xi_x * dpsi_mx)
    b = (psi_mx * dpsi_x - m * psi_x * dpsi_mx) / (psi_mx * dxi_x - m * xi_x * dpsi_mx)
    return n, a, b


def amplitudes(x, m, theta_s):
    n, a, b = coefficients(x, m)
    mu = np.cos(np.atleast_1d(theta_s))
    pi_prev = np.zeros_like(mu)
    pi_n = np.ones_like(mu)
    S1 = np.zeros(mu.shape, dtype=complex)
    S2 = np.zeros(mu.shape, dtype=complex)
    for k in n:
        tau_n = k * mu * pi_n - (k + 1) * pi_prev
        c = (2 * k + 1) / (k * (k + 1))
        S1 += c * (a[k - 1] * pi_n + b[k - 1] * tau_n)
        S2 += c * (a[k - 1] * tau_n + b[k - 1] * pi_n)
        pi_prev, pi_n = pi_n, ((2 * k + 1) * mu * pi_n - (k + 1) * pi_prev) / k
    return S1, S2


def rcs_eplane(k0, radius, eps_c, theta_s, mu_r=1.0):
    m = np.sqrt(np.conj(complex(eps_c)) * mu_r)
    _, S2 = amplitudes(k0 * radius, m, theta_s)
    return 4 * np.pi * np.abs(S2) ** 2 / k0 ** 2


def efficiencies(x, m):
    """Extinction and scattering efficiencies (Bohren & Huffman, Sec. 4.4):
    Q_ext = (2/x^2) sum (2n+1) Re(a_n + b_n), Q_sca = (2/x^2) sum (2n+1)(|a_n|^2 + |b_n|^2);
    cross sections are Q times pi a^2, absorption = extinction - scattering."""
    n, a, b = coefficients(x, m)
    q_ext = 2.0 / x ** 2 * np.sum((2 * n + 1) * np.real(a + b))
    q_sca = 2.0 / x ** 2 * np.sum((2 * n + 1) * (np.abs(a) ** 2 + np.abs(b) ** 2))
    return float(q_ext), float(q_sca)
