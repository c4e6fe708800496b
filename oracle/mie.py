"""Mie series for one homogeneous sphere (FP64), used only as a pin.

Test infrastructure only (see ``oracle/__init__``).

Textbook closed form (Bohren & Huffman 1983, Sec. 4.4), written out from the
mathematics: with size parameter x = k a, relative index m = n_in / n_out,
Riccati-Bessel psi_n(z) = z j_n(z) and xi_n(z) = z h_n^(1)(z),

  a_n = [m psi_n(mx) psi_n'(x) - psi_n(x) psi_n'(mx)]
        / [m psi_n(mx) xi_n'(x) - xi_n(x) psi_n'(mx)]
  b_n = [psi_n(mx) psi_n'(x) - m psi_n(x) psi_n'(mx)]
        / [psi_n(mx) xi_n'(x) - m xi_n(x) psi_n'(mx)]

  C_sca = 2 pi / k^2 sum (2n+1)(|a_n|^2 + |b_n|^2)
  C_ext = 2 pi / k^2 sum (2n+1) Re(a_n + b_n)

(non-magnetic sphere).  |a_n|, Re a_n do not depend on the time convention,
so these cross sections pin the e^{j omega t} solver directly.
"""
import numpy as np
import scipy.special as sp


def _psi(n, z):
    j = sp.spherical_jn(n, z)
    dj = sp.spherical_jn(n, z, derivative=True)
    return z * j, j + z * dj


def _xi1(n, z):
    h = sp.spherical_jn(n, z) + 1j * sp.spherical_yn(n, z)
    dh = sp.spherical_jn(n, z, derivative=True) + 1j * sp.spherical_yn(n, z, derivative=True)
    return z * h, h + z * dh


def mie_coefficients(x, m, n_max):
    """Arrays a_n, b_n for n = 1..n_max."""
    a = np.zeros(n_max, dtype=complex)
    b = np.zeros(n_max, dtype=complex)
    for n in range(1, n_max + 1):
        px, dpx = _psi(n, x)
        pmx, dpmx = _psi(n, m * x)
        xx, dxx = _xi1(n, x)
        a[n - 1] = (m * pmx * dpx - px * dpmx) / (m * pmx * dxx - xx * dpmx)
        b[n - 1] = (pmx * dpx - m * px * dpmx) / (pmx * dxx - m * xx * dpmx)
    return a, b


def mie_cross_sections(k, radius, m, n_max):
    """(C_sca, C_ext) truncated at n_max, for background wavenumber k."""
    a, b = mie_coefficients(k * radius, m, n_max)
    n = np.arange(1, n_max + 1)
    pref = 2.0 * np.pi / k ** 2
    csca = pref * np.sum((2 * n + 1) * (np.abs(a) ** 2 + np.abs(b) ** 2))
    cext = pref * np.sum((2 * n + 1) * np.real(a + b))
    return float(csca), float(cext)


def mie_converged_order(x):
    """Wiscombe-style truncation order x + 4 x^{1/3} + 2 (plus a margin)."""
    return int(np.ceil(x + 4.0 * x ** (1.0 / 3.0) + 2.0)) + 10
