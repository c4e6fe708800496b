"""Special functions for the oracle (FP64, SciPy as the library primitive).

Test infrastructure only (see ``oracle/__init__``).
"""
import numpy as np
import scipy.special as sp
from math import factorial


def sph_j(l, z):
    """Spherical Bessel function of the first kind j_l(z)."""
    return sp.spherical_jn(l, z)


def sph_y(l, z):
    """Spherical Bessel function of the second kind y_l(z)."""
    return sp.spherical_yn(l, z)


def sph_h2(l, z):
    """Spherical Hankel function of the second kind h_l^(2) = j_l - j y_l.

    It is the outgoing wave for the e^{j omega t} convention (Eq. 23)."""
    return sp.spherical_jn(l, z) - 1j * sp.spherical_yn(l, z)


def riccati_psi(l, x):
    """Riccati-Bessel psi_l(x) = x j_l(x) and its derivative."""
    j = sp.spherical_jn(l, x)
    dj = sp.spherical_jn(l, x, derivative=True)
    return x * j, j + x * dj


def riccati_xi(l, x):
    """Riccati-Hankel xi_l(x) = x h_l^(2)(x) and its derivative."""
    h = sp.spherical_jn(l, x) - 1j * sp.spherical_yn(l, x)
    dh = sp.spherical_jn(l, x, derivative=True) - 1j * sp.spherical_yn(l, x, derivative=True)
    return x * h, h + x * dh


def legendre_upto(L, x):
    """Legendre polynomials P_0(x) .. P_L(x) (Eq. 23) by Bonnet's three-term
    recurrence (l + 1) P_{l+1} = (2l + 1) x P_l - l P_{l-1}, ascending in l;
    returns an array (L + 1, *x.shape)."""
    x = np.asarray(x, dtype=float)
    P = np.empty((L + 1,) + x.shape)
    P[0] = 1.0
    if L >= 1:
        P[1] = x
    for l in range(1, L):
        P[l + 1] = ((2 * l + 1) * x * P[l] - l * P[l - 1]) / (l + 1)
    return P


def gauss_legendre(n):
    """n-point Gauss-Legendre rule on [-1, 1], nodes sorted descending
    (so that theta = arccos(x) ascends)."""
    x, w = np.polynomial.legendre.leggauss(n)
    order = np.argsort(-x)
    return x[order], w[order]


def assoc_legendre(l, m, x):
    """Associated Legendre P_l^m(x) WITHOUT the Condon-Shortley phase,
    P_l^m(x) = (1 - x^2)^{m/2} d^m P_l / dx^m  (so P_1^1 = +sin theta)."""
    if m > l or m < 0:
        return np.zeros_like(np.asarray(x, dtype=float))
    return (-1.0) ** m * sp.lpmv(m, l, x)


def shell_index(l):
    """Order of the real harmonics inside the shell of degree l:
    (m, kind) = (0,'c'), (1,'c'), (1,'s'), (2,'c'), (2,'s'), ..., (l,'s')."""
    out = [(0, 'c')]
    for m in range(1, l + 1):
        out.append((m, 'c'))
        out.append((m, 's'))
    return out


def mode_list(n_modes):
    """The first n_modes real harmonics (l >= 1) in ascending l, then the
    within-shell order of ``shell_index``: list of (l, m, kind)."""
    out = []
    l = 1
    while len(out) < n_modes:
        for (m, kind) in shell_index(l):
            out.append((l, m, kind))
            if len(out) == n_modes:
                break
        l += 1
    return out


def real_ylm(l, m, kind, theta, phi):
    """Orthonormal real spherical harmonic on the unit sphere and the two
    components of its surface gradient.

    Returns (Y, dY/dtheta, (1/sin theta) dY/dphi).  Normalisation:
    Y_l0 = N_l0 P_l(cos t), Y_lm^c = sqrt2 N_lm P_l^m cos(m phi),
    Y_lm^s = sqrt2 N_lm P_l^m sin(m phi), N_lm^2 = (2l+1)/(4 pi) (l-m)!/(l+m)!.
    The points must avoid the poles (all rules used here do)."""
    theta = np.asarray(theta, dtype=float)
    phi = np.asarray(phi, dtype=float)
    x = np.cos(theta)
    s = np.sin(theta)
    nlm = np.sqrt((2 * l + 1) / (4 * np.pi) * factorial(l - m) / factorial(l + m))
    p = assoc_legendre(l, m, x)
    # d P_l^m(cos t) / dt (no Condon-Shortley phase)
    if m == 0:
        dp = -assoc_legendre(l, 1, x)
    else:
        dp = 0.5 * ((l + m) * (l - m + 1) * assoc_legendre(l, m - 1, x)
                    - assoc_legendre(l, m + 1, x))
    if m == 0:
        ang, dang = np.ones_like(phi), np.zeros_like(phi)
        c = nlm
    elif kind == 'c':
        ang, dang = np.cos(m * phi), -m * np.sin(m * phi)
        c = np.sqrt(2.0) * nlm
    else:
        ang, dang = np.sin(m * phi), m * np.cos(m * phi)
        c = np.sqrt(2.0) * nlm
    Y = c * p * ang
    Yt = c * dp * ang
    Yp = c * p / s * dang
    return Y, Yt, Yp


def sphere_frame(theta, phi):
    """Unit vectors r_hat, theta_hat, phi_hat at (theta, phi); shape (..., 3)."""
    st, ct = np.sin(theta), np.cos(theta)
    sp_, cp = np.sin(phi), np.cos(phi)
    r = np.stack([st * cp, st * sp_, ct], axis=-1)
    t = np.stack([ct * cp, ct * sp_, -st], axis=-1)
    f = np.stack([-sp_, cp, np.zeros_like(phi)], axis=-1)
    return r, t, f
