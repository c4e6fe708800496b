"""Closed-form static modes and self block of a sphere (FP64).

Test infrastructure only (see ``oracle/__init__``).

Static modes (Sec. III).  On a sphere of radius a the eigenproblems of the
electrostatic operator T_0^par (Eqs. 21-23) and of the magnetostatic operator
T_0^perp (Eqs. 24-25) are solved by vector spherical harmonics:

  longitudinal  psi^par_lm  = grad_1 Y_lm / (a sqrt(l(l+1)))      (curl-free)
  transverse    psi^perp_lm = r_hat x psi^par_lm                    (div-free)

with real orthonormal Y_lm, so every mode has unit L2 norm on the surface.
surface divergence: div psi^par = -sqrt(l(l+1)) Y_lm / a^2, div psi^perp = 0.
Eigenvalues (derived from the Laplace expansion of g_0 = 1/(4 pi R)):
  gamma^par_l  = l(l+1) / ((2l+1) a)   (ascending in l, as Sec. III orders them)
  gamma^perp_l = a / (2l+1)            (descending in l).
The mode set is {psi^perp_1..N_perp, psi^par_1..N_par} (Sec. III, last
paragraph), l ascending and, within a shell, m = 0, 1c, 1s, 2c, 2s, ...

Self block (Eq. 16 with delta = 1).  Expanding g in spherical waves,
g = -j k sum_l j_l(k r<) h_l^(2)(k r>) sum_m Y_lm Y_lm', the operators are
diagonal per (l, m).  With x = k a, psi_l = x j_l, xi_l = x h^(2)_l:

  T^{perp perp}_l = -psi_l(x) xi_l(x)
  T^{par par}_l   = -psi'_l(x) xi'_l(x)
  K^{par perp}_l  = K^{perp par}_l = -(j/2) (psi_l xi'_l + psi'_l xi_l)

(T and K as fixed in ``oracle/__init__``; the K entry is the principal value,
the mean of the limits from both sides, since the +-1/2 residues cancel
between the inner and outer media in the PMCHWT combination.)
"""
import numpy as np

from .special import (gauss_legendre, mode_list, real_ylm, riccati_psi,
                      riccati_xi, sphere_frame)


class SphereShape:
    """A sphere shape: radius a (in wavelengths) and mode counts."""

    def __init__(self, radius, n_perp, n_par):
        self.a = float(radius)
        self.n_perp = int(n_perp)
        self.n_par = int(n_par)
        self.perp = mode_list(self.n_perp)
        self.par = mode_list(self.n_par)

    @property
    def n_psi(self):
        return self.n_perp + self.n_par

    def modes(self):
        """List of (type, l, m, kind), type 0 = transverse, 1 = longitudinal."""
        return [(0,) + t for t in self.perp] + [(1,) + t for t in self.par]


def sphere_rule(a, n_theta, n_phi):
    """Surface quadrature on a sphere of radius a centred at the origin:
    Gauss-Legendre in cos(theta) times the trapezoid rule in phi with
    phi_j = 2 pi j / n_phi.  Returns a dict with theta, phi (Q,),
    points r (Q,3), r_hat, theta_hat, phi_hat (Q,3) and weights w (Q,)."""
    x, wx = gauss_legendre(n_theta)
    th = np.arccos(x)
    ph = 2.0 * np.pi * np.arange(n_phi) / n_phi
    TH, PH = np.meshgrid(th, ph, indexing='ij')
    W = np.outer(wx, np.full(n_phi, 2.0 * np.pi / n_phi)) * a * a
    TH, PH, W = TH.ravel(), PH.ravel(), W.ravel()
    rh, th_h, ph_h = sphere_frame(TH, PH)
    return dict(theta=TH, phi=PH, r=a * rh, r_hat=rh, theta_hat=th_h,
                phi_hat=ph_h, w=W)


def eval_modes(shape, rule):
    """Mode fields and surface divergences at the rule's points.

    Returns psi (N_psi, Q, 3) real and div (N_psi, Q) real."""
    a = shape.a
    Q = rule['w'].size
    psi = np.zeros((shape.n_psi, Q, 3))
    div = np.zeros((shape.n_psi, Q))
    th_h, ph_h = rule['theta_hat'], rule['phi_hat']
    for i, (typ, l, m, kind) in enumerate(shape.modes()):
        Y, Yt, Yp = real_ylm(l, m, kind, rule['theta'], rule['phi'])
        c = 1.0 / (a * np.sqrt(l * (l + 1)))
        if typ == 1:        # longitudinal: grad_1 Y / (a sqrt(l(l+1)))
            psi[i] = c * (Yt[:, None] * th_h + Yp[:, None] * ph_h)
            div[i] = -np.sqrt(l * (l + 1)) * Y / (a * a)
        else:               # transverse: r_hat x longitudinal
            psi[i] = c * (-Yp[:, None] * th_h + Yt[:, None] * ph_h)
    return psi, div


def static_eigenvalues(shape):
    """(gamma^perp, gamma^par) of the closed-form sphere modes."""
    a = shape.a
    gp = np.array([a / (2 * l + 1) for (l, m, k) in shape.perp])
    gl = np.array([l * (l + 1) / ((2 * l + 1) * a) for (l, m, k) in shape.par])
    return gp, gl


def medium_operators(shape, k):
    """T and K (N_psi x N_psi) of one homogeneous medium with wavenumber k
    on the sphere itself (closed form, see module docstring)."""
    n = shape.n_psi
    T = np.zeros((n, n), dtype=complex)
    K = np.zeros((n, n), dtype=complex)
    x = k * shape.a
    modes = shape.modes()
    for i, (typ, l, m, kind) in enumerate(modes):
        ps, dps = riccati_psi(l, x)
        xi, dxi = riccati_xi(l, x)
        T[i, i] = -ps * xi if typ == 0 else -dps * dxi
        kk = -0.5j * (ps * dxi + dps * xi)
        for j, (typ2, l2, m2, kind2) in enumerate(modes):
            if typ2 != typ and (l2, m2, kind2) == (l, m, kind):
                K[i, j] = kk
    return T, K


def self_block(shape, k_out, zeta_out, k_in, zeta_in):
    """Z_s = [zeta- T- + zeta+ T+, K- + K+; -(K- + K+), T-/zeta- + T+/zeta+]
    (Eq. 16 with mu = nu), size 2 N_psi, ordered [electric; magnetic]."""
    To, Ko = medium_operators(shape, k_out)
    Ti, Ki = medium_operators(shape, k_in)
    n = shape.n_psi
    Z = np.zeros((2 * n, 2 * n), dtype=complex)
    Z[:n, :n] = zeta_out * To + zeta_in * Ti
    Z[:n, n:] = Ko + Ki
    Z[n:, :n] = -(Ko + Ki)
    Z[n:, n:] = To / zeta_out + Ti / zeta_in
    return Z
