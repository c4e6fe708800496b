"""Test helper: a sphere described as data (SampledShape) on a rotated
quadrature rule, so that shapes given by points, weights, mode fields and a
self block are checked against the closed-form sphere and the Mie series."""
import numpy as np

from oracle import pmchwt as pm
from oracle import sphere as osp


def rotation(seed):
    q, _ = np.linalg.qr(np.random.default_rng(seed).standard_normal((3, 3)))
    return q * np.sign(np.linalg.det(q))


def rotated_sphere(a, n_perp, n_par, scene_media, n_theta=16, n_phi=32, seed=0):
    """SampledShape of a sphere of radius a whose Gauss-Legendre x trapezoid
    rule is rotated by a seeded random rotation; the mode fields are the
    closed-form ones at the rotated points, the self block the closed form
    for scene_media = (k_out, zeta_out, k_in, zeta_in)."""
    base = osp.sphere_rule(a, n_theta, n_phi)
    r = base['r'] @ rotation(seed).T
    rh = r / a
    th = np.arccos(np.clip(rh[:, 2], -1.0, 1.0))
    ph = np.mod(np.arctan2(rh[:, 1], rh[:, 0]), 2 * np.pi)
    _, th_h, ph_h = osp.sphere_frame(th, ph)
    rule = dict(theta=th, phi=ph, r=r, r_hat=rh, theta_hat=th_h, phi_hat=ph_h, w=base['w'])
    sh = osp.SphereShape(a, n_perp, n_par)
    psi, div = osp.eval_modes(sh, rule)
    Zs = osp.self_block(sh, *scene_media)
    return pm.SampledShape(r, base['w'], psi, div, Zs, n_perp, n_par)


def media(eps_in, eps_out=1.0):
    sc = pm.Scene([[0.0, 0.0, 0.0]], [0], [(0.1, 1, 1)], eps_in=eps_in, eps_out=eps_out)
    return sc.outer.k, sc.outer.zeta, sc.inner.k, sc.inner.zeta
