"""Pins of the oracle's rotated shapes (the in-plane rotations of Sec. V's
brick and nanofin arrays) against what physics fixes, independently of the
rotation formula itself:

* one fin turned by alpha under an x-polarised wave scatters as the unturned
  fin under the wave whose polarisation is turned by -alpha, with every
  far-field vector turned by alpha (F_alpha(R k) = R F_0(k)); extinction is
  the same;
* turning a whole two-fin configuration (centres, fin angles and the
  incident polarisation) turns its far field the same way: this exercises
  the exterior blocks between differently turned shapes;
* a planted mistake (sample points turned, mode fields not) breaks both.
"""
import numpy as np
import pytest

from oracle import mesh as om
from oracle import pmchwt as pm
from paper_2407_21724_gb300 import workloads


def _R(a):
    c, s = np.cos(a), np.sin(a)
    return np.array([[c, -s, 0.0], [s, c, 0.0], [0.0, 0.0, 1.0]])


@pytest.fixture(scope="module")
def fin():
    V, T = workloads.box_mesh(*workloads.FIN, 5, 1, 6)
    return om.MeshModes(om.Mesh(V, T), 6, 6).sampled(pm.Medium(1.0), pm.Medium(4.0))


DIRS = np.array([[0, 0, 1.0], [0, 0, -1.0], [0.6, 0, 0.8], [0, 0.8, -0.6], [0.48, 0.36, 0.8],
                 [1.0, 0, 0]])
KH = np.array([0.0, 0.0, 1.0])


def _far(centres, shapes, ids, pol):
    sc = pm.Scene(centres, ids, shapes, eps_in=4.0)
    x = np.linalg.solve(pm.dense_matrix(sc), pm.rhs(sc, KH, pol))
    return sc, x


def _turned_points_only(sh, a):
    return pm.SampledShape(sh.r @ _R(a).T, sh.w, sh.psi, sh.div, sh.Zs, sh.n_perp, sh.n_par)


def test_single_fin_rotation(fin):
    a = 0.7
    R = _R(a)
    ex = np.array([1.0, 0.0, 0.0], dtype=complex)
    sc1, x1 = _far([[0, 0, 0.0]], [pm.rotated_about_z(fin, a)], [0], ex)
    sc0, x0 = _far([[0, 0, 0.0]], [fin], [0], R.T @ ex)
    F1 = pm.far_field(sc1, x1, DIRS @ R.T)
    F0 = pm.far_field(sc0, x0, DIRS) @ R.T
    assert np.max(np.abs(F1 - F0)) < 1e-10 * np.max(np.abs(F0))
    e1 = pm.extinction_cross_section(sc1, x1, KH, ex)
    e0 = pm.extinction_cross_section(sc0, x0, KH, R.T @ ex)
    assert abs(e1 - e0) < 1e-10 * abs(e0)
    # the answer depends on the angle (the fin is not symmetric under it)
    sc2, x2 = _far([[0, 0, 0.0]], [fin], [0], ex)
    assert abs(pm.extinction_cross_section(sc2, x2, KH, ex) - e1) > 0.05 * abs(e1)
    # planted: points turned, fields not
    scb, xb = _far([[0, 0, 0.0]], [_turned_points_only(fin, a)], [0], ex)
    Fb = pm.far_field(scb, xb, DIRS @ R.T)
    assert np.max(np.abs(Fb - F0)) > 0.05 * np.max(np.abs(F0))


def test_turned_configuration(fin):
    """Two fins at angles 0.3 and 1.9 a half pitch apart, and the same pair
    with everything turned by 1.1."""
    a = 1.1
    R = _R(a)
    C = np.array([[-0.25, 0.0, 0.0], [0.25, 0.0, 0.0]])
    pol = np.array([1.0, 0.5j, 0.0]) / np.sqrt(1.25)
    base = [pm.rotated_about_z(fin, 0.3), pm.rotated_about_z(fin, 1.9)]
    turned = [pm.rotated_about_z(fin, 0.3 + a), pm.rotated_about_z(fin, 1.9 + a)]
    sc0, x0 = _far(C, base, [0, 1], pol)
    sc1, x1 = _far(C @ R.T, turned, [0, 1], R @ pol)
    F0 = pm.far_field(sc0, x0, DIRS) @ R.T
    F1 = pm.far_field(sc1, x1, DIRS @ R.T)
    assert np.max(np.abs(F1 - F0)) < 1e-9 * np.max(np.abs(F0))
    # planted: the turned pair with unturned mode fields
    bad = [_turned_points_only(base[0], a), _turned_points_only(base[1], a)]
    scb, xb = _far(C @ R.T, bad, [0, 1], R @ pol)
    assert np.max(np.abs(pm.far_field(scb, xb, DIRS @ R.T) - F0)) > 0.05 * np.max(np.abs(F0))
