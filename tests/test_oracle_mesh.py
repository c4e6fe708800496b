"""Pins of the mesh part of the oracle (oracle/mesh.py) against what the
mathematics fixes, independently of the oracle's own formulas:

* closed-form triangle integrals against adaptive quadrature (off the
  triangle), polar integration about the point (on it), the divergence
  theorem (edge integrals of R) and central differences (the gradient);
* RWG / star / loop structure: star charges sum to zero, loops carry no
  divergence, the Gram matrix equals a fine quadrature;
* static eigenvalues of a meshed sphere against the closed forms
  gamma_par = l(l+1)/((2l+1) a) and gamma_perp = a/(2l+1) (Sec. III; the
  spherical harmonics are eigenfunctions of the single-layer operator with
  eigenvalue a/(2l+1)), their multiplicities 2l+1 (the icosahedral mesh keeps
  l = 1, 2 irreducible) and their exact scaling with the radius;
* the self block: the cross sections of one meshed dielectric sphere converge
  to the Mie series as the mesh is refined, extinction equals scattering
  (lossless), and a planted sign error in K or a dropped smooth part breaks
  both.
"""
import numpy as np
import pytest
from scipy import integrate

from oracle import mesh as om
from oracle import mie
from oracle import pmchwt as pm
from paper_2407_21724_gb300 import workloads

TRI = np.array([[0.0, 0.0, 0.0], [1.0, 0.1, 0.0], [0.3, 0.8, 0.0]])
NRM = np.array([0.0, 0.0, 1.0])


def _fine_rule(tri, level=5):
    """Points and weights of the 7-point rule on 4^level sub-triangles."""
    tris = [tri]
    for _ in range(level):
        nxt = []
        for a, b, c in tris:
            ab, bc, ca = (a + b) / 2, (b + c) / 2, (c + a) / 2
            nxt += [np.array(t) for t in ((a, ab, ca), (ab, b, bc), (ca, bc, c), (ab, bc, ca))]
        tris = nxt
    T = np.array(tris)
    area = 0.5 * np.linalg.norm(np.cross(T[:, 1] - T[:, 0], T[:, 2] - T[:, 0]), axis=1)
    P = np.einsum('qa,tac->tqc', om.TRI7_B, T).reshape(-1, 3)
    W = (area[:, None] * om.TRI7_W[None, :]).ravel()
    return P, W


def test_triangle_integrals_off_the_triangle():
    P, W = _fine_rule(TRI)
    pts = np.array([[0.4, 0.3, 0.7], [1.5, 1.2, -0.4], [-0.8, 0.2, 0.0], [2.0, -0.5, 0.0], [0.4, 0.3, -0.3]])
    I0, I1, I2 = om.triangle_integrals(pts, TRI, NRM)
    for k, r in enumerate(pts):
        d = r[None, :] - P
        R = np.linalg.norm(d, axis=1)
        assert abs(I0[k] - np.sum(W / R)) < 1e-9 * abs(I0[k])
        assert np.allclose(I1[k], np.sum(W[:, None] * (-d) / R[:, None], axis=0), rtol=0, atol=1e-9)
        assert np.allclose(I2[k], np.sum(W[:, None] * d / R[:, None] ** 3, axis=0), rtol=0, atol=1e-8)


def test_triangle_gradient_and_divergence_theorem():
    pts = np.array([[0.4, 0.3, 0.2], [1.2, 0.9, -0.5], [0.2, 0.1, 0.05]])
    I0, I1, I2 = om.triangle_integrals(pts, TRI, NRM)
    eps = 1e-5
    for k, r in enumerate(pts):
        grad = np.zeros(3)
        for d in range(3):
            e = np.zeros(3)
            e[d] = eps
            grad[d] = (om.triangle_integrals(r + e, TRI, NRM)[0][0] -
                       om.triangle_integrals(r - e, TRI, NRM)[0][0]) / (2 * eps)
        assert np.allclose(I2[k], -grad, atol=1e-7)
        # in-plane part of int (r' - r)/R = sum over edges m * int R dl
        h = (r - TRI[0]) @ NRM
        rho = r - h * NRM
        acc = np.zeros(3)
        for i in range(3):
            a, b = TRI[i], TRI[(i + 1) % 3]
            m = np.cross((b - a) / np.linalg.norm(b - a), NRM)
            L = np.linalg.norm(b - a)
            val, _ = integrate.quad(lambda s: np.linalg.norm(r - (a + (b - a) * s / L)), 0, L, epsabs=1e-13)
            acc += m * val
        inplane = I1[k] + h * I0[k] * NRM          # I1 = int (r' - rho)/R - h n I0
        assert np.allclose(inplane, acc, atol=1e-10)
        assert np.allclose(rho, r - h * NRM)


def test_triangle_integrals_on_the_triangle():
    """Points inside the triangle (the self term): polar integration about
    the point, int 1/R dS' = sum_edges int rho(alpha) d alpha and
    int (r' - r)/R dS' = sum_edges int u(alpha) rho(alpha)^2/2 d alpha."""
    for bary in ([1 / 3, 1 / 3, 1 / 3], [0.7, 0.2, 0.1], [0.05, 0.9, 0.05]):
        r = np.array(bary) @ TRI
        I0, I1, I2 = om.triangle_integrals(r[None, :], TRI, NRM)
        s0, s1 = 0.0, np.zeros(3)
        for i in range(3):
            a, b = TRI[i] - r, TRI[(i + 1) % 3] - r
            a0, a1 = np.arctan2(a[1], a[0]), np.arctan2(b[1], b[0])
            if a1 < a0:
                a1 += 2 * np.pi
            e = b - a
            nrm_e = np.array([e[1], -e[0]]) / np.linalg.norm(e)
            dist = abs(a[:2] @ nrm_e)

            def rho(al):
                u = np.array([np.cos(al), np.sin(al)])
                return dist / abs(u @ nrm_e)
            s0 += integrate.quad(rho, a0, a1, epsabs=1e-14, epsrel=1e-13, limit=200)[0]
            for d in range(2):
                f = (lambda al, d=d: (np.cos(al) if d == 0 else np.sin(al)) * rho(al) ** 2 / 2)
                s1[d] += integrate.quad(f, a0, a1, epsabs=1e-14, epsrel=1e-13, limit=200)[0]
        assert abs(I0[0] - s0) < 1e-11 * s0
        assert np.allclose(I1[0], s1, atol=1e-11)
        assert abs(I2[0][2]) == 0.0                # principal value: no normal part


@pytest.fixture(scope="module")
def spheres():
    return {lev: om.Mesh(*workloads.icosphere(1.0, lev)) for lev in (1, 2)}


def test_rwg_structure(spheres):
    m = spheres[1]
    S = m.stars()
    # the dropped star is minus the sum of the others: every edge of the last
    # triangle appears once, every other edge twice with opposite signs
    last = set(m.eo[-1])
    for e in range(m.n_edges):
        nz = S[e][S[e] != 0]
        assert len(nz) == (1 if e in last else 2)
        if len(nz) == 2:
            assert nz.sum() == 0
    # loops are divergence-free on every triangle
    L = m.loops()
    div = np.zeros((len(m.T), L.shape[1]))
    for t in range(len(m.T)):
        for a in range(3):
            div[t] += 2 * m.h[t, a] * L[m.eo[t, a]]
    assert np.max(np.abs(div)) < 1e-12
    # the Gram matrix against a fine rule on two triangles sharing an edge
    G = m.gram()
    e = 5
    tris = [t for t in range(len(m.T)) if e in m.eo[t]]
    val = 0.0
    for t in tris:
        a = list(m.eo[t]).index(e)
        P, W = _fine_rule(m.V[m.T[t]], level=2)
        f = m.h[t, a] * (P - m.V[m.T[t, a]])
        val += np.sum(W * np.sum(f * f, axis=1))
    assert abs(G[e, e] - val) < 1e-12 * val
    assert np.all(np.linalg.eigvalsh(G) > 0)


def test_sphere_static_eigenvalues(spheres):
    exact_perp = {1: 1 / 3, 2: 1 / 5}
    exact_par = {1: 2 / 3, 2: 6 / 5}
    err = {}
    for lev, m in spheres.items():
        mm = om.MeshModes(m, 8, 8)
        gp, gl = mm.gamma_perp_all, mm.gamma_par_all
        # multiplicities: l = 1 three-fold, l = 2 five-fold, to rounding
        for g in (gp, gl):
            assert np.ptp(g[0:3]) < 1e-10 * g[0] and np.ptp(g[3:8]) < 1e-10 * g[3]
        err[lev] = (abs(gp[0] / exact_perp[1] - 1), abs(gp[3] / exact_perp[2] - 1),
                    abs(gl[0] / exact_par[1] - 1), abs(gl[3] / exact_par[2] - 1))
    # second-order convergence of the l = 1 values and of gamma_perp at l = 2
    for i in (0, 1, 2):
        assert err[2][i] < err[1][i] / 3
    assert err[2][0] < 0.02 and err[2][1] < 0.05 and err[2][2] < 0.01 and err[2][3] < 0.01


def test_static_eigenvalues_scale_with_radius(spheres):
    """gamma_perp ~ a and gamma_par ~ 1/a exactly (the kernels are
    homogeneous): a wrong power of a length anywhere breaks this."""
    m1 = spheres[1]
    m2 = om.Mesh(2.5 * m1.V, m1.T)
    a, b = om.MeshModes(m1, 6, 6), om.MeshModes(m2, 6, 6)
    assert np.allclose(b.gamma_perp, 2.5 * a.gamma_perp, rtol=1e-12)
    assert np.allclose(b.gamma_par, a.gamma_par / 2.5, rtol=1e-12)


def _sphere_cross_sections(lev, plant=None):
    a = 0.15
    outer, inner = pm.Medium(1.0), pm.Medium(4.0)
    mm = om.MeshModes(om.Mesh(*workloads.icosphere(a, lev)), 8, 8)
    sh = mm.sampled(outer, inner)
    if plant == 'k_sign':
        n = sh.n_psi
        sh.Zs[:n, n:] *= -1
        sh.Zs[n:, :n] *= -1
    sc = pm.Scene([[0.0, 0.0, 0.0]], [0], [sh], eps_in=4.0)
    kh, pol = [0.0, 0.0, 1.0], [1.0, 0.0, 0.0]
    x = np.linalg.solve(sh.Zs, pm.rhs(sc, kh, pol))
    return pm.scattering_cross_section(sc, x), pm.extinction_cross_section(sc, x, kh, pol)


def test_meshed_sphere_converges_to_mie():
    cs_mie, _ = mie.mie_cross_sections(2 * np.pi, 0.15, 2.0, 20)
    e = {}
    for lev in (1, 2):
        cs, ce = _sphere_cross_sections(lev)
        assert abs(ce - cs) < 1e-3 * cs            # lossless: extinction = scattering
        e[lev] = abs(cs / cs_mie - 1)
    assert e[2] < e[1] / 3 and e[2] < 0.08


def test_planted_mistakes_are_caught(monkeypatch):
    cs_mie, _ = mie.mie_cross_sections(2 * np.pi, 0.15, 2.0, 20)
    cs, ce = _sphere_cross_sections(1, plant='k_sign')
    assert abs(ce - cs) > 0.05 * cs or abs(cs / cs_mie - 1) > 0.5
    # the static kernel alone (no smooth remainder of the retarded one)
    monkeypatch.setattr(om, "_smooth_kernels", lambda k, R: (0.0 * R + 0j, 0.0 * R + 0j))
    cs, ce = _sphere_cross_sections(1)
    assert abs(ce - cs) > 0.05 * cs or abs(cs / cs_mie - 1) > 0.5
