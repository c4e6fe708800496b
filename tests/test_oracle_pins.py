"""Pins of the FP64 oracle against closed forms, textbook results and
invariants (no GPU).  Each test names what it pins and why a plausible
mistake in the oracle would fail it."""
import math

import numpy as np
import pytest

from oracle import mlfma as ml
from oracle import pmchwt as pm
from oracle.gmres import block_diag_precond, gmres
from oracle.mie import mie_converged_order, mie_cross_sections
from oracle.special import gauss_legendre, mode_list, real_ylm, sph_h2, sph_j
from oracle.sphere import SphereShape, eval_modes, sphere_rule, static_eigenvalues


def _lattice(n, pitch=0.5):
    xs = (np.arange(n) - (n - 1) / 2) * pitch
    return np.array([[x, y, 0.0] for y in xs for x in xs])


# ------------------------------------------------------------- special functions
def test_real_harmonics_orthonormal_and_gradient():
    """Real Y_lm are orthonormal on the unit sphere (quadrature exact to 1e-14)
    and the analytic surface gradient matches central finite differences."""
    rule = sphere_rule(1.0, 12, 24)
    modes = mode_list(15)
    Y = np.array([real_ylm(l, m, k, rule['theta'], rule['phi'])[0] for (l, m, k) in modes])
    G = (Y * rule['w']) @ Y.T
    assert np.max(np.abs(G - np.eye(len(modes)))) < 1e-13
    th, ph, h = 0.7, 1.3, 1e-6
    for (l, m, k) in modes:
        _, Yt, Yp = real_ylm(l, m, k, th, ph)
        ft = (real_ylm(l, m, k, th + h, ph)[0] - real_ylm(l, m, k, th - h, ph)[0]) / (2 * h)
        fp = (real_ylm(l, m, k, th, ph + h)[0] - real_ylm(l, m, k, th, ph - h)[0]) / (2 * h)
        assert abs(Yt - ft) < 1e-8 and abs(Yp - fp / math.sin(th)) < 1e-8


# ------------------------------------------------------------- static modes
@pytest.mark.parametrize("a", [0.08, 0.15, 0.2])
def test_sphere_modes_orthonormal_divergence(a):
    """Static modes have unit L2 norm and are mutually orthogonal (Gram = I);
    transverse modes are divergence-free and the longitudinal divergence obeys
    Gauss: int psi . grad_S f = -int (div psi) f for f = c . r."""
    sh = SphereShape(a, 16, 16)
    rule = sphere_rule(a, 16, 32)
    psi, div = eval_modes(sh, rule)
    w = rule['w']
    G = np.einsum('nqc,mqc,q->nm', psi, psi, w)
    assert np.max(np.abs(G - np.eye(32))) < 1e-13
    assert np.max(np.abs(np.einsum('nqc,qc->nq', psi, rule['r_hat']))) < 1e-14  # tangential
    assert np.max(np.abs(div[:16])) == 0.0
    c = np.array([0.3, -0.5, 0.8])
    gradf = c[None, :] - rule['r_hat'] * (rule['r_hat'] @ c)[:, None]
    f = rule['r'] @ c
    lhs = np.einsum('nqc,qc,q->n', psi, gradf, w)
    rhs = -np.einsum('nq,q,q->n', div, f, w)
    assert np.max(np.abs(lhs - rhs)) < 1e-13


def test_static_eigenvalue_order():
    """Sec. III orders longitudinal modes by ascending and transverse modes by
    descending static eigenvalue; the closed forms obey both."""
    gp, gl = static_eigenvalues(SphereShape(0.15, 24, 24))
    assert np.all(np.diff(gp) <= 0) and np.all(np.diff(gl) >= 0)


def test_transverse_pattern_closed_form():
    """Eq. 26 by quadrature equals the closed form for transverse modes,
    psi_hat^perp_lm(k) = 4 pi a (-j)^l j_l(ka) (khat x grad_1 Y_lm)(khat)/sqrt(l(l+1))."""
    a = 0.2
    sc = pm.Scene([[0, 0, 0]], [0], [(a, 15, 15)], eps_in=4.0, n_theta=16, n_phi=32)
    M = ml.MLFMA.__new__(ml.MLFMA)
    M.scene, M.k = sc, sc.outer.k
    M.grids = [ml.Grid(10)]
    P = M._pattern(0)
    g = M.grids[0]
    th = np.arccos(g.khat[:, 2])
    ph = np.mod(np.arctan2(g.khat[:, 1], g.khat[:, 0]), 2 * np.pi)
    k = sc.outer.k
    for n, (l, m, kind) in enumerate(mode_list(15)):
        _, Yt, Yp = real_ylm(l, m, kind, th, ph)
        c = 4 * np.pi * a * (-1j) ** l * sph_j(l, k * a) / math.sqrt(l * (l + 1))
        assert np.max(np.abs(P[n, 0] - c * (-Yp))) < 1e-13
        assert np.max(np.abs(P[n, 1] - c * Yt)) < 1e-13


# ------------------------------------------------------------- self block vs Mie
@pytest.mark.parametrize("lmax", [1, 2, 3])
@pytest.mark.parametrize("a,eps", [(0.15, 4.0), (0.2, 4.0), (0.1, 2.25)])
def test_single_sphere_matches_truncated_mie(lmax, a, eps):
    """With full shells l <= lmax the closed-form self block (Eq. 16), the RHS
    (Eqs. 18-19) and the far field reproduce the Mie series truncated at lmax
    exactly: C_sca and C_ext to 1e-12.  A sign error in T, K, zeta or the RHS
    breaks this."""
    nm = lmax * (lmax + 2)
    sc = pm.Scene([[0.1, -0.2, 0.05]], [0], [(a, nm, nm)], eps_in=eps, n_theta=20, n_phi=40)
    x = np.linalg.solve(sc.self_block(0), pm.rhs(sc, [0, 0, 1], [1, 0, 0]))
    cs = pm.scattering_cross_section(sc, x, 24)
    ce = pm.extinction_cross_section(sc, x, [0, 0, 1], [1, 0, 0])
    ms, me = mie_cross_sections(sc.outer.k, a, math.sqrt(eps), lmax)
    assert abs(cs / ms - 1) < 1e-12 and abs(ce / me - 1) < 1e-12


def test_single_sphere_converges_to_mie():
    """l <= 4 (24 modes/current) against the converged Mie series: the
    remaining error is the l >= 5 Mie terms, below 1e-6 at ka = 0.94."""
    sc = pm.Scene([[0, 0, 0]], [0], [(0.15, 24, 24)], eps_in=4.0, n_theta=20, n_phi=40)
    x = np.linalg.solve(sc.self_block(0), pm.rhs(sc, [0, 0, 1], [1, 0, 0]))
    cs = pm.scattering_cross_section(sc, x, 24)
    nconv = mie_converged_order(sc.outer.k * 0.15)
    ms, _ = mie_cross_sections(sc.outer.k, 0.15, 2.0, nconv)
    assert abs(cs / ms - 1) < 1e-6


def test_sampled_shape_reproduces_mie():
    """A sphere given as data (points of a randomly rotated surface rule, the
    mode fields there, the self block) through the general shape path
    reproduces the truncated Mie series, so nothing in that path depends on
    the closed-form sphere grid."""
    from tests.sampled import media, rotated_sphere
    lmax, a, eps = 2, 0.15, 4.0
    nm = lmax * (lmax + 2)
    sh = rotated_sphere(a, nm, nm, media(eps), n_theta=20, n_phi=40, seed=3)
    sc = pm.Scene([[0.1, -0.2, 0.05]], [0], [sh], eps_in=eps)
    x = np.linalg.solve(sc.self_block(0), pm.rhs(sc, [0, 0, 1], [1, 0, 0]))
    cs = pm.scattering_cross_section(sc, x, 24)
    ce = pm.extinction_cross_section(sc, x, [0, 0, 1], [1, 0, 0])
    ms, me = mie_cross_sections(sc.outer.k, a, math.sqrt(eps), lmax)
    assert abs(cs / ms - 1) < 1e-10 and abs(ce / me - 1) < 1e-10


def test_sampled_shape_matches_closed_form_array():
    """In a 3x3 array, a sphere given as data on a rotated rule and the
    closed-form sphere give the same Galerkin matrix to quadrature accuracy."""
    from tests.sampled import media, rotated_sphere
    C = _lattice(3)
    sh = rotated_sphere(0.15, 8, 8, media(4.0), n_theta=16, n_phi=32, seed=5)
    Z0 = pm.dense_matrix(pm.Scene(C, [0] * 9, [(0.15, 8, 8)], eps_in=4.0))
    Z1 = pm.dense_matrix(pm.Scene(C, [0] * 9, [sh], eps_in=4.0))
    assert np.linalg.norm(Z1 - Z0) / np.linalg.norm(Z0) < 1e-10


# ------------------------------------------------------------- off-diagonal blocks
@pytest.fixture(scope="module")
def small_dense():
    sc = pm.Scene(_lattice(3), [0] * 9, [(0.15, 8, 8)], eps_in=4.0, n_theta=12, n_phi=24)
    return sc, pm.dense_matrix(sc)


def test_reciprocity(small_dense):
    """Real modes make T and K symmetric under (mu,m) <-> (nu,n), so
    Z^T = D Z D with D = diag(I, -I) per particle."""
    sc, Z = small_dense
    D = np.ones(Z.shape[0])
    D.reshape(sc.p, 2, sc.n_psi)[:, 1, :] = -1
    assert np.linalg.norm(Z.T - D[:, None] * Z * D[None, :]) / np.linalg.norm(Z) < 1e-14


def test_optical_theorem_lossless_array(small_dense):
    """For lossless particles C_ext (forward amplitude) = C_sca (integrated
    far field): energy conservation of the whole coupled system."""
    sc, Z = small_dense
    for khat, pol in (([0, 0, 1], [1, 0, 0]), ([0.3, 0, 0.9539392014169456], [0, 1, 0])):
        x = np.linalg.solve(Z, pm.rhs(sc, khat, pol))
        cs = pm.scattering_cross_section(sc, x, 40)
        ce = pm.extinction_cross_section(sc, x, khat, pol)
        assert abs(ce / cs - 1) < 1e-10


def test_optical_theorem_catches_planted_K_sign(monkeypatch):
    """Plant a flipped K in the oracle's off-diagonal blocks: energy
    conservation must fail by far more than its 1e-10 tolerance."""
    orig = pm.exterior_TK

    def flipped(*args):
        T, K = orig(*args)
        return T, -K
    monkeypatch.setattr(pm, "exterior_TK", flipped)
    sc = pm.Scene(_lattice(3), [0] * 9, [(0.15, 8, 8)], eps_in=4.0, n_theta=10, n_phi=20)
    x = np.linalg.solve(pm.dense_matrix(sc), pm.rhs(sc, [0, 0, 1], [1, 0, 0]))
    cs = pm.scattering_cross_section(sc, x, 40)
    ce = pm.extinction_cross_section(sc, x, [0, 0, 1], [1, 0, 0])
    assert abs(ce / cs - 1) > 1e-2


def test_offdiag_quadrature_converged():
    """Exterior blocks at 1 wavelength are converged in the surface rule."""
    blocks = []
    for n in (12, 20):
        sc = pm.Scene([[0, 0, 0], [1.0, 0, 0]], [0, 0], [(0.2, 16, 16)], eps_in=4.0,
                      n_theta=n, n_phi=2 * n)
        blocks.append(pm.exterior_block(sc, 0, [0, 0, 0], 0, [1.0, 0, 0]))
    assert np.linalg.norm(blocks[0] - blocks[1]) / np.linalg.norm(blocks[1]) < 1e-10


def test_well_separated_spheres_decouple():
    """Two spheres 40 wavelengths apart: each current tends to the isolated
    sphere's (coupling ~ 1/(k d)); the relative change is below 1e-2."""
    sh = [(0.15, 8, 8)]
    one = pm.Scene([[0, 0, 0]], [0], sh, eps_in=4.0)
    x1 = np.linalg.solve(one.self_block(0), pm.rhs(one, [0, 0, 1], [1, 0, 0]))
    two = pm.Scene([[0, 0, 0], [40.0, 0, 0]], [0, 0], sh, eps_in=4.0)
    x2 = np.linalg.solve(pm.dense_matrix(two), pm.rhs(two, [0, 0, 1], [1, 0, 0]))
    assert np.linalg.norm(x2[:32] - x1) / np.linalg.norm(x1) < 1e-2


# ------------------------------------------------------------- MLFMA pieces
def _addition_error(L, Xn, dn=0.35):
    k = 2 * np.pi
    g = ml.Grid(L)
    rng = np.random.default_rng(L)
    errs = []
    for _ in range(5):
        X = rng.standard_normal(3)
        X *= Xn / np.linalg.norm(X)
        d = rng.standard_normal(3)
        d *= dn / np.linalg.norm(d)
        T = ml.translation_function(k, L, g.khat, X)
        approx = np.sum(g.w * np.exp(-1j * k * (g.khat @ d)) * T)
        R = np.linalg.norm(X + d)
        exact = np.exp(-1j * k * R) / (4 * np.pi * R)
        errs.append(abs(approx - exact) / abs(exact))
    return max(errs)


@pytest.mark.parametrize("L,tol", [(10, 1e-6), (14, 1e-10), (20, 1e-13)])
def test_addition_theorem(L, tol):
    """Eq. 22: sum_k w e^{-j k khat.d} T_L(khat, X) reproduces g(|X + d|)
    for |d| < |X| (here |X| = 3, |d| = 0.35); the error falls with L."""
    assert _addition_error(L, 3.0) < tol


def test_addition_theorem_breaks_when_L_far_above_kX():
    """Sec. IV warns that h_l diverges for small arguments: with L = 40 at
    k|X| = 3 pi the truncated series loses every digit, which is why the
    truncation per level follows kd rather than a fixed doubling."""
    assert _addition_error(14, 1.5) < 1e-8
    assert _addition_error(40, 1.5) > 1.0


def test_interpolation_reproduces_cubics():
    """4x4 Lagrange reproduces tensor cubics in (theta, phi) exactly away
    from the poles and the phi seam."""
    src, dst = ml.Grid(10), ml.Grid(17)
    I = ml.interpolation_matrix(src, dst)
    TH, PH = np.meshgrid(src.theta, src.phi, indexing='ij')
    f = lambda t, p: (1 + 2 * t - t ** 2 + 0.3 * t ** 3) * (0.5 - p + 0.2 * p ** 2 - 0.01 * p ** 3)
    out = I @ f(TH, PH).ravel()
    Tt, Tp = np.meshgrid(dst.theta, dst.phi, indexing='ij')
    exact = f(Tt, Tp).ravel()
    dphi = 2 * np.pi / src.n_phi
    ok = ((Tt > src.theta[1]) & (Tt < src.theta[-2]) & (Tp > 2 * dphi) & (Tp < 2 * np.pi - 3 * dphi)).ravel()
    assert ok.sum() > 100
    assert np.max(np.abs(out[ok] - exact[ok])) < 1e-12


def test_interpolation_pole_reflection():
    """A smooth tangential field (components of a constant Cartesian vector)
    interpolates near the poles as well as elsewhere; dropping the sign
    flip of the reflected taps would leave O(1) errors there."""
    c = np.array([0.4, -0.7, 0.6])
    errs = []
    for (La, Lb) in ((10, 17), (20, 34)):
        src, dst = ml.Grid(La), ml.Grid(Lb)
        I = ml.interpolation_matrix(src, dst)
        for basis_s, basis_d in ((src.that, dst.that), (src.phat, dst.phat)):
            out = I @ (basis_s @ c)
            errs.append(np.max(np.abs(out - basis_d @ c)))
    assert errs[0] < 2e-3 and errs[1] < 2e-3
    assert errs[2] < errs[0] / 8 and errs[3] < errs[1] / 8


def test_anterpolation_is_weighted_adjoint():
    """<I f, g>_{W_parent} = <f, A g>_{W_child} with A = W_c^{-1} I^T W_p."""
    src, dst = ml.Grid(10), ml.Grid(17)
    I = ml.interpolation_matrix(src, dst)
    rng = np.random.default_rng(3)
    f = rng.standard_normal(src.K) + 1j * rng.standard_normal(src.K)
    g = rng.standard_normal(dst.K) + 1j * rng.standard_normal(dst.K)
    lhs = np.sum(dst.w * (I @ f) * g)
    rhs = np.sum(src.w * f * ((I.T @ (dst.w * g)) / src.w))
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_single_level_fmm_blocks_match_dense():
    """Eqs. 24-25 with Eq. 26 patterns and Eq. 23 at large L reproduce the
    dense T and K of a pair two wavelengths apart to 1e-11 (L = 20, inside
    the stable range L < ~1.6 k|X|): pins the k-space forms, their signs and
    the (theta, phi) algebra of the receive step."""
    sc = pm.Scene([[0, 0, 0], [2.0, 0.5, 0]], [0, 1], [(0.15, 8, 8), (0.2, 8, 8)], eps_in=4.0,
                  n_theta=16, n_phi=32)
    T0, K0 = pm.exterior_TK(sc, 0, sc.centres[0], 1, sc.centres[1])
    M = ml.MLFMA.__new__(ml.MLFMA)
    M.scene, M.k = sc, sc.outer.k
    L = 20
    M.grids = [ml.Grid(L)]
    P0, P1 = M._pattern(0), M._pattern(1)
    g = M.grids[0]
    T = ml.translation_function(M.k, L, g.khat, sc.centres[0] - sc.centres[1])
    wT = g.w * T
    Tf = -1j * M.k * (np.einsum('mk,nk,k->mn', P0[:, 0], np.conj(P1[:, 0]), wT)
                      + np.einsum('mk,nk,k->mn', P0[:, 1], np.conj(P1[:, 1]), wT))
    Kf = -1j * M.k * (np.einsum('mk,nk,k->mn', P0[:, 0], np.conj(P1[:, 1]), wT)
                      - np.einsum('mk,nk,k->mn', P0[:, 1], np.conj(P1[:, 0]), wT))
    assert np.linalg.norm(Tf - T0) / np.linalg.norm(T0) < 1e-11
    assert np.linalg.norm(Kf - K0) / np.linalg.norm(K0) < 1e-11


@pytest.fixture(scope="module")
def mixed5():
    rng = np.random.default_rng(7)
    ids = rng.integers(0, 2, size=25)
    sc = pm.Scene(_lattice(5), ids, [(0.12, 8, 8), (0.18, 8, 8)], eps_in=4.0,
                  n_theta=12, n_phi=24)
    return sc, pm.dense_matrix(sc)


def test_tree_covers_every_pair_once(mixed5):
    """Near pairs plus interaction lists (mapped down to particles) cover
    every ordered pair exactly once."""
    sc, _ = mixed5
    t = ml.Tree(sc.centres, 0.5)
    count = np.zeros((sc.p, sc.p), dtype=int)
    for (mu, nu) in t.near_pairs():
        count[mu, nu] += 1
    anc = [np.arange(sc.p)]
    for s in range(t.n_levels - 1):
        anc.append(t.levels[s]['parent'][anc[-1]])
    for s, lev in enumerate(t.levels):
        for (b, bb, _) in lev['il']:
            count[np.ix_(anc[s] == b, anc[s] == bb)] += 1
    assert np.all(count == 1)


def test_mlfma_matches_dense(mixed5):
    """MLFMA product vs the dense Galerkin product: FMM accuracy at L0 = 10,
    improving as L0 grows."""
    sc, Z = mixed5
    rng = np.random.default_rng(0)
    x = (rng.standard_normal(Z.shape[0]) + 1j * rng.standard_normal(Z.shape[0])) / math.sqrt(2)
    y0 = Z @ x
    e10 = np.linalg.norm(ml.MLFMA(sc, 0.5, L0=10).matvec(x) - y0) / np.linalg.norm(y0)
    e16 = np.linalg.norm(ml.MLFMA(sc, 0.5, L0=16).matvec(x) - y0) / np.linalg.norm(y0)
    assert e10 < 1e-3 and e16 < e10 / 3


# ------------------------------------------------------------- GMRES
def test_gmres_matches_direct_solve(mixed5):
    """Block-diagonal right-preconditioned GMRES reaches the requested true
    residual and agrees with the direct solution to that accuracy."""
    sc, Z = mixed5
    b = pm.rhs(sc, [0, 0, 1], [1, 0, 0])
    x, info = gmres(lambda v: Z @ v, b, precond=block_diag_precond(sc), tol=1e-8)
    assert info['resid_true'] <= 1e-8
    xd = np.linalg.solve(Z, b)
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) < 1e-6
    x2, info2 = gmres(lambda v: Z @ v, b, precond=block_diag_precond(sc), tol=1e-8, restart=7)
    assert info2['resid_true'] <= 1e-8


def _reciprocity_gap(M, sc, seed=1):
    """|u^T A v - (Dv)^T A (Du)| / |u^T A v| for the operator M.matvec."""
    rng = np.random.default_rng(seed)
    n = sc.n_unknowns
    u = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    v = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    D = np.ones(n)
    D.reshape(sc.p, 2, sc.n_psi)[:, 1, :] = -1
    a = u @ M.matvec(v)
    return abs(a - (D * v) @ M.matvec(D * u)) / abs(a)


def test_mlfma_is_reciprocal(mixed5):
    """The MLFMA operator keeps the Galerkin symmetry Z^T = D Z D exactly (to
    rounding), not only to FMM accuracy: receive patterns mirror the
    aggregation patterns, each translation is symmetric in the box pair, and
    anterpolation is the weighted adjoint of interpolation (Sec. IV).  This
    holds at any array size, so it also checks products too large for the
    oracle to compute."""
    sc, _ = mixed5
    assert _reciprocity_gap(ml.MLFMA(sc, 0.5, L0=10), sc) < 1e-12


def test_mlfma_reciprocity_catches_unweighted_anterpolation(mixed5, monkeypatch):
    """Plant plain transposed interpolation (quadrature weights dropped) in
    the downward pass: the operator stays accurate to a few digits but loses
    its symmetry by far more than rounding."""
    sc, _ = mixed5

    def plain_transpose(self, s, in_parent):
        lev, par = self.tree.levels[s], self.tree.levels[s + 1]
        gp = self.grids[s + 1]
        out = np.zeros((len(lev['ij']), self.grids[s].K, 4), dtype=complex)
        for c in range(len(lev['ij'])):
            B = lev['parent'][c]
            shift = np.exp(-1j * self.k * (gp.khat @ (lev['centre'][c] - par['centre'][B])))
            out[c] = self.interp[s].T @ (shift[:, None] * in_parent[B])
        return out
    monkeypatch.setattr(ml.MLFMA, "downward", plain_transpose)
    assert _reciprocity_gap(ml.MLFMA(sc, 0.5, L0=10), sc) > 1e-6


# ------------------------------------------------------------- Mie series itself
def test_mie_reproduces_published_bhmie_example():
    """oracle.mie against printed values (tests/golden/bhmie_sphere.json, cited
    there): the textbook's sample sphere, m = 1.55, x = 2 pi 0.525/0.6328.
    Q_sca and Q_ext pin |a_n|, |b_n| and Re(a_n + b_n); the backscattering
    efficiency Q_back = |sum (2n+1)(-1)^n (a_n - b_n)|^2 / x^2 also pins the
    relative phase of a_n and b_n, so a swapped or sign-flipped coefficient fails."""
    import json
    import os
    from oracle.mie import mie_coefficients
    with open(os.path.join(os.path.dirname(__file__), "golden", "bhmie_sphere.json")) as f:
        g = json.load(f)
    x = 2 * np.pi * g["radius"] / g["wavelength"]
    m = g["refractive_index"]
    nmax = mie_converged_order(x)
    cs, ce = mie_cross_sections(1.0, x, m, nmax)
    a, b = mie_coefficients(x, m, nmax)
    n = np.arange(1, nmax + 1)
    qb = abs(np.sum((2 * n + 1) * (-1.0) ** n * (a - b))) ** 2 / x ** 2
    half_ulp = 0.5 * 10.0 ** (1 - g["digits"])      # half a unit in the last printed digit
    assert abs(cs / (np.pi * x * x) - g["Q_sca"]) <= half_ulp
    assert abs(ce / (np.pi * x * x) - g["Q_ext"]) <= half_ulp
    assert abs(qb - g["Q_back"]) <= half_ulp


# ------------------------------------------------------------- near field vs Mie
def _mie_scattered_field(k, a, m, nmax, pts, zeta=1.0):
    """Scattered E, H of a sphere of radius a at the origin (relative index m,
    lossless) for the incident field E = x exp(-j k z), summed over n <= nmax.
    Textbook vector spherical wave series (Bohren & Huffman 1983, Sec. 4.4):
    with E_n = i^n (2n+1)/(n(n+1)) and outgoing waves h_n^(1) (their
    e^{-i w t} convention),
      E_s = sum E_n (i a_n N_e1n - b_n M_o1n),
      H_s = (1/zeta) sum E_n (i b_n N_o1n + a_n M_e1n),
    with angular functions pi_n = P_n^1 / sin(theta), tau_n = dP_n^1/dtheta
    from their three-term recurrences.  For real m the e^{j w t} fields are
    the complex conjugates of those."""
    import scipy.special as sps
    from oracle.mie import mie_coefficients
    an, bn = mie_coefficients(k * a, m, nmax)
    P = np.asarray(pts, dtype=float).reshape(-1, 3)
    r = np.linalg.norm(P, axis=1)
    th, ph = np.arccos(P[:, 2] / r), np.arctan2(P[:, 1], P[:, 0])
    mu, st, cp, sp_ = np.cos(th), np.sin(th), np.cos(ph), np.sin(ph)
    rho = k * r
    Es = np.zeros((r.size, 3), dtype=complex)      # (r, theta, phi) components
    Hs = np.zeros_like(Es)
    pi_m2, pi_m1 = np.zeros_like(mu), np.zeros_like(mu)     # pi_{n-2}, pi_{n-1}
    for n in range(1, nmax + 1):
        pi_n = np.ones_like(mu) if n == 1 else (2 * n - 1) / (n - 1) * mu * pi_m1 - n / (n - 1) * pi_m2
        tau = n * mu * pi_n - (n + 1) * pi_m1
        h = sps.spherical_jn(n, rho) + 1j * sps.spherical_yn(n, rho)
        dh = sps.spherical_jn(n, rho, True) + 1j * sps.spherical_yn(n, rho, True)
        dz = (h + rho * dh) / rho                          # [rho h_n]' / rho
        zero = np.zeros_like(mu)
        Mo = np.stack([zero, cp * pi_n * h, -sp_ * tau * h], 1)
        Me = np.stack([zero, -sp_ * pi_n * h, -cp * tau * h], 1)
        No = np.stack([sp_ * n * (n + 1) * st * pi_n * h / rho, sp_ * tau * dz, cp * pi_n * dz], 1)
        Ne = np.stack([cp * n * (n + 1) * st * pi_n * h / rho, cp * tau * dz, -sp_ * pi_n * dz], 1)
        En = 1j ** n * (2 * n + 1) / (n * (n + 1))
        Es += En * (1j * an[n - 1] * Ne - bn[n - 1] * Mo)
        Hs += En / zeta * (1j * bn[n - 1] * No + an[n - 1] * Me)
        pi_m2, pi_m1 = pi_m1, pi_n
    rh = np.stack([st * cp, st * sp_, mu], 1)
    thh = np.stack([mu * cp, mu * sp_, -st], 1)
    phh = np.stack([-sp_, cp, np.zeros_like(mu)], 1)
    cart = lambda F: F[:, :1] * rh + F[:, 1:2] * thh + F[:, 2:3] * phh
    return np.conj(cart(Es)), np.conj(cart(Hs))


def _single_sphere_near_case():
    """Sphere r = 0.15, eps_r = 4 (BJ-style dielectric), full shells l <= 3,
    solved for x-polarised normal incidence; 12 seeded points at 2a..5a."""
    a = 0.15
    sc = pm.Scene([[0, 0, 0]], [0], [(a, 15, 15)], eps_in=4.0, n_theta=24, n_phi=48)
    x = np.linalg.solve(sc.self_block(0), pm.rhs(sc, [0, 0, 1], [1, 0, 0]))
    d = np.random.default_rng(0).standard_normal((12, 3))
    d /= np.linalg.norm(d, axis=1)[:, None]
    pts = d * (np.linspace(2.0, 5.0, 12) * a)[:, None]
    return sc, a, x, pts


def _near_rel(sc, a, x, pts):
    E, H = pm.near_field(sc, x, pts)
    Em, Hm = _mie_scattered_field(sc.outer.k, a, 2.0, 3, pts, sc.outer.zeta)
    return (float(np.max(np.abs(E - Em)) / np.max(np.abs(Em))),
            float(np.max(np.abs(H - Hm)) / np.max(np.abs(Hm))))


def test_near_field_matches_mie_series():
    """near_field (direct surface quadrature of the Eq. 1-9 field operators)
    against the Mie scattered field: with full shells l <= 3 the closed-form
    self block reproduces a_n, b_n for n <= 3 exactly, so the currents'
    field IS the n <= 3 partial sum of the series, at every point outside
    the sphere.  E and H to 1e-12 (the 24 x 48 rule is exact far beyond the
    harmonic content reaching r >= 2a)."""
    eE, eH = _near_rel(*_single_sphere_near_case())
    assert eE < 1e-12 and eH < 1e-12


def test_near_field_far_zone_is_far_field():
    """r e^{j k r} E_s(r rhat) -> F(rhat) of far_field, with the O(1/(k r))
    remainder halving when r doubles (distance 10^3 and 2x10^3 wavelengths)."""
    sc, a, x, _ = _single_sphere_near_case()
    k = sc.outer.k
    d = np.random.default_rng(1).standard_normal((6, 3))
    d /= np.linalg.norm(d, axis=1)[:, None]
    F = pm.far_field(sc, x, d)
    err = []
    for R in (1e3, 2e3):
        E, _ = pm.near_field(sc, x, d * R)
        err.append(np.max(np.abs(E * R * np.exp(1j * k * R) - F)) / np.max(np.abs(F)))
    assert err[0] < 10.0 / (k * 1e3)
    assert 0.4 < err[1] / err[0] < 0.6


@pytest.mark.parametrize("plant", ["K_of_M_sign", "scalar_potential_sign"])
def test_near_field_pin_catches_planted_mistakes(plant, monkeypatch):
    """Planted in the oracle, on the CPU: a flipped sign of the K{M} term in
    E, or of the -(j/k) grad int g div' term of L, must break the Mie pin."""
    if plant == "K_of_M_sign":
        monkeypatch.setattr(pm, "_fields", lambda z, LJ, KJ, LM, KM: (-z * LJ - KM, -KJ - LM / z))
    else:
        monkeypatch.setattr(pm, "_L_op", lambda k, g, dg, cur, dv:
                            -1j * k * (g @ cur) + (1j / k) * np.einsum('pqc,q->pc', dg, dv))
    eE, eH = _near_rel(*_single_sphere_near_case())
    assert max(eE, eH) > 1e-3


def test_legendre_recurrence():
    """legendre_upto (Bonnet's recurrence, used for T_L of Eq. 23) against the
    library's P_l for l <= 40 and the orthogonality int P_l P_m = 2/(2l+1)
    delta_lm by a Gauss-Legendre rule exact for the products, l, m <= 320."""
    import scipy.special as sps
    from oracle.special import legendre_upto
    x = np.linspace(-1.0, 1.0, 2001)
    P = legendre_upto(40, x)
    for l in range(41):
        assert np.max(np.abs(P[l] - sps.eval_legendre(l, x))) < 1e-13
    xg, wg = gauss_legendre(330)
    Q = legendre_upto(320, xg)
    G = (Q * wg) @ Q.T
    assert np.max(np.abs(G - np.diag(2.0 / (2 * np.arange(321) + 1)))) < 1e-12
