"""Galerkin PMCHWT operator in the static-mode basis by direct quadrature (FP64).

Test infrastructure only (see ``oracle/__init__``).

This is the plain definition the MLFMA approximates (Sec. II, Eqs. 1-19):
every block Z^{mu nu} (Eq. 16) is a 2N_psi x 2N_psi matrix over the modes of
particles mu and nu.  Self blocks come from the closed form in
``oracle.sphere``; every other block involves only the outer medium (Sec. IV,
below Eq. 19's discussion of near/far) and is the double surface integral

  T_mn = -j k sum_q sum_q' w w' [psi_m . psi_n' - div psi_m div' psi_n' / k^2] g
  K_mn = - sum_q sum_q' w w' psi_m . (psi_n' x grad' g)
  grad' g(r - r') = (r - r') (1 + j k R) exp(-j k R) / (4 pi R^3)

on a fixed surface rule (Gauss-Legendre in cos theta times trapezoid in phi).
Units: lengths in vacuum wavelengths, zeta normalised by the vacuum impedance.
"""
import numpy as np

from .sphere import SphereShape, eval_modes, self_block, sphere_rule


class Medium:
    """Homogeneous medium of relative (eps, mu) at vacuum wavelength lam."""

    def __init__(self, eps, mu=1.0, lam=1.0):
        self.eps = complex(eps)
        self.mu = complex(mu)
        n = np.sqrt(self.eps * self.mu)
        self.k = 2.0 * np.pi / lam * n
        if abs(np.imag(self.k)) == 0.0:
            self.k = float(np.real(self.k))
        self.zeta = np.sqrt(self.mu / self.eps)
        if np.imag(self.zeta) == 0.0:
            self.zeta = float(np.real(self.zeta))


class SampledShape:
    """A shape given as data rather than in closed form (the form in which a
    meshed particle's static modes reach the solver, Sec. V stages ii-iv):
    surface quadrature points r (Q,3) relative to the particle centre and
    weights w (Q,), the N_perp + N_par mode fields psi (N_psi,Q,3) and surface
    divergences div (N_psi,Q) at those points, and the self block Z_s
    (2 N_psi, 2 N_psi) for the scene's media (Eq. 16 with mu = nu)."""

    def __init__(self, r, w, psi, div, Zs, n_perp, n_par):
        self.r = np.asarray(r, dtype=float).reshape(-1, 3)
        self.w = np.asarray(w, dtype=float).ravel()
        self.psi = np.asarray(psi, dtype=float)
        self.div = np.asarray(div, dtype=float)
        self.Zs = np.asarray(Zs, dtype=complex)
        self.n_perp, self.n_par = int(n_perp), int(n_par)
        assert self.psi.shape == (self.n_psi, self.w.size, 3) and self.div.shape == (self.n_psi, self.w.size)
        assert self.Zs.shape == (2 * self.n_psi, 2 * self.n_psi)

    @property
    def n_psi(self):
        return self.n_perp + self.n_par

    @property
    def a(self):
        return float(np.max(np.linalg.norm(self.r, axis=1)))


def rotated_about_z(sh, angle):
    """The sampled shape turned by `angle` about the z axis through its centre
    (the in-plane rotations of Sec. V's brick and nanofin arrays): with R the
    rotation, a point r goes to R r and a tangential field to R psi there; the
    weights and surface divergences stay, and so does the self block (the
    operators T and K are unchanged by a rotation of both arguments)."""
    c, s = np.cos(angle), np.sin(angle)
    R = np.array([[c, -s, 0.0], [s, c, 0.0], [0.0, 0.0, 1.0]])
    return SampledShape(sh.r @ R.T, sh.w, sh.psi @ R.T, sh.div, sh.Zs, sh.n_perp, sh.n_par)


class Scene:
    """p particles: centres (p,3), shape ids (p,), shapes, inner/outer media,
    and the surface rule (n_theta, n_phi) used for every surface integral."""

    def __init__(self, centres, shape_ids, shapes, eps_in, eps_out=1.0,
                 mu_in=1.0, mu_out=1.0, lam=1.0, n_theta=16, n_phi=32):
        self.centres = np.asarray(centres, dtype=float).reshape(-1, 3)
        self.shape_ids = np.asarray(shape_ids, dtype=int).ravel()
        self.inner = Medium(eps_in, mu_in, lam)
        self.outer = Medium(eps_out, mu_out, lam)
        self.shapes = []
        for s in shapes:
            self.shapes.append(self._shape(s))
        self.n_theta, self.n_phi = n_theta, n_phi
        npsi = {s.n_psi for s in self.shapes}
        assert len(npsi) == 1, "all shapes share one mode count"
        self.n_psi = npsi.pop()
        self._rules = {}

    def _shape(self, s):
        """Closed-form spheres from (radius, n_perp, n_par); meshed shapes
        from dicts with kind 'mesh' (verts, tris, n_perp, n_par), their modes
        and self block computed here (``oracle.mesh``); dicts with kind
        'rotated' (base, angle) turn an earlier shape about z."""
        if isinstance(s, (SphereShape, SampledShape)):
            return s
        if isinstance(s, dict) and s.get('kind') == 'rotated':
            return rotated_about_z(self.shapes[s['base']], s['angle'])
        if isinstance(s, dict) and s.get('kind') == 'mesh':
            from .mesh import Mesh, MeshModes
            return MeshModes(Mesh(s['verts'], s['tris']), s['n_perp'], s['n_par']).sampled(self.outer, self.inner)
        return SphereShape(*s)

    @property
    def p(self):
        return self.centres.shape[0]

    @property
    def n_unknowns(self):
        return 2 * self.n_psi * self.p

    def shape_data(self, s):
        """(rule, psi, div) of shape s on the scene's surface rule."""
        if s not in self._rules:
            sh = self.shapes[s]
            if isinstance(sh, SampledShape):
                self._rules[s] = ({'r': sh.r, 'w': sh.w}, sh.psi, sh.div)
            else:
                rule = sphere_rule(sh.a, self.n_theta, self.n_phi)
                psi, div = eval_modes(sh, rule)
                self._rules[s] = (rule, psi, div)
        return self._rules[s]

    def self_block(self, s):
        sh = self.shapes[s]
        if isinstance(sh, SampledShape):
            return sh.Zs
        return self_block(sh, self.outer.k, self.outer.zeta, self.inner.k, self.inner.zeta)


def exterior_TK(scene, s_m, c_m, s_n, c_n):
    """T and K (N_psi x N_psi) of the outer medium between a particle of shape
    s_m at c_m (testing) and one of shape s_n at c_n (source), by quadrature."""
    k = scene.outer.k
    rm, psm, dvm = scene.shape_data(s_m)
    rn, psn, dvn = scene.shape_data(s_n)
    P = rm['r'] + np.asarray(c_m)[None, :]
    Pp = rn['r'] + np.asarray(c_n)[None, :]
    d = P[:, None, :] - Pp[None, :, :]
    R = np.sqrt(np.sum(d * d, axis=-1))
    e = np.exp(-1j * k * R)
    G = e / (4.0 * np.pi * R)
    gp = (1.0 + 1j * k * R) * e / (4.0 * np.pi * R ** 3)
    Am = psm * rm['w'][None, :, None]      # weighted test functions
    An = psn * rn['w'][None, :, None]
    Dm = dvm * rm['w'][None, :]
    Dn = dvn * rn['w'][None, :]
    T = np.zeros((psm.shape[0], psn.shape[0]), dtype=complex)
    for c in range(3):
        T += Am[:, :, c] @ G @ An[:, :, c].T
    T = -1j * k * T + (1j / k) * (Dm @ G @ Dn.T)
    # psi_m . (psi_n x v) = sum eps_abc psi_m,a psi_n,b v_c
    K = np.zeros_like(T)
    for (a, b, c, sgn) in ((0, 1, 2, 1), (1, 2, 0, 1), (2, 0, 1, 1),
                           (0, 2, 1, -1), (2, 1, 0, -1), (1, 0, 2, -1)):
        K += sgn * (Am[:, :, a] @ (gp * d[:, :, c]) @ An[:, :, b].T)
    return T, -K


def exterior_block(scene, s_m, c_m, s_n, c_n):
    """Z^{mu nu} for mu != nu (Eq. 16 with delta = 0): [zT, K; -K, T/z]."""
    T, K = exterior_TK(scene, s_m, c_m, s_n, c_n)
    z = scene.outer.zeta
    return np.block([[z * T, K], [-K, T / z]])


def dense_matrix(scene, offset_cache=True):
    """The full Galerkin matrix Z (N x N), N = 2 N_psi p.  Unknown order:
    particle, then [electric modes, magnetic modes].  Blocks that depend only
    on (shape, shape, centre difference) are computed once."""
    p, n2 = scene.p, 2 * scene.n_psi
    Z = np.zeros((p * n2, p * n2), dtype=complex)
    cache = {}
    for mu in range(p):
        for nu in range(p):
            sm, sn = scene.shape_ids[mu], scene.shape_ids[nu]
            if mu == nu:
                key = ('self', sm)
                if key not in cache:
                    cache[key] = scene.self_block(sm)
            else:
                dc = scene.centres[mu] - scene.centres[nu]
                key = (sm, sn) + tuple(np.round(dc, 12)) if offset_cache else (mu, nu)
                if key not in cache:
                    cache[key] = exterior_block(scene, sm, dc, sn, np.zeros(3))
            Z[mu * n2:(mu + 1) * n2, nu * n2:(nu + 1) * n2] = cache[key]
    return Z


def plane_wave(khat, pol):
    """Unit-amplitude plane wave E = pol exp(-j k khat.r), H = khat x E / zeta."""
    khat = np.asarray(khat, dtype=float)
    khat = khat / np.linalg.norm(khat)
    return khat, np.asarray(pol, dtype=complex)


def rhs(scene, khat, pol):
    """V = [<psi_n, E_inc>; <psi_n, H_inc>] per particle (Eqs. 5, 18, 19),
    flattened in the unknown order of ``dense_matrix``."""
    khat, pol = plane_wave(khat, pol)
    k, z = scene.outer.k, scene.outer.zeta
    hpol = np.cross(khat, pol) / z
    out = np.zeros((scene.p, 2, scene.n_psi), dtype=complex)
    for mu in range(scene.p):
        rule, psi, _ = scene.shape_data(scene.shape_ids[mu])
        r = rule['r'] + scene.centres[mu][None, :]
        ph = np.exp(-1j * k * (r @ khat)) * rule['w']
        out[mu, 0] = np.einsum('nqc,c,q->n', psi, pol, ph)
        out[mu, 1] = np.einsum('nqc,c,q->n', psi, hpol, ph)
    return out.reshape(-1)


def radiation_integrals(scene, x, dirs):
    """J_hat(r) = int J e^{j k r.r'} dS' and M_hat(r) for unit directions
    dirs (n,3); returns two complex arrays (n,3)."""
    k = scene.outer.k
    xx = np.asarray(x).reshape(scene.p, 2, scene.n_psi)
    dirs = np.asarray(dirs, dtype=float).reshape(-1, 3)
    J = np.zeros((dirs.shape[0], 3), dtype=complex)
    M = np.zeros_like(J)
    for mu in range(scene.p):
        rule, psi, _ = scene.shape_data(scene.shape_ids[mu])
        r = rule['r'] + scene.centres[mu][None, :]
        ph = np.exp(1j * k * (dirs @ r.T)) * rule['w'][None, :]     # (n, Q)
        fe = np.einsum('n,nqc->qc', xx[mu, 0], psi)
        fm = np.einsum('n,nqc->qc', xx[mu, 1], psi)
        J += ph @ fe
        M += ph @ fm
    return J, M


def far_field(scene, x, dirs):
    """F(r) with E_s ~ F exp(-j k r)/r:  F = (j k / 4 pi)[zeta (I - rr) J_hat - r x M_hat]."""
    dirs = np.asarray(dirs, dtype=float).reshape(-1, 3)
    J, M = radiation_integrals(scene, x, dirs)
    k, z = scene.outer.k, scene.outer.zeta
    Jt = J - dirs * np.sum(dirs * J, axis=1)[:, None]
    return (1j * k / (4.0 * np.pi)) * (z * Jt - np.cross(dirs, M))


def scattering_cross_section(scene, x, n_theta=48):
    """C_sca = int |F|^2 dOmega (unit incident amplitude), Gauss-Legendre x
    trapezoid rule on the sphere of directions."""
    from .special import gauss_legendre, sphere_frame
    n_phi = 2 * n_theta
    c, w = gauss_legendre(n_theta)
    th = np.arccos(c)
    ph = 2 * np.pi * np.arange(n_phi) / n_phi
    TH, PH = np.meshgrid(th, ph, indexing='ij')
    W = np.outer(w, np.full(n_phi, 2 * np.pi / n_phi)).ravel()
    r, _, _ = sphere_frame(TH.ravel(), PH.ravel())
    F = far_field(scene, x, r)
    return float(np.sum(W * np.sum(np.abs(F) ** 2, axis=1)))


def extinction_cross_section(scene, x, khat, pol):
    """Optical theorem for e^{j omega t}: C_ext = -(4 pi / k) Im(e* . F(k_inc))."""
    khat, pol = plane_wave(khat, pol)
    F = far_field(scene, x, khat[None, :])[0]
    return float(-(4 * np.pi / scene.outer.k) * np.imag(np.vdot(pol, F)) / np.vdot(pol, pol).real)


def _L_op(k, g, dg, cur, dv):
    """L{X} = -j k int g X - (j/k) grad int g div'X at the field points; g and
    dg = grad_r g carry the quadrature weights, cur (Q,3) and dv (Q,) are X
    and div'X at the quadrature points."""
    return -1j * k * (g @ cur) - (1j / k) * np.einsum('pqc,q->pc', dg, dv)


def _K_op(dg, cur):
    """K{X} = curl int g X = int grad_r g x X."""
    Kx = np.einsum('pqc,qd->pcd', dg, cur)              # grad g (x) X
    return np.stack([Kx[:, 1, 2] - Kx[:, 2, 1], Kx[:, 2, 0] - Kx[:, 0, 2],
                     Kx[:, 0, 1] - Kx[:, 1, 0]], axis=1)


def _fields(z, LJ, KJ, LM, KM):
    """Scattered fields of the equivalent currents J, M (the sign conventions
    of the package docstring): E = -zeta L{J} + K{M}, H = -K{J} - L{M}/zeta."""
    return -z * LJ + KM, -KJ - LM / z


def near_field(scene, x, points):
    """Scattered E and H at points outside every particle (n,3) by direct
    surface quadrature with the full Green's dyadic:
      E = -zeta L{J} + K{M},  H = -K{J} - L{M}/zeta,
      L{X} = -j k int g X - (j/k) grad int g div'X,  K{X} = curl int g X."""
    k, z = scene.outer.k, scene.outer.zeta
    xx = np.asarray(x).reshape(scene.p, 2, scene.n_psi)
    pts = np.asarray(points, dtype=float).reshape(-1, 3)
    E = np.zeros((pts.shape[0], 3), dtype=complex)
    H = np.zeros_like(E)
    for mu in range(scene.p):
        rule, psi, div = scene.shape_data(scene.shape_ids[mu])
        rq = rule['r'] + scene.centres[mu][None, :]
        d = pts[:, None, :] - rq[None, :, :]
        R = np.sqrt(np.sum(d * d, axis=-1))
        e = np.exp(-1j * k * R)
        g = e / (4 * np.pi * R) * rule['w'][None, :]
        # grad_r g = -(r - r')(1 + j k R) e / (4 pi R^3)
        dg = -(d * ((1 + 1j * k * R) * e / (4 * np.pi * R ** 3) * rule['w'][None, :])[..., None])
        out = []
        for c in range(2):
            cur = np.einsum('n,nqc->qc', xx[mu, c], psi)     # (Q,3)
            dv = np.einsum('n,nq->q', xx[mu, c], div)          # (Q,)
            out.append((_L_op(k, g, dg, cur, dv), _K_op(dg, cur)))
        (LJ, KJ), (LM, KM) = out
        Eq, Hq = _fields(z, LJ, KJ, LM, KM)
        E += Eq
        H += Hq
    return E, H
