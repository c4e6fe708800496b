"""Static modes of a meshed particle and its PMCHWT self block (FP64).

Test infrastructure only (see ``oracle/__init__``).

Sec. III (Eqs. 21-25): the longitudinal static modes solve the electrostatic
eigenproblem T0_par j = gamma j expanded and tested in star functions, the
transverse ones the magnetostatic problem T0_perp j = gamma j in loop
functions.  In Galerkin form, with RWG functions f_e and g0 = 1/(4 pi R):

  A_par v = gamma G v,   A_par = S^T [int int (div f)(div' f') g0] S
  A_perp v = gamma G v,  A_perp = L^T [int int f . f' g0] L,   G = Gram

(stars S and loops L as RWG combinations).  The N_par smallest gamma_par
and the N_perp largest gamma_perp are kept (Sec. III, below Eq. 25), each
mode unit-normalised (v^T G v = 1), and the mode -> RWG matrix M of Eq. 20
holds the transverse modes first.

Sec. II (Eqs. 13-16) with the basis change of Eq. 20: the self block is
assembled on the RWG functions, Z_rwg for each medium from

  T = -j k int int [f . f' - div f div' f' / k^2] G,
  K = - int int f . (f' x grad' G)        (principal value)

and then compressed, Z_s = M Z_rwg M^T for every block of Eq. 16.  The
singular part of the kernels is integrated in closed form over the source
triangle (the inner integral), the rest by a fixed rule (Sec. IV, below
Eq. 19: the techniques of Graglia 1993 and Hodges 1997):

  int 1/R dS',  int (r' - r)/R dS',  int (r - r')/R^3 dS'

as closed forms of the triangle's edges; the outer integral and the smooth
remainders G - g0 and grad'(G - g0) by Radon's 7-point degree-5 rule.  The
mode fields reach the solver sampled at a 3-point degree-2 rule per
triangle (``MeshModes.sampled``).

Conventions (shared with ``oracle.pmchwt``): lengths in vacuum wavelengths,
time factor e^{j omega t}, G = exp(-j k R)/(4 pi R),
grad' G = (r - r')(1 + j k R) exp(-j k R)/(4 pi R^3).
"""
import numpy as np
import scipy.linalg

from .pmchwt import SampledShape

_S15 = np.sqrt(15.0)
# Radon's 7-point rule (exact for polynomials of degree 5): barycentric
# points and weights summing to 1
_A1, _A2 = (6.0 - _S15) / 21.0, (6.0 + _S15) / 21.0
TRI7_B = np.array([[1 / 3, 1 / 3, 1 / 3],
                   [1 - 2 * _A1, _A1, _A1], [_A1, 1 - 2 * _A1, _A1], [_A1, _A1, 1 - 2 * _A1],
                   [1 - 2 * _A2, _A2, _A2], [_A2, 1 - 2 * _A2, _A2], [_A2, _A2, 1 - 2 * _A2]])
TRI7_W = np.array([9 / 40] + [(155 - _S15) / 1200] * 3 + [(155 + _S15) / 1200] * 3)
# 3-point rule (exact for degree 2): the sampling of the mode fields
TRI3_B = np.array([[2 / 3, 1 / 6, 1 / 6], [1 / 6, 2 / 3, 1 / 6], [1 / 6, 1 / 6, 2 / 3]])
TRI3_W = np.full(3, 1 / 3)

_FOURPI = 4.0 * np.pi


class Mesh:
    """A closed, consistently oriented genus-0 triangle mesh (outward normals)
    and its RWG functions.

    Edge e joins the vertices (i, j), i < j, edges in lexicographic order.
    T+ of an edge is the triangle in whose vertex cycle the edge runs i -> j,
    T- the other.  f_e = l_e/(2 A+) (r - v+) on T+ and l_e/(2 A-) (v- - r) on
    T-, v+- the vertices opposite the edge.  Triangle t, corner a carries the
    half function h[t, a] (r - V[T[t, a]]) of edge eo[t, a] (the edge
    opposite the corner), h = +-l/(2 A)."""

    def __init__(self, verts, tris):
        self.V = np.asarray(verts, dtype=float).reshape(-1, 3)
        self.T = np.asarray(tris, dtype=np.int64).reshape(-1, 3)
        V, T = self.V, self.T
        p0, p1, p2 = V[T[:, 0]], V[T[:, 1]], V[T[:, 2]]
        cr = np.cross(p1 - p0, p2 - p0)
        self.area = 0.5 * np.linalg.norm(cr, axis=1)
        self.normal = cr / (2.0 * self.area[:, None])
        directed = {}
        for t in range(len(T)):
            for a in range(3):
                i, j = T[t, (a + 1) % 3], T[t, (a + 2) % 3]
                if (i, j) in directed:
                    raise ValueError("edge used twice in one direction: inconsistent orientation")
                directed[(i, j)] = (t, a)
        edges = sorted({(min(i, j), max(i, j)) for (i, j) in directed})
        if any((j, i) not in directed for (i, j) in directed):
            raise ValueError("open or non-manifold mesh")
        if len(V) - len(edges) + len(T) != 2:
            raise ValueError("mesh is not a closed genus-0 surface")
        vol = np.sum(np.einsum('ij,ij->i', p0, np.cross(p1, p2))) / 6.0
        if vol <= 0:
            raise ValueError("normals point inwards")
        self.edges = np.array(edges, dtype=np.int64)
        self.length = np.linalg.norm(V[self.edges[:, 1]] - V[self.edges[:, 0]], axis=1)
        self.eo = np.zeros((len(T), 3), dtype=np.int64)
        self.h = np.zeros((len(T), 3))
        for e, (i, j) in enumerate(edges):
            tp, ap = directed[(i, j)]
            tm, am = directed[(j, i)]
            self.eo[tp, ap], self.eo[tm, am] = e, e
            self.h[tp, ap] = self.length[e] / (2.0 * self.area[tp])
            self.h[tm, am] = -self.length[e] / (2.0 * self.area[tm])

    @property
    def n_edges(self):
        return len(self.edges)

    def points(self, bary):
        """Rule points (nt, nq, 3) for barycentric coordinates bary (nq, 3)."""
        P = self.V[self.T]                                  # (nt, 3, 3)
        return np.einsum('qa,tac->tqc', bary, P)

    def incidence(self):
        """H (n_edges, 3 nt): H[eo[t, a], 3 t + a] = 1."""
        H = np.zeros((self.n_edges, 3 * len(self.T)))
        H[self.eo.ravel(), np.arange(3 * len(self.T))] = 1.0
        return H

    def stars(self):
        """S (n_edges, nt - 1): star t = sum_a sign f_eo[t,a], flowing out of t
        (the last triangle's star, the negative sum of the others, is
        dropped)."""
        S = np.zeros((self.n_edges, len(self.T)))
        for t in range(len(self.T)):
            for a in range(3):
                S[self.eo[t, a], t] = np.sign(self.h[t, a])
        return S[:, :-1]

    def loops(self):
        """L (n_edges, nv - 1): loop v = n x grad(lambda_v), lambda_v the hat
        function of vertex v, as RWG combination: the coefficient of f_e is
        the loop's flux density across e out of T+ (the RWG function's is 1).
        The last vertex's loop is dropped."""
        V, T = self.V, self.T
        L = np.zeros((self.n_edges, len(V)))
        for t in range(len(T)):
            n = self.normal[t]
            for a in range(3):
                if self.h[t, a] <= 0:
                    continue                                   # visit each edge from T+
                e = self.eo[t, a]
                i, j = T[t, (a + 1) % 3], T[t, (a + 2) % 3]    # the edge, in t's cycle
                m = np.cross((V[j] - V[i]) / self.length[e], n)   # outward edge normal in t
                for v in (i, j):
                    k = list(T[t]).index(v)
                    w1, w2 = T[t, (k + 1) % 3], T[t, (k + 2) % 3]
                    grad = np.cross(n, V[w2] - V[w1]) / (2.0 * self.area[t])
                    L[e, v] = np.cross(n, grad) @ m
        return L[:, :-1]

    def gram(self):
        """G[e, e'] = int f_e . f_e' dS (the 7-point rule is exact)."""
        P = self.points(TRI7_B)
        w = self.area[:, None] * TRI7_W[None, :]
        Gh = np.zeros((3 * len(self.T), 3 * len(self.T)))
        for t in range(len(self.T)):
            F = self.h[t][:, None, None] * (P[t][None, :, :] - self.V[self.T[t]][:, None, :])
            Gh[3 * t:3 * t + 3, 3 * t:3 * t + 3] = np.einsum('aqc,bqc,q->ab', F, F, w[t])
        H = self.incidence()
        return H @ Gh @ H.T


def triangle_integrals(r, tri, normal):
    """Closed forms over one flat triangle tri (3,3) (vertices in the order
    of the outward normal) at points r (P,3):

      I0 = int 1/R dS',  I1 = int (r' - r)/R dS',  I2 = int (r - r')/R^3 dS'

    with R = |r - r'|.  I2 is the principal value for points in the plane
    of the triangle (normal part 0).  Per edge i (p_i -> p_i+1): unit
    direction s, outward in-plane normal m = s x n, coordinates s+- of the
    edge ends along s from the projection rho of r, signed distance t0 =
    (p_i - rho) . m, R0^2 = t0^2 + h^2, R+- = sqrt(s+-^2 + R0^2),
    f = ln((R+ + s+)/(R- + s-)) and the subtended angle
    beta = atan(t0 s+/(R0^2 + |h| R+)) - atan(t0 s-/(R0^2 + |h| R-)):

      I0 = sum t0 f - |h| sum beta
      int (r' - rho)/R dS' = 1/2 sum m (R0^2 f + s+ R+ - s- R-)
      I2 = n sign(h) sum beta + sum m f."""
    r = np.asarray(r, dtype=float).reshape(-1, 3)
    n = np.asarray(normal, dtype=float)
    h = (r - tri[0]) @ n
    rho = r - h[:, None] * n[None, :]
    ah = np.abs(h)
    I0 = np.zeros(len(r))
    Ip = np.zeros((len(r), 3))
    I2 = np.zeros((len(r), 3))
    bsum = np.zeros(len(r))
    for i in range(3):
        a, b = tri[i], tri[(i + 1) % 3]
        le = np.linalg.norm(b - a)
        s = (b - a) / le
        m = np.cross(s, n)
        sp = (b - rho) @ s
        sm = (a - rho) @ s
        t0 = (a - rho) @ m
        R02 = t0 * t0 + h * h
        Rp = np.sqrt(sp * sp + R02)
        Rm = np.sqrt(sm * sm + R02)
        # ln((R+ + s+)/(R- + s-)); for an edge wholly behind the foot point
        # the equal ratio (R- - s-)/(R+ - s+) avoids the cancellation
        behind = sp < 0
        with np.errstate(divide='ignore', invalid='ignore'):
            f = np.where(behind, np.log((Rm - sm) / (Rp - sp)), np.log((Rp + sp) / (Rm + sm)))
            beta = np.arctan2(t0 * sp, R02 + ah * Rp) - np.arctan2(t0 * sm, R02 + ah * Rm)
        beta = np.where(R02 > 0, beta, 0.0)
        I0 += t0 * f - ah * beta
        Ip += 0.5 * (R02 * f + sp * Rp - sm * Rm)[:, None] * m[None, :]
        I2 += f[:, None] * m[None, :]
        bsum += beta
    I1 = Ip - (h * I0)[:, None] * n[None, :]
    sgn = np.where(ah > 1e-12 * max(1.0, np.max(np.abs(tri))), np.sign(h), 0.0)
    I2 += (sgn * bsum)[:, None] * n[None, :]
    return I0, I1, I2


def _smooth_kernels(k, R):
    """(G - g0) and the factor of (r - r') in grad'(G - g0), at distances R:
    (exp(-j k R) - 1)/(4 pi R) and ((1 + j k R) exp(-j k R) - 1)/(4 pi R^3),
    with their limits -j k/(4 pi) and 0 at R = 0 and short Taylor series for
    k R < 0.01 (the differences cancel there)."""
    x = k * R
    small = x < 0.01
    Rs = np.where(R > 0, R, 1.0)
    with np.errstate(divide='ignore', invalid='ignore'):
        e = np.exp(-1j * x)
        g1 = (e - 1.0) / (_FOURPI * Rs)
        f1 = ((1.0 + 1j * x) * e - 1.0) / (_FOURPI * Rs ** 3)
    # series: (e^{-jx} - 1)/x = -j - x/2 + j x^2/6 + x^3/24 - j x^4/120
    #         ((1 + jx) e^{-jx} - 1)/x^2 = 1/2 - j x/3 - x^2/8 + j x^3/30 + x^4/144
    gs = k * (-1j - x / 2 + 1j * x ** 2 / 6 + x ** 3 / 24 - 1j * x ** 4 / 120) / _FOURPI
    fs = k * k * (0.5 - 1j * x / 3 - x ** 2 / 8 + 1j * x ** 3 / 30 + x ** 4 / 144) / (_FOURPI * Rs)
    g1 = np.where(small, gs, g1)
    f1 = np.where(small, fs, f1)
    f1 = np.where(R > 0, f1, 0.0)
    return g1, f1


def inner_integrals(mesh, r, t_src, k):
    """Inner integrals over source triangle t_src at points r (P,3):
    S = int G dS', V = int (r' - r) G dS', U = int (r - r') F dS' with
    grad' G = (r - r') F.  Singular parts in closed form
    (``triangle_integrals``), the remainders by the 7-point rule; k = 0
    gives the static kernel g0 alone."""
    tri = mesh.V[mesh.T[t_src]]
    I0, I1, I2 = triangle_integrals(r, tri, mesh.normal[t_src])
    S = I0 / _FOURPI + 0j
    Vv = I1 / _FOURPI + 0j
    U = I2 / _FOURPI + 0j
    if k != 0:
        rp = TRI7_B @ tri                                    # (7,3)
        wp = mesh.area[t_src] * TRI7_W
        d = r[:, None, :] - rp[None, :, :]                   # r - r'
        R = np.sqrt(np.sum(d * d, axis=-1))
        g1, f1 = _smooth_kernels(k, R)
        S = S + (g1 * wp).sum(axis=1)
        Vv = Vv - np.einsum('pq,pqc->pc', g1 * wp, d)
        U = U + np.einsum('pq,pqc->pc', f1 * wp, d)
    return S, Vv, U


def rwg_operators(mesh, k):
    """RWG matrices (n_edges square) of one medium:
    A_vec = int int f . f' G, A_div = int int div f div' f' G and
    K = -int int f . (f' x grad' G) (principal value: a triangle with itself
    gives 0, the integrand being a triple product of vectors in its plane).
    Outer integral: the 7-point rule on the test triangle."""
    nt = len(mesh.T)
    P = mesh.points(TRI7_B)                                  # (nt,7,3)
    W = mesh.area[:, None] * TRI7_W[None, :]
    Avh = np.zeros((3 * nt, 3 * nt), dtype=complex)
    Adh = np.zeros((3 * nt, 3 * nt), dtype=complex)
    Kh = np.zeros((3 * nt, 3 * nt), dtype=complex)
    Vt = mesh.V[mesh.T]                                      # (nt,3,3) corners
    for ts in range(nt):
        S, Vv, U = inner_integrals(mesh, P.reshape(-1, 3), ts, k)
        S, Vv, U = S.reshape(nt, 7), Vv.reshape(nt, 7, 3), U.reshape(nt, 7, 3)
        U[ts] = 0.0
        hb = mesh.h[ts]
        for b in range(3):
            vb = Vt[ts, b]
            # int f_b(r') G dS' = h_b (V + (r - v_b) S); int f_b x grad'G = h_b (r - v_b) x U
            Fb = hb[b] * (Vv + (P - vb) * S[..., None])      # (nt,7,3)
            Cb = hb[b] * np.cross(P - vb, U)
            for a in range(3):
                Ta = mesh.h[:, a][:, None, None] * (P - Vt[:, a][:, None, :])   # test f_a at the points
                Avh[a::3, 3 * ts + b] = np.einsum('tqc,tqc,tq->t', Ta, Fb, W)
                Kh[a::3, 3 * ts + b] = -np.einsum('tqc,tqc,tq->t', Ta, Cb, W)
            Adh[:, 3 * ts + b] = np.repeat((S * W).sum(axis=1), 3) * (2 * mesh.h.ravel()) * 2 * hb[b]
    H = mesh.incidence()
    return H @ Avh @ H.T, H @ Adh @ H.T, H @ Kh @ H.T


class MeshModes:
    """Static modes of a mesh (Sec. III): n_perp transverse (loops, largest
    gamma first) and n_par longitudinal (stars, smallest gamma first)."""

    def __init__(self, mesh, n_perp, n_par):
        self.mesh = mesh
        self.n_perp, self.n_par = int(n_perp), int(n_par)
        G = mesh.gram()
        Av, Ad, _ = rwg_operators(mesh, 0.0)
        Av, Ad = Av.real, Ad.real
        S, L = mesh.stars(), mesh.loops()
        # the exact operators are symmetric; the outer rule against the closed
        # inner integral is not, so the symmetric parts are diagonalised
        Ap, Al = L.T @ Av @ L, S.T @ Ad @ S
        gl, vl = scipy.linalg.eigh(0.5 * (Ap + Ap.T), L.T @ G @ L)     # ascending
        gs, vs = scipy.linalg.eigh(0.5 * (Al + Al.T), S.T @ G @ S)
        self.gamma_perp_all, self.gamma_par_all = gl[::-1], gs
        self.gamma_perp = gl[::-1][:self.n_perp]
        self.gamma_par = gs[:self.n_par]
        Mp = (L @ vl[:, ::-1][:, :self.n_perp]).T
        Ml = (S @ vs[:, :self.n_par]).T
        M = np.vstack([Mp, Ml])
        # sign: the largest RWG coefficient of each mode positive
        idx = np.argmax(np.abs(M), axis=1)
        M *= np.sign(M[np.arange(len(M)), idx])[:, None]
        self.M = M
        self.G = G

    @property
    def n_psi(self):
        return self.n_perp + self.n_par

    def fields(self, bary):
        """Mode fields (n_psi, nt*nq, 3) and divergences (n_psi, nt*nq) at
        the rule points of every triangle, with the points (nt*nq, 3)."""
        mesh = self.mesh
        P = mesh.points(bary)
        nt, nq = P.shape[0], P.shape[1]
        C = self.M[:, mesh.eo] * mesh.h[None, :, :]             # (n_psi, nt, 3)
        Vt = mesh.V[mesh.T]
        psi = np.einsum('nta,taqc->ntqc', C, P[:, None, :, :] - Vt[:, :, None, :])
        div = 2.0 * C.sum(axis=2)                                # per triangle
        return (psi.reshape(self.n_psi, nt * nq, 3),
                np.repeat(div, nq, axis=1), P.reshape(nt * nq, 3))

    def self_block(self, outer, inner):
        """Z_s (Eq. 16 with delta = 1) for media outer, inner (objects with k
        and zeta, e.g. ``oracle.pmchwt.Medium``), compressed by Eq. 20."""
        n = self.n_psi
        blocks = []
        for med in (outer, inner):
            Av, Ad, K = rwg_operators(self.mesh, med.k)
            T = -1j * med.k * Av + (1j / med.k) * Ad
            blocks.append((self.M @ T @ self.M.T, self.M @ K @ self.M.T, med.zeta))
        (To, Ko, zo), (Ti, Ki, zi) = blocks
        Z = np.zeros((2 * n, 2 * n), dtype=complex)
        Z[:n, :n] = zo * To + zi * Ti
        Z[:n, n:] = Ko + Ki
        Z[n:, :n] = -(Ko + Ki)
        Z[n:, n:] = To / zo + Ti / zi
        return Z

    def sampled(self, outer, inner):
        """The shape as the solver takes it (``oracle.pmchwt.SampledShape``):
        3-point rule per triangle, fields, divergences and the self block."""
        psi, div, r = self.fields(TRI3_B)
        w = np.repeat(self.mesh.area, 3) / 3.0
        return SampledShape(r, w, psi, div, self.self_block(outer, inner), self.n_perp, self.n_par)


def _sampled_task(args):
    spec, eps_out, eps_in = args
    from .pmchwt import Medium
    mm = MeshModes(Mesh(spec['verts'], spec['tris']), spec['n_perp'], spec['n_par'])
    return mm.sampled(Medium(eps_out), Medium(eps_in))


def sampled_shapes(specs, eps_in, eps_out=1.0, workers=1):
    """``MeshModes.sampled`` of several mesh specs (dicts with verts, tris,
    n_perp, n_par) for real media, in a pool of spawned processes when
    workers > 1 (each shape independent)."""
    jobs = [(s, eps_out, eps_in) for s in specs]
    if workers <= 1 or len(jobs) <= 1:
        return [_sampled_task(j) for j in jobs]
    import multiprocessing as mp
    with mp.get_context('spawn').Pool(min(workers, len(jobs))) as pool:
        return pool.map(_sampled_task, jobs)
