"""The MLFMA-SMR matrix-vector product, step by step, in FP64 (Sec. IV).

Test infrastructure only (see ``oracle/__init__``).

Steps, in the order the paper composes them:

1. Grouping (Sec. IV, Fig. 1): every particle is its own finest-level group;
   coarser levels are a quadtree over the lattice (parent = 2x2 children by
   integer index).  Near = self + the 8 lattice neighbours; every other pair
   is translated at the finest level where their boxes are not adjacent but
   their parents are (the interaction list, IL).  Off the lattice a particle
   belongs to the cell nearest its centre; where a cell holds several
   particles the finest boxes are the occupied cells (their particles'
   spectra summed), and near pairs are all pairs in the same or adjacent
   cells.
2. k-space sampling (Sec. V): L_0 = 10 at the finest level, K = 2(L+1)^2
   points per level: L+1 Gauss-Legendre nodes in cos(theta) times 2L+2
   uniform phi_j = 2 pi j / (2L+2).  Coarser levels take the paper's
   truncation rule L = kd + 1.8 d0^{2/3} (kd)^{1/3}, d = sqrt(2) x box size
   (Sec. IV, text after Eq. 26, exponent 1/3; the ``double`` rule L_0 2^s is
   available but its Hankel functions overflow the useful range past level 3).
3. Patterns (Eq. 26): psi_hat_n(k) = int psi_n e^{-j k khat.(r - r_mu)} dS
   on the level-0 grid, transverse (theta, phi) components.
4. Aggregation: outgoing spectra of each finest box, four fields
   (A_e theta, A_e phi, A_m theta, A_m phi), A = sum_n alpha_n conj(psi_hat_n),
   shifted from the particle centre to the box centre.
5. Interpolation (4x4 Lagrange, Sec. V) from each child grid to its parent's,
   then the shift exp(j k khat.(c_child - c_parent)), summed over children.
6. Translation (Eqs. 22-23): incoming(b) += T_L(khat, c_b - c_b') outgoing(b').
7. Anterpolation: the quadrature-weighted adjoint W_c^{-1} I^T W_p of the
   interpolation, applied after the shift exp(-j k khat.(c_child - c_parent)).
8. Receive (Eqs. 24-25): y_e += -j k sum_k w psi_hat_m . [zeta B_e + B_m x khat]
   and y_m += -j k sum_k w psi_hat_m . [-B_e x khat + B_m / zeta].
9. Near SpMV: y_mu += sum_{nu in near(mu)} Z^{mu nu} x_nu.
"""
import math

import numpy as np
import scipy.sparse as sps

from .pmchwt import exterior_block
from .special import gauss_legendre, legendre_upto, sph_h2, sphere_frame


# ---------------------------------------------------------------- grouping
class Tree:
    """Quadtree over particles on a square lattice of spacing ``pitch``."""

    def __init__(self, centres, pitch):
        C = np.asarray(centres, dtype=float)
        self.pitch = float(pitch)
        self.origin = C[:, :2].min(axis=0)
        self.z0 = float(C[:, 2].mean())
        ij = np.rint((C[:, :2] - self.origin) / self.pitch).astype(np.int64)
        self.ij0 = ij
        # one particle per cell: the finest boxes are the particles, in their
        # order; else the occupied cells, ordered like every coarser level
        self.one_per_cell = len({tuple(t) for t in ij}) == len(ij)
        self.members = {}         # cell -> its particles, ascending
        for mu, t in enumerate(ij):
            self.members.setdefault(tuple(t), []).append(mu)
        self.levels = []          # per level: dict(ij, centre, index, parent)
        ij_s = ij
        s = 0
        while True:
            if s == 0 and self.one_per_cell:
                keys = ij
            else:
                keys = np.unique(ij_s, axis=0)
                keys = keys[np.lexsort((keys[:, 0], keys[:, 1]))]
            index = {tuple(t): n for n, t in enumerate(keys)}
            cen = np.zeros((len(keys), 3))
            half = (2 ** s - 1) / 2.0
            cen[:, :2] = self.origin + (keys * 2 ** s + half) * self.pitch
            cen[:, 2] = self.z0
            self.levels.append(dict(ij=keys, centre=cen, index=index))
            self.levels[-1]['il'] = self._interaction_list(s)
            # entries of target b are il[il_ptr[b]:il_ptr[b + 1]] (listed by target)
            tb = np.array([e[0] for e in self.levels[-1]['il']], dtype=np.int64)
            self.levels[-1]['il_ptr'] = np.searchsorted(tb, np.arange(len(keys) + 1))
            if np.max(keys.max(axis=0) - keys.min(axis=0)) <= 1:
                break                      # every box adjacent: nothing above
            ij_s = keys // 2
            s += 1
        while len(self.levels) > 1 and not self.levels[-1]['il']:
            self.levels.pop()
        # the finest box of every particle
        idx0 = self.levels[0]['index']
        self.cell = np.array([idx0[tuple(t)] for t in ij], dtype=np.int64)
        # parents / children
        for s in range(len(self.levels) - 1):
            par = self.levels[s + 1]['index']
            self.levels[s]['parent'] = np.array([par[tuple(t // 2)] for t in self.levels[s]['ij']])
        self.n_levels = len(self.levels)

    def _interaction_list(self, s):
        """(b, b', (dx, dy)) with parents adjacent or equal, boxes not adjacent."""
        lev = self.levels[s]
        out = []
        for b, t in enumerate(lev['ij']):
            px, py = t // 2
            for qx in (px - 1, px, px + 1):
                for qy in (py - 1, py, py + 1):
                    for cx in (2 * qx, 2 * qx + 1):
                        for cy in (2 * qy, 2 * qy + 1):
                            if max(abs(cx - t[0]), abs(cy - t[1])) <= 1:
                                continue
                            bb = lev['index'].get((cx, cy))
                            if bb is not None:
                                out.append((b, bb, (int(t[0] - cx), int(t[1] - cy))))
        return out

    def near_pairs(self, mus=None):
        """(mu, nu) with nu in mu's cell or one of the 8 neighbouring cells
        (self included), for the particles mus (default all) in ascending
        order."""
        out = []
        for mu in (range(len(self.ij0)) if mus is None else mus):
            t = self.ij0[mu]
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    for nu in self.members.get((t[0] + dx, t[1] + dy), ()):
                        out.append((mu, nu))
        return out


# ---------------------------------------------------------------- k-space
def truncation(k, box, level, L0=10, rule='formula', digits=3.0):
    """Truncation order L at a level (see module docstring, step 2)."""
    if level == 0:
        return L0
    if rule == 'double':
        return L0 * 2 ** level
    kd = k * math.sqrt(2.0) * box * 2 ** level
    return int(math.ceil(kd + 1.8 * digits ** (2.0 / 3.0) * kd ** (1.0 / 3.0)))


class Grid:
    """K = (L+1)(2L+2) directions: theta ascending (GL in cos theta), phi_j = 2 pi j / N_phi."""

    def __init__(self, L):
        self.L = L
        self.n_theta = L + 1
        self.n_phi = 2 * L + 2
        x, w = gauss_legendre(self.n_theta)
        self.theta = np.arccos(x)
        self.w_theta = w
        self.phi = 2.0 * np.pi * np.arange(self.n_phi) / self.n_phi
        TH, PH = np.meshgrid(self.theta, self.phi, indexing='ij')
        self.khat, self.that, self.phat = sphere_frame(TH.ravel(), PH.ravel())
        self.w = np.outer(w, np.full(self.n_phi, 2.0 * np.pi / self.n_phi)).ravel()

    @property
    def K(self):
        return self.n_theta * self.n_phi


def lagrange_weights(nodes, t):
    """Lagrange basis values at t for the given nodes."""
    n = len(nodes)
    out = np.ones(n)
    for a in range(n):
        for b in range(n):
            if b != a:
                out[a] *= (t - nodes[b]) / (nodes[a] - nodes[b])
    return out


def interpolation_matrix(src, dst):
    """Sparse (K_dst x K_src) 4x4 Lagrange interpolation of a (theta, phi)
    component field, with the stencil reflected through the poles:
    (-theta, phi) == (theta, phi + pi) and both spherical components change
    sign there.  Stencil: theta nodes i0-1..i0+2 with i0 the last node
    <= theta_t; phi nodes j0-1..j0+2 with j0 = floor(phi_t / dphi)."""
    nt, nph = src.n_theta, src.n_phi
    # extended theta nodes: index i in [-2, nt+1]
    def ext(i):
        if i < 0:
            return -src.theta[-1 - i], -1 - i, True
        if i >= nt:
            return 2 * np.pi - src.theta[2 * nt - 1 - i], 2 * nt - 1 - i, True
        return src.theta[i], i, False
    rows, cols, vals = [], [], []
    dphi = 2 * np.pi / nph
    for it, tt in enumerate(dst.theta):
        i0 = int(np.searchsorted(src.theta, tt, side='right')) - 1   # last node <= tt
        taps = [ext(i) for i in range(i0 - 1, i0 + 3)]
        wt = lagrange_weights(np.array([t[0] for t in taps]), tt)
        for jp, pt in enumerate(dst.phi):
            j0 = int(math.floor(pt / dphi))
            jn = np.arange(j0 - 1, j0 + 3)
            wp = lagrange_weights(jn * dphi, pt)
            r = it * dst.n_phi + jp
            for a, (_, isrc, refl) in enumerate(taps):
                for b in range(4):
                    j = jn[b] + (nph // 2 if refl else 0)
                    rows.append(r)
                    cols.append(isrc * nph + (j % nph))
                    vals.append(wt[a] * wp[b] * (-1.0 if refl else 1.0))
    return sps.csr_matrix((vals, (rows, cols)), shape=(dst.K, src.K))


def _interp_task(args):
    return interpolation_matrix(*args)


def _translation_task(args):
    return translation_function(*args)


def translation_function(k, L, khat, X):
    """T_L(khat, X) of Eq. 23 for all rows of khat (K,3), X a 3-vector."""
    X = np.asarray(X, dtype=float)
    r = np.linalg.norm(X)
    c = khat @ (X / r)
    out = np.zeros(khat.shape[0], dtype=complex)
    P = legendre_upto(L, c)
    for l in range(L + 1):
        out += (-1j) ** l * (2 * l + 1) * sph_h2(l, k * r) * P[l]
    return (-1j * k / (4 * np.pi) ** 2) * out


# ---------------------------------------------------------------- operator
class MLFMA:
    """MLFMA operator of a Scene on a square lattice of spacing ``pitch``."""

    def __init__(self, scene, pitch, L0=10, rule='formula', digits=3.0, pmap=map):
        """pmap: a map function (e.g. a process pool's) for the independent
        interpolation matrices and translation tables; the values are the
        same whichever map computes them."""
        self.scene = scene
        self.tree = Tree(scene.centres, pitch)
        k = scene.outer.k
        self.k = k
        self.zeta = scene.outer.zeta
        self.grids = [Grid(truncation(k, pitch, s, L0, rule, digits))
                      for s in range(self.tree.n_levels)]
        self.interp = list(pmap(_interp_task, [(self.grids[s], self.grids[s + 1])
                                                for s in range(self.tree.n_levels - 1)]))
        self.patterns = [self._pattern(s) for s in range(len(scene.shapes))]
        keys, tasks = [], []
        for s, lev in enumerate(self.tree.levels):
            box = pitch * 2 ** s
            for o in sorted({o for (_, _, o) in lev['il']}):
                keys.append((s, o))
                tasks.append((k, self.grids[s].L, self.grids[s].khat, (o[0] * box, o[1] * box, 0.0)))
        self.T = [dict() for _ in self.tree.levels]
        for (s, o), tab in zip(keys, pmap(_translation_task, tasks)):
            self.T[s][o] = tab
        self._near_cache = {}

    # ---- setup
    def _pattern(self, s):
        """(N_psi, 2, K_0) receiving patterns psi_hat . (theta_hat, phi_hat), Eq. 26."""
        rule, psi, _ = self.scene.shape_data(s)
        g = self.grids[0]
        ph = np.exp(-1j * self.k * (g.khat @ rule['r'].T)) * rule['w'][None, :]   # (K, Q)
        vec = np.einsum('kq,nqc->nkc', ph, psi)
        return np.stack([np.einsum('nkc,kc->nk', vec, g.that),
                         np.einsum('nkc,kc->nk', vec, g.phat)], axis=1)

    def near_block(self, mu, nu):
        sc = self.scene
        sm, sn = sc.shape_ids[mu], sc.shape_ids[nu]
        if mu == nu:
            key = ('self', sm)
            if key not in self._near_cache:
                self._near_cache[key] = sc.self_block(sm)
        else:
            d = tuple(self.tree.ij0[mu] - self.tree.ij0[nu])
            dc = sc.centres[mu] - sc.centres[nu]
            key = (sm, sn, d) + tuple(np.round(dc, 12))
            if key not in self._near_cache:
                self._near_cache[key] = exterior_block(sc, sm, dc, sn, np.zeros(3))
        return self._near_cache[key]

    # ---- steps
    # Every step takes an optional subset of the boxes (or particles) it
    # writes and an optional output array: a subset's rows are computed with
    # exactly the operations, in exactly the order, of the full step, so
    # disjoint subsets can run in separate processes (oracle.parallel).
    def near(self, x, mus=None, out=None):
        sc = self.scene
        n2 = 2 * sc.n_psi
        xx = x.reshape(sc.p, n2)
        y = np.zeros_like(xx) if out is None else out.reshape(sc.p, n2)
        if mus is not None:
            y[mus] = 0.0
        for mu, nu in self.tree.near_pairs(mus):
            y[mu] += self.near_block(mu, nu) @ xx[nu]
        return y.reshape(-1)

    def aggregate(self, x, mus=None, out=None, boxes=None):
        """Level-0 outgoing spectra (n_box_0, K_0, 4): each particle's, shifted
        from its centre to its cell's, summed over the cell's particles.
        `mus` (one particle per cell) or `boxes` restrict the rows written."""
        sc = self.scene
        xx = x.reshape(sc.p, 2, sc.n_psi)
        g = self.grids[0]
        t = self.tree
        assert mus is None or t.one_per_cell, "particle subsets need one particle per cell"
        if out is None:
            out = np.zeros((len(t.levels[0]['ij']), g.K, 4), dtype=complex)
        cen = t.levels[0]['centre']
        if boxes is not None:
            out[boxes] = 0.0
            mus = [mu for b in boxes for mu in t.members[tuple(t.levels[0]['ij'][b])]]
        for mu in (range(sc.p) if mus is None else mus):
            b = t.cell[mu]
            P = self.patterns[sc.shape_ids[mu]]               # (N, 2, K)
            shift = np.exp(1j * self.k * (g.khat @ (sc.centres[mu] - cen[b])))
            for c in range(2):
                for comp in range(2):
                    v = shift * (xx[mu, c] @ np.conj(P[:, comp, :]))
                    if t.one_per_cell and boxes is None:
                        out[b, :, 2 * c + comp] = v
                    else:
                        out[b, :, 2 * c + comp] += v
        return out

    def upward(self, s, out_s, parents=None, out=None):
        """Level s+1 outgoing spectra from level s (interpolate, shift, sum)."""
        lev, par = self.tree.levels[s], self.tree.levels[s + 1]
        gp = self.grids[s + 1]
        if out is None:
            out = np.zeros((len(par['ij']), gp.K, 4), dtype=complex)
        I = self.interp[s]
        children = range(len(lev['ij']))
        if parents is not None:
            out[parents] = 0.0
            keep = np.zeros(len(par['ij']), dtype=bool)
            keep[parents] = True
            children = [c for c in children if keep[lev['parent'][c]]]
        for c in children:
            B = lev['parent'][c]
            shift = np.exp(1j * self.k * (gp.khat @ (lev['centre'][c] - par['centre'][B])))
            out[B] += shift[:, None] * (I @ out_s[c])
        return out

    def translate(self, s, out_s, targets=None, inc=None):
        lev = self.tree.levels[s]
        if inc is None:
            inc = np.zeros_like(out_s)
        il = lev['il']
        if targets is not None:
            inc[targets] = 0.0
            ptr = lev['il_ptr']
            il = [e for b in targets for e in il[ptr[b]:ptr[b + 1]]]
        for (b, bb, o) in il:
            inc[b] += self.T[s][o][:, None] * out_s[bb]
        return inc

    def downward(self, s, in_parent, children=None, out=None):
        """Contribution to level-s incoming spectra from level s+1."""
        lev, par = self.tree.levels[s], self.tree.levels[s + 1]
        gc, gp = self.grids[s], self.grids[s + 1]
        I = self.interp[s]
        if out is None:
            out = np.zeros((len(lev['ij']), gc.K, 4), dtype=complex)
        for c in (range(len(lev['ij'])) if children is None else children):
            B = lev['parent'][c]
            shift = np.exp(-1j * self.k * (gp.khat @ (lev['centre'][c] - par['centre'][B])))
            v = (gp.w * shift)[:, None] * in_parent[B]
            out[c] = (I.T @ v) / gc.w[:, None]
        return out

    def receive(self, inc0, mus=None, out=None):
        sc = self.scene
        g = self.grids[0]
        k, z = self.k, self.zeta
        cen = self.tree.levels[0]['centre']
        y = np.zeros((sc.p, 2, sc.n_psi), dtype=complex) if out is None else out.reshape(sc.p, 2, sc.n_psi)
        for mu in (range(sc.p) if mus is None else mus):
            b = self.tree.cell[mu]
            P = self.patterns[sc.shape_ids[mu]]
            shift = np.exp(-1j * k * (g.khat @ (sc.centres[mu] - cen[b])))
            B = inc0[b] * (g.w * shift)[:, None]
            Bet, Bep, Bmt, Bmp = B[:, 0], B[:, 1], B[:, 2], B[:, 3]
            y[mu, 0] = -1j * k * (P[:, 0, :] @ (z * Bet + Bmp) + P[:, 1, :] @ (z * Bep - Bmt))
            y[mu, 1] = -1j * k * (P[:, 0, :] @ (-Bep + Bmt / z) + P[:, 1, :] @ (Bet + Bmp / z))
        return y.reshape(-1)

    def far(self, x):
        """Far-field part of the product (steps 4-8)."""
        nl = self.tree.n_levels
        outs = [self.aggregate(x)]
        for s in range(nl - 1):
            outs.append(self.upward(s, outs[s]))
        ins = [self.translate(s, outs[s]) for s in range(nl)]
        for s in range(nl - 2, -1, -1):
            ins[s] = ins[s] + self.downward(s, ins[s + 1])
        return self.receive(ins[0])

    def matvec(self, x):
        x = np.asarray(x, dtype=complex).reshape(-1)
        return self.near(x) + self.far(x)
