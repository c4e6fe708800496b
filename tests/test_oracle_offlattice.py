"""Pins of the oracle on particles off the lattice (Sec. V, non-lattice
arrays): a jittered lattice, a sparse golden-angle spiral, the paper's dense
spiral (several particles per finest cell) and a two-layer scene whose layers
are 0.5 wavelengths apart (the 2.5D bilayer of Sec. V on one quadtree).

The MLFMA product is pinned against the dense Galerkin product, whose
exterior blocks are computed for the exact centre offsets with no expansion
at all; FMM accuracy at L0 = 10 and its improvement with L0 carry over from
the lattice.  Two planted mistakes in the oracle's centre shifts (the shift
between a particle and its finest-group centre dropped, or its sign flipped
in aggregation and receive) fail the same bar by a wide margin, and every
ordered pair is still covered once by near pairs plus interaction lists.
"""
import math

import numpy as np
import pytest

from oracle import mlfma as ml
from oracle import pmchwt as pm
from paper_2407_21724_gb300 import workloads


def _scene(C, ids):
    return pm.Scene(C, ids, [(0.10, 8, 8), (0.14, 8, 8)], eps_in=4.0, n_theta=12, n_phi=24)


@pytest.fixture(scope="module")
def jittered():
    C = workloads.lattice(5, 5)
    rng = np.random.default_rng(11)
    d = np.zeros_like(C)
    d[:, :2] = rng.uniform(-0.08, 0.08, size=(25, 2))
    ids = rng.integers(0, 2, size=25)
    lat = C.copy()
    sc = _scene(C + d, ids)
    return sc, pm.dense_matrix(sc), lat, ids


@pytest.fixture(scope="module")
def spiral():
    w = workloads.make("spiral", n=24, d_min=0.75)
    sc = _scene(w["centres"], w["shape_ids"] % 2)
    return sc, pm.dense_matrix(sc)


def _x(n, seed=0):
    rng = np.random.default_rng(seed)
    return (rng.standard_normal(n) + 1j * rng.standard_normal(n)) / math.sqrt(2)


def _err(M, Z, x):
    y0 = Z @ x
    return np.linalg.norm(M.matvec(x) - y0) / np.linalg.norm(y0)


def test_tree_covers_every_pair_once_off_lattice(jittered, spiral):
    for sc in (jittered[0], spiral[0]):
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


def test_offlattice_mlfma_matches_dense(jittered, spiral):
    for sc, Z in (jittered[:2], spiral):
        x = _x(Z.shape[0])
        e10 = _err(ml.MLFMA(sc, 0.5, L0=10), Z, x)
        e16 = _err(ml.MLFMA(sc, 0.5, L0=16), Z, x)
        assert e10 < 1e-3 and e16 < e10 / 3, (e10, e16)


class _Shifted(ml.MLFMA):
    """The oracle with its aggregation and receive shifts taken from other
    centres (a planted mistake); near blocks keep the true offsets."""

    def __init__(self, sc, pitch, fake):
        super().__init__(sc, pitch)
        self.fake = fake

    def _with(self, f, *a, **k):
        saved = self.scene.centres
        self.scene.centres = self.fake
        try:
            return f(*a, **k)
        finally:
            self.scene.centres = saved

    def aggregate(self, *a, **k):
        return self._with(super().aggregate, *a, **k)

    def receive(self, *a, **k):
        return self._with(super().receive, *a, **k)


def test_planted_shift_mistakes_are_caught(jittered):
    sc, Z, lat, _ = jittered
    x = _x(Z.shape[0])
    e = _err(ml.MLFMA(sc, 0.5), Z, x)
    dropped = _err(_Shifted(sc, 0.5, lat), Z, x)                  # displacement ignored
    flipped = _err(_Shifted(sc, 0.5, 2 * lat - sc.centres), Z, x)  # sign of the shift flipped
    assert dropped > 20 * e and flipped > 20 * e, (e, dropped, flipped)


@pytest.fixture(scope="module")
def dense_spiral():
    """The paper's spacing: c = sqrt(3) R, here with R = 0.1 (neighbours about
    1.4 diameters apart), so a 0.5-wavelength cell holds up to 3 centres."""
    n, R = 30, 0.1
    i = np.arange(1, n + 1)
    ga = 2 * np.pi / ((1 + np.sqrt(5)) / 2) ** 2
    C = np.zeros((n, 3))
    C[:, 0], C[:, 1] = np.sqrt(3) * R * np.sqrt(i) * np.cos(i * ga), np.sqrt(3) * R * np.sqrt(i) * np.sin(i * ga)
    sc = pm.Scene(C, np.arange(n) % 2, [(R, 8, 8), (0.8 * R, 8, 8)], eps_in=4.0, n_theta=12, n_phi=24)
    return sc, pm.dense_matrix(sc)


@pytest.fixture(scope="module")
def bilayer():
    """Two 3 x 3 layers of spheres at z = -0.25 and 0.25, the upper one
    turned by 5 degrees about z and shifted; cells of 0.6 wavelengths."""
    lo = workloads.lattice(3, 3, pitch=0.66)
    a = np.radians(5.0)
    R = np.array([[np.cos(a), -np.sin(a), 0], [np.sin(a), np.cos(a), 0], [0, 0, 1.0]])
    hi = lo @ R.T + [0.2, 0.1, 0.0]
    lo[:, 2], hi[:, 2] = -0.25, 0.25
    C = np.vstack([lo, hi])
    sc = pm.Scene(C, np.r_[np.zeros(9, int), np.ones(9, int)], [(0.1, 8, 8), (0.08, 8, 8)], eps_in=4.0,
                  n_theta=12, n_phi=24)
    return sc, pm.dense_matrix(sc)


def test_several_particles_per_cell(dense_spiral, bilayer):
    for (sc, Z), pitch in ((dense_spiral, 0.5), (bilayer, 0.6)):
        t = ml.Tree(sc.centres, pitch)
        assert not t.one_per_cell
        # every ordered pair once: near pairs plus interaction lists
        count = np.zeros((sc.p, sc.p), dtype=int)
        for (mu, nu) in t.near_pairs():
            count[mu, nu] += 1
        anc = [t.cell]
        for s in range(t.n_levels - 1):
            anc.append(t.levels[s]['parent'][anc[-1]])
        for s, lev in enumerate(t.levels):
            for (b, bb, _) in lev['il']:
                count[np.ix_(anc[s] == b, anc[s] == bb)] += 1
        assert np.all(count == 1)
        x = _x(Z.shape[0])
        e10 = _err(ml.MLFMA(sc, pitch, L0=10), Z, x)
        e16 = _err(ml.MLFMA(sc, pitch, L0=16), Z, x)
        assert e10 < 2e-3 and e16 < e10 / 3, (e10, e16)


class _LastOnly(ml.MLFMA):
    """Planted: a cell's spectrum is its last particle's, not the sum."""

    def aggregate(self, x, mus=None, out=None):
        t = self.tree
        t.one_per_cell = True
        try:
            return super().aggregate(x, mus, out)
        finally:
            t.one_per_cell = False


def test_planted_cell_sum_mistake_is_caught(dense_spiral):
    sc, Z = dense_spiral
    x = _x(Z.shape[0])
    e = _err(ml.MLFMA(sc, 0.5), Z, x)
    assert _err(_LastOnly(sc, 0.5), Z, x) > 20 * e
