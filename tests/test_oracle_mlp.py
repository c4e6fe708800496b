"""Pins of the learned-part oracle: backpropagation against central
differences, and the neighbourhood features against their definition."""
import numpy as np

from oracle import mlp
from paper_2407_21724_gb300 import workloads


def test_backprop_matches_central_differences():
    dims = [12, 7, 6, 5, 4]
    p = workloads.mlp_params(dims, 3).astype(np.float64)
    rng = np.random.default_rng(1)
    X = rng.standard_normal((9, 12))
    T = rng.standard_normal((9, 4))
    loss, g = mlp.loss_grad(p, dims, X, T)
    h = 1e-6
    fd = np.zeros_like(p)
    for i in range(p.size):
        e = np.zeros_like(p)
        e[i] = h
        fd[i] = (mlp.loss_grad(p + e, dims, X, T)[0] - mlp.loss_grad(p - e, dims, X, T)[0]) / (2 * h)
    assert np.linalg.norm(g - fd) / np.linalg.norm(fd) < 1e-7


def test_slots_are_the_48_lattice_points_within_two_wavelengths():
    sl = mlp.slots()
    assert len(sl) == 48 and len(set(sl)) == 48
    d2 = [dx * dx + dy * dy for dx, dy in sl]
    assert d2 == sorted(d2) and d2[0] == 1 and d2[-1] == 16


def test_features_count_neighbours():
    w = workloads.make("random", n=9, seed=2, modes=16)
    C = w["centres"]
    F = mlp.features(C, w["shape_ids"], np.zeros(len(C), dtype=int), [[0, 0, 1.0]], [[1, 0, 0]])
    assert F.shape == (81, 448)
    centre = 4 * 9 + 4                        # middle of the 9x9 array: every slot present
    assert F[centre, 8:432:9].sum() == 48
    corner = 0                                # corner: quarter disc without the axes' far side
    expect = sum(1 for dx, dy in mlp.slots() if dx >= 0 and dy >= 0)
    assert F[corner, 8:432:9].sum() == expect
    assert np.all(F[:, 432:440].sum(axis=1) == 1)
    # one-hot of each present neighbour matches its shape id
    s = 0
    dx, dy = mlp.slots()[s]
    nb = (4 + dy) * 9 + (4 + dx)
    assert F[centre, 9 * s + w["shape_ids"][nb]] == 1.0
