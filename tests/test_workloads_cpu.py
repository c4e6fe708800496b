"""The seeded input generators (no method arithmetic): the geometry the
off-lattice, rotated and two-layer workloads promise."""
from collections import Counter

import numpy as np

from paper_2407_21724_gb300 import workloads


def _cells(C, pitch):
    f = (C[:, :2] - C[:, :2].min(axis=0)) / pitch
    ij = np.rint(f).astype(int)
    return ij, (f - ij) * pitch


def test_box_mesh_is_closed_and_outward():
    V, T = workloads.box_mesh(0.3, 0.1, 0.5, 6, 2, 7)
    assert len(T) == 4 * (6 * 2 + 2 * 7 + 6 * 7)
    edges = Counter()
    for a, b, c in T:
        for e in ((a, b), (b, c), (c, a)):
            edges[e] += 1
    # every directed edge once, and its reverse once: closed and consistently oriented
    assert all(v == 1 for v in edges.values()) and all(edges[(b, a)] == 1 for (a, b) in edges)
    n = np.cross(V[T[:, 1]] - V[T[:, 0]], V[T[:, 2]] - V[T[:, 0]])
    vol = np.sum(np.einsum('ij,ij->i', V[T[:, 0]], n)) / 6
    assert abs(vol - 0.3 * 0.1 * 0.5) < 1e-12


def test_spirals():
    # the paper's positions: i = 1..n at c sqrt(i), angle i * 2 pi / phi^2
    w = workloads.make("spiral_dense", n=50, R=0.1)
    C = w["centres"]
    ga = 2 * np.pi / ((1 + np.sqrt(5)) / 2) ** 2
    i = np.arange(1, 51)
    assert np.allclose(np.hypot(C[:, 0], C[:, 1]), np.sqrt(3) * 0.1 * np.sqrt(i))
    assert np.allclose(np.angle(C[:, 0] + 1j * C[:, 1]), np.angle(np.exp(1j * i * ga)))
    # the sparse spiral keeps one centre per cell and its particles within the cell
    w = workloads.make("spiral", n=400)
    ij, d = _cells(w["centres"], w["pitch"])
    assert len({tuple(t) for t in ij}) == len(ij)
    assert np.max(np.hypot(d[:, 0], d[:, 1])) + max(r for r, _, _ in w["shapes"]) < w["pitch"]
    # the dense one has cells with several centres
    ij, _ = _cells(workloads.make("spiral_dense", n=400)["centres"], 0.5)
    assert max(Counter(map(tuple, ij)).values()) > 1


def test_jitter_and_moire():
    w0 = workloads.make("random", n=10, seed=3)
    w = workloads.make("jittered", n=10, seed=3, jitter=0.02)
    d = w["centres"] - w0["centres"]
    assert np.all(np.abs(d[:, :2]) <= 0.02) and np.all(d[:, 2] == 0) and np.any(d != 0)
    assert np.array_equal(w["shape_ids"], w0["shape_ids"])
    m = workloads.make("moire", m=6, shape="sphere")
    C = m["centres"]
    lo, hi = C[C[:, 2] < 0], C[C[:, 2] > 0]
    assert len(lo) == len(hi) == 2 * 36 and np.allclose(hi[:, 2] - lo[:, 2], 0.5)
    # the upper layer is the lower one turned by 5 degrees
    a = np.radians(5.0)
    R = np.array([[np.cos(a), -np.sin(a)], [np.sin(a), np.cos(a)]])
    assert np.allclose(lo[:, :2] @ R.T, hi[:, :2])
    # nearest neighbours in a layer are one honeycomb side apart
    dd = np.sqrt(((lo[:, None, :2] - lo[None, :, :2]) ** 2).sum(-1))
    np.fill_diagonal(dd, np.inf)
    assert np.isclose(dd.min(), 400 / 600)


def test_pb_lens_angles():
    w = workloads.make("pbfins", n=12, bins=16)
    th = workloads.pb_angles(w["centres"], w["focal"])
    assert np.all((th >= 0) & (th < np.pi))
    b = w["shape_ids"]
    assert b.min() >= 0 and b.max() < 16
    err = np.angle(np.exp(2j * (th - b * np.pi / 16))) / 2       # modulo pi
    assert np.max(np.abs(err)) <= np.pi / 32 + 1e-12
    assert [s["angle"] for s in w["shapes"][1:]] == [k * np.pi / 16 for k in range(1, 16)]
