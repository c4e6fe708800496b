"""The process-parallel oracle product (used only to time the CPU baseline)
is bit-identical to the serial oracle product, and each step with a subset
of its boxes reproduces those rows of the full step."""
import numpy as np

from oracle import mlfma as oml
from oracle import pmchwt as opm
from oracle.parallel import ParallelMLFMA
from paper_2407_21724_gb300 import workloads


def test_parallel_oracle_product_is_bit_identical():
    # 12 x 12 (3 levels) with two radii, so that few distinct near blocks
    # need computing
    w = workloads.make("random", n=12, seed=9, modes=4)
    w["shape_ids"] = w["shape_ids"] % 2
    sc = opm.Scene(w["centres"], w["shape_ids"], w["shapes"][:2], eps_in=w["eps_in"])
    rng = np.random.default_rng(3)
    x = rng.standard_normal(sc.n_unknowns) + 1j * rng.standard_normal(sc.n_unknowns)
    y0 = oml.MLFMA(sc, w["pitch"]).matvec(x)
    P = ParallelMLFMA(sc, w["pitch"], workers=3)
    try:
        y1 = P.matvec(x)
        y2 = P.matvec(x)
    finally:
        P.close()
    assert np.array_equal(y0, y1) and np.array_equal(y1, y2)


def test_parallel_oracle_product_with_shared_cells_is_bit_identical():
    # the paper's spiral spacing: up to 4 particles per cell, the level-0
    # boxes written by box subsets
    w = workloads.make("spiral_dense", n=24, R=0.1, modes=3)
    sc = opm.Scene(w["centres"], w["shape_ids"], w["shapes"], eps_in=w["eps_in"], n_theta=8, n_phi=16)
    rng = np.random.default_rng(4)
    x = rng.standard_normal(sc.n_unknowns) + 1j * rng.standard_normal(sc.n_unknowns)
    M = oml.MLFMA(sc, w["pitch"])
    assert not M.tree.one_per_cell
    y0 = M.matvec(x)
    P = ParallelMLFMA(sc, w["pitch"], workers=3)
    try:
        y1 = P.matvec(x)
    finally:
        P.close()
    assert np.array_equal(y0, y1)
