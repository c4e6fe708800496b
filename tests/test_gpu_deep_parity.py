"""Element-wise parity with the FP64 oracle on a tree as deep as the
metalens's: a 200 x 200 random-radius lattice thinned to 2 % of its sites
(seeded), so the oracle finishes in about a minute while the tree keeps the
lens's 7 levels (L up to 309) and its upper-level box counts (166, 49, 16
boxes at levels 4-6 against the lens's 169, 49, 16).  The context is set up
the way the benchmark runs: launch variants autotuned for the FP32 product,
tensor cores on, products through captured CUDA graphs.  Checked:
  - every level's outgoing and incoming spectra of the FP64 product <= 1e-12,
    and the FP64 product <= 1e-10 (the product's stated bar);
  - the FP32 product <= 2e-5 and its level spectra <= 1e-5 (the tuned
    single-precision kernels at every level)."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from oracle import mlfma as oml
from oracle import pmchwt as opm
from paper_2407_21724_gb300 import smr, workloads


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


@pytest.fixture(scope="module")
def deep():
    w = workloads.make("sparse", n=200, fill=0.02, seed=21727)
    ctx = smr.scene_from_workload(w)
    smr.smr_autotune(ctx, smr.SMR_PREC_FP32)
    info = smr.smr_info(ctx)
    sc = opm.Scene(w["centres"], w["shape_ids"], w["shapes"], eps_in=w["eps_in"])
    M = oml.MLFMA(sc, w["pitch"])
    rng = np.random.default_rng(7)
    n = info["n_unknowns"]
    x = (rng.standard_normal(n) + 1j * rng.standard_normal(n)) / math.sqrt(2)
    outs = [M.aggregate(x)]
    for s in range(M.tree.n_levels - 1):
        outs.append(M.upward(s, outs[s]))
    ins = [M.translate(s, outs[s]) for s in range(M.tree.n_levels)]
    for s in range(M.tree.n_levels - 2, -1, -1):
        ins[s] = ins[s] + M.downward(s, ins[s + 1])
    y = M.near(x) + M.receive(ins[0])
    yield dict(ctx=ctx, info=info, M=M, x=x, outs=outs, ins=ins, y=y)
    smr.smr_destroy(ctx)


def _graph_product(d, prec):
    xd = torch.from_numpy(d["x"]).cuda()
    yd = torch.empty_like(xd)
    smr.smr_matvec_graph(d["ctx"], xd, yd, prec)
    smr.smr_sync(d["ctx"])
    return yd.cpu().numpy()


def test_deep_tree_matches_oracle_structure(deep):
    info, t = deep["info"], deep["M"].tree
    assert info["n_levels"] == t.n_levels == 7
    assert info["L"] == [g.L for g in deep["M"].grids]
    for s in range(t.n_levels):
        assert info["n_box"][s] == len(t.levels[s]["ij"])
        assert info["n_il"][s] == len(t.levels[s]["il"])


def test_deep_fp64_level_spectra_and_product(deep):
    y = _graph_product(deep, smr.SMR_PREC_FP64)
    for s in range(deep["M"].tree.n_levels):
        go = smr.smr_copy_level(deep["ctx"], s, 0)[..., 0]
        gi = smr.smr_copy_level(deep["ctx"], s, 1)[..., 0]
        assert rel(go, deep["outs"][s]) < 1e-12, ("out", s, rel(go, deep["outs"][s]))
        assert rel(gi, deep["ins"][s]) < 1e-12, ("in", s, rel(gi, deep["ins"][s]))
    assert rel(y, deep["y"]) < 1e-10


def test_deep_fp32_level_spectra_and_product(deep):
    y = _graph_product(deep, smr.SMR_PREC_FP32)
    for s in range(deep["M"].tree.n_levels):
        go = smr.smr_copy_level(deep["ctx"], s, 0)[..., 0]
        gi = smr.smr_copy_level(deep["ctx"], s, 1)[..., 0]
        assert rel(go, deep["outs"][s]) < 1e-5, ("out", s, rel(go, deep["outs"][s]))
        assert rel(gi, deep["ins"][s]) < 1e-5, ("in", s, rel(gi, deep["ins"][s]))
    assert rel(y, deep["y"]) < 2e-5


def _direct_product(d, prec):
    xd = torch.from_numpy(d["x"]).cuda()
    yd = torch.empty_like(xd)
    smr.smr_matvec(d["ctx"], xd, yd, prec)
    smr.smr_sync(d["ctx"])
    return yd.cpu().numpy()


VARIANTS = [(smr.SMR_STEP_INTERPOLATE, v) for v in (0, 1, 2, 3)] + \
           [(smr.SMR_STEP_ANTERPOLATE, v) for v in (0, 1, 2, 4, 5)] + \
           [(smr.SMR_STEP_TRANSLATE, v) for v in (1, 2, 3, 4, 5)]


@pytest.mark.parametrize("prec", [smr.SMR_PREC_FP64, smr.SMR_PREC_FP32])
def test_deep_every_launch_variant(deep, prec):
    """Every launch variant the autotuner can choose, forced at every level
    in turn (staged and gather interpolation and anterpolation, the
    per-parent anterpolation, every translation tiling), gives the oracle's
    product: FP64 <= 1e-10, FP32 <= 2e-5; for the staged and per-parent FP32
    kernels every level spectrum <= 1e-5."""
    ctx = deep["ctx"]
    try:
        for step, v in VARIANTS:
            smr.smr_set_variant(ctx, step, -1, prec, v)
            y = _direct_product(deep, prec)
            assert rel(y, deep["y"]) < (1e-10 if prec == smr.SMR_PREC_FP64 else 2e-5), (step, v)
            staged = (step == smr.SMR_STEP_INTERPOLATE and v in (0, 3)) or \
                (step == smr.SMR_STEP_ANTERPOLATE and v in (4, 5)) or (step == smr.SMR_STEP_TRANSLATE and v == 5)
            if staged and prec == smr.SMR_PREC_FP32:
                for s in range(deep["M"].tree.n_levels):
                    go = smr.smr_copy_level(ctx, s, 0)[..., 0]
                    gi = smr.smr_copy_level(ctx, s, 1)[..., 0]
                    assert rel(go, deep["outs"][s]) < 1e-5, ("out", s, step, v)
                    assert rel(gi, deep["ins"][s]) < 1e-5, ("in", s, step, v)
            smr.smr_set_variant(ctx, step, -1, prec, 0)
    finally:
        smr.smr_autotune(ctx, smr.SMR_PREC_FP32)          # leave the tuned variants for later tests
