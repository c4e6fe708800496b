"""Parity at full size: the 200 x 200 metalens (40,000 pillars, 32 modes per
current, 2,560,000 unknowns) and the 100 x 100 random array with 64
right-hand sides, set up and launched the way the benchmark times them
(autotuned launch variants, tensor cores on, CUDA-graph products).

The oracle cannot run an MLFMA product this large, so the checks are either
outputs it computes one at a time (near-field rows of sampled particles from
their own blocks, far-field amplitudes at sampled directions, right-hand
side entries of sampled particles) or properties that hold at any size:
the Galerkin reciprocity u^T A v = (D v)^T A (D u), D = diag(I, -I) per
particle, which the MLFMA keeps to rounding (weighted-adjoint anterpolation,
mirrored receive patterns); FP32 against FP64 products; batched columns
against single products; and the solver's answer against an independent
FP64 residual."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle import mlfma as oml
from oracle import pmchwt as opm
from paper_2407_21724_gb300 import smr, workloads


def crandn(n, seed):
    rng = np.random.default_rng(seed)
    return (rng.standard_normal(n) + 1j * rng.standard_normal(n)) / math.sqrt(2)


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def dsign(p, n_psi, R=1):
    """D = diag(I, -I) per particle (electric +, magnetic -), R columns."""
    d = np.ones((p, 2, n_psi, R))
    d[:, 1] = -1
    return torch.from_numpy(d.reshape(-1)).cuda()


class Full:
    def __init__(self, name, kw, autotune=True):
        self.w = workloads.make(name, **kw)
        self.ctx = smr.scene_from_workload(self.w)
        if autotune:
            smr.smr_autotune(self.ctx, smr.SMR_PREC_FP32)
        self.info = smr.smr_info(self.ctx)
        self.n = self.info["n_unknowns"]
        self.p = len(self.w["centres"])
        self.n_psi = self.info["n_psi"]
        self.sc = opm.Scene(self.w["centres"], self.w["shape_ids"], self.w["shapes"],
                            eps_in=self.w["eps_in"])

    def product(self, x, prec, R=1, graph=False):
        y = torch.empty_like(x)
        (smr.smr_matvec_graph if graph else smr.smr_matvec)(self.ctx, x, y, prec, R=R)
        torch.cuda.synchronize()
        return y


@pytest.fixture(scope="module")
def lens():
    c = Full("metalens", dict(n=200, focal=50.0))
    yield c
    smr.smr_destroy(c.ctx)


# particles at the four corners, on two edges, at the centre and inside
SAMPLED = (0, 199, 39800, 39999, 100, 20000, 20100, 12345, 31007)


def test_lens_near_rows_match_oracle_blocks(lens):
    """Near-field rows of sampled particles (self block plus the 8 lattice
    neighbours, Eq. 16) against the oracle's blocks, FP64, at full size."""
    x = crandn(lens.n, 101)
    xd = torch.from_numpy(x).cuda()
    yn, yf = torch.empty_like(xd), torch.empty_like(xd)
    smr.smr_matvec_parts(lens.ctx, xd, yn, yf, smr.SMR_PREC_FP64)
    torch.cuda.synchronize()
    yn = yn.cpu().numpy().reshape(lens.p, -1)
    sc = lens.sc
    ij = oml.Tree(sc.centres, lens.w["pitch"]).ij0
    xx = x.reshape(lens.p, -1)
    blocks = {}
    for mu in SAMPLED:
        want = np.zeros(xx.shape[1], dtype=complex)
        for nu in np.nonzero(np.max(np.abs(ij - ij[mu]), axis=1) <= 1)[0]:
            sm, sn = sc.shape_ids[mu], sc.shape_ids[nu]
            key = ("self", sm) if mu == nu else (sm, sn, tuple(ij[mu] - ij[nu]))
            if key not in blocks:
                blocks[key] = sc.self_block(sm) if mu == nu else \
                    opm.exterior_block(sc, sm, sc.centres[mu] - sc.centres[nu], sn, np.zeros(3))
            want += blocks[key] @ xx[nu]
        assert rel(yn[mu], want) < 1e-12, (mu, rel(yn[mu], want))


def test_lens_fp64_product_is_reciprocal(lens):
    """u^T A v = (D v)^T A (D u) for the whole FP64 product at full size: a
    wrong sign, index, shift or weight at any level of the tree breaks it."""
    u = torch.from_numpy(crandn(lens.n, 102)).cuda()
    v = torch.from_numpy(crandn(lens.n, 103)).cuda()
    D = dsign(lens.p, lens.n_psi)
    a = torch.sum(u * lens.product(v, smr.SMR_PREC_FP64)).item()
    b = torch.sum(D * v * lens.product(D * u, smr.SMR_PREC_FP64)).item()
    assert abs(a - b) / abs(a) < 1e-11, abs(a - b) / abs(a)


def test_lens_tuned_fp32_product_matches_fp64(lens):
    """The benchmark's product (autotuned FP32, tensor-core aggregation and
    receive, graph launch) against the FP64 product: the FP32 bar."""
    x = torch.from_numpy(crandn(lens.n, 104)).cuda()
    y64 = lens.product(x, smr.SMR_PREC_FP64)
    y32 = lens.product(x, smr.SMR_PREC_FP32, graph=True)
    smr.smr_sync(lens.ctx)
    e = (torch.linalg.norm(y32 - y64) / torch.linalg.norm(y64)).item()
    assert e < 2e-5, e
    # graph and kernel-by-kernel launches compute the same FP32 product
    y32d = lens.product(x, smr.SMR_PREC_FP32)
    assert torch.equal(y32, y32d)


def test_lens_far_field_matches_oracle(lens):
    """Far-field amplitudes at sampled directions against the oracle's
    radiation integrals over all 40,000 particles."""
    x = crandn(lens.n, 105)
    rng = np.random.default_rng(106)
    d = rng.standard_normal((4, 3))
    d[0] = (0, 0, 1)
    d /= np.linalg.norm(d, axis=1)[:, None]
    F = torch.empty(4 * 3, dtype=torch.complex128, device="cuda")
    smr.smr_far_field(lens.ctx, torch.from_numpy(x).cuda(), d, F)
    torch.cuda.synchronize()
    assert rel(F.cpu().numpy().reshape(4, 3), opm.far_field(lens.sc, x, d)) < 1e-11


def test_lens_rhs_matches_oracle_on_sampled_particles(lens):
    """Plane-wave right-hand side entries of sampled particles (Eqs. 18-19)
    at full size: each particle's entries depend on its own shape and
    centre only, so the oracle evaluates them on those particles alone."""
    khat, pol = lens.w["incidences"][0]
    b = torch.empty(lens.n, dtype=torch.complex128, device="cuda")
    smr.smr_rhs_plane_waves_arrays(lens.ctx, [khat], [pol], b)
    torch.cuda.synchronize()
    idx = np.array(SAMPLED)
    sub = opm.Scene(lens.w["centres"][idx], lens.w["shape_ids"][idx], lens.w["shapes"],
                    eps_in=lens.w["eps_in"])
    want = opm.rhs(sub, khat, pol).reshape(len(idx), -1)
    got = b.cpu().numpy().reshape(lens.p, -1)[idx]
    assert rel(got, want) < 1e-12


def test_lens_mixed_solve_meets_tolerance_by_independent_residual(lens):
    """The benchmark's solve (FP32 inner products, FP64 outer residual,
    block-diagonal preconditioner, tol 1e-4), checked by a separate FP64
    product: ||b - A x|| / ||b|| <= 1e-4."""
    khat, pol = lens.w["incidences"][0]
    b = torch.empty(lens.n, dtype=torch.complex128, device="cuda")
    smr.smr_rhs_plane_waves_arrays(lens.ctx, [khat], [pol], b)
    x = torch.zeros_like(b)
    rc, st = smr.smr_solve(lens.ctx, b, x, tol=1e-4, precision=smr.SMR_PREC_FP32, maxit=3000)
    assert rc == smr.SMR_OK, rc
    r = b - lens.product(x, smr.SMR_PREC_FP64)
    res = (torch.linalg.norm(r) / torch.linalg.norm(b)).item()
    assert res <= 1e-4, res
    assert abs(res - st["resid_true"]) <= 1e-3 * res


@pytest.fixture(scope="module")
def batched():
    c = Full("random", dict(n=100, seed=21725), autotune=False)
    yield c
    smr.smr_destroy(c.ctx)


def test_batched64_columns_match_single_products(batched):
    """64 right-hand sides in one product (the batched configuration) at full
    size: FP64 columns equal single-column FP64 products to rounding, FP32
    columns meet the FP32 bar, and the batched FP64 product is reciprocal
    column by column."""
    R = 64
    c = batched
    X = torch.from_numpy(crandn(c.n * R, 107)).cuda()
    Y64 = c.product(X, smr.SMR_PREC_FP64, R=R).view(c.n, R)
    Y32 = c.product(X, smr.SMR_PREC_FP32, R=R).view(c.n, R)
    Xv = X.view(c.n, R)
    for r in (0, 17, 63):
        y1 = c.product(Xv[:, r].contiguous(), smr.SMR_PREC_FP64)
        e = (torch.linalg.norm(Y64[:, r] - y1) / torch.linalg.norm(y1)).item()
        assert e < 1e-13, (r, e)
    e32 = (torch.linalg.norm(Y32 - Y64, dim=0) / torch.linalg.norm(Y64, dim=0)).max().item()
    assert e32 < 2e-5, e32
    D = dsign(c.p, c.n_psi, R).view(c.n, R)
    U = torch.from_numpy(crandn(c.n * R, 108)).cuda().view(c.n, R)
    a = torch.sum(U * Y64, dim=0)
    b = torch.sum(D * Xv * c.product((D * U).contiguous().view(-1), smr.SMR_PREC_FP64, R=R).view(c.n, R), dim=0)
    gap = (torch.abs(a - b) / torch.abs(a)).max().item()
    assert gap < 1e-11, gap


def _oracle_box_out(w, level, bx, by, x):
    """Outgoing spectrum (K_level, 4) of the lens box (bx, by) at `level`,
    from the oracle run on that box's particles alone.  One anchor particle
    two boxes to the right of it (a box of its own, zero coefficients) lets
    the sub-scene's tree reach `level`; the box's lower-left site is the
    sub-scene's origin, so its boxes and centres coincide with the lens's."""
    pitch = w["pitch"]
    C = w["centres"]
    lo = C[:, :2].min(axis=0)
    ij = np.rint((C[:, :2] - lo) / pitch).astype(int)
    sel = np.nonzero(((ij[:, 0] >> level) == bx) & ((ij[:, 1] >> level) == by))[0]
    assert len(sel) == 4 ** level                       # a full box of the lens
    corner = lo + np.array([bx, by]) * (2 ** level) * pitch
    anchor = np.array([[corner[0] + 2 * (2 ** level) * pitch, corner[1], C[0, 2]]])
    sc = opm.Scene(np.vstack([C[sel], anchor]), np.concatenate([w["shape_ids"][sel], [0]]),
                   w["shapes"], eps_in=w["eps_in"])
    M = oml.MLFMA(sc, pitch)
    assert M.tree.n_levels == level + 1 and M.tree.levels[level]["index"][(0, 0)] == 0
    n2 = 2 * sc.n_psi
    xs = np.concatenate([x.reshape(-1, n2)[sel], np.zeros((1, n2))]).reshape(-1)
    out = M.aggregate(xs)
    for s in range(level):
        out = M.upward(s, out)
    return out[0]


def test_lens_upper_level_spectra_match_oracle_subtrees(lens):
    """Level-4, 5 and 6 outgoing spectra (L = 87, 162, 309) of sampled lens
    boxes after the autotuned FP64 product, element-wise against the oracle's
    aggregation and interpolation over each box's subtree (256, 1,024 and
    4,096 particles): <= 1e-12."""
    x = crandn(lens.n, 104)
    lens.product(torch.from_numpy(x).cuda(), smr.SMR_PREC_FP64)
    for level, bx, by in ((4, 5, 7), (5, 2, 3), (6, 1, 2)):
        nbx = ((200 - 1) >> level) + 1
        got = smr.smr_copy_level(lens.ctx, level, 0)[by * nbx + bx, :, :, 0]
        want = _oracle_box_out(lens.w, level, bx, by, x)
        assert rel(got, want) < 1e-12, (level, rel(got, want))
