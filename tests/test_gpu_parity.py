"""GPU FP64 path vs the FP64 oracle, element by element, through the C ABI.

Bar (the product's stated target): relative error <= 1e-10 per product in
FP64; tables and level spectra are compared element-wise at the same bar.
The FP32 path is compared against the same oracle and its error is bounded
by what single precision allows (<= 2e-5 relative per product here)."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from oracle import gmres as ogm
from oracle import mlfma as oml
from oracle import pmchwt as opm
from paper_2407_21724_gb300 import smr, workloads

TOL64 = 1e-10


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def crandn(n, seed):
    rng = np.random.default_rng(seed)
    return (rng.standard_normal(n) + 1j * rng.standard_normal(n)) / math.sqrt(2)


class Case:
    def __init__(self, w, **opts):
        self.w = w
        self.ctx = smr.scene_from_workload(w, **opts)
        self.info = smr.smr_info(self.ctx)
        self.sc = opm.Scene(w["centres"], w["shape_ids"], w["shapes"], eps_in=w["eps_in"],
                            n_theta=opts.get("n_theta", 16), n_phi=opts.get("n_phi", 32))
        rule = "double" if opts.get("level_rule", 0) == 1 else "formula"
        self.M = oml.MLFMA(self.sc, w["pitch"], L0=opts.get("L0", 10), rule=rule)

    def gpu_matvec(self, x, prec=smr.SMR_PREC_FP64):
        xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()
        yd = torch.empty_like(xd)
        smr.smr_matvec(self.ctx, xd, yd, prec, R=xd.numel() // self.info["n_unknowns"])
        torch.cuda.synchronize()
        return yd.cpu().numpy()


@pytest.fixture(scope="module")
def c1():
    c = Case(workloads.make("spheres8x8"))
    yield c
    smr.smr_destroy(c.ctx)


@pytest.fixture(scope="module")
def rnd():
    # 13 x 11 random radii, 8 shapes, 32 modes per current: several boxes per
    # level, odd sizes (ragged tail at every level)
    w = workloads.make("random", n=13, seed=5, modes=16)
    keep = np.ones(len(w["centres"]), dtype=bool)
    keep[[0, 17, 40, 101]] = False           # holes in the lattice
    keep[-13:-2] = False                     # ragged last row
    w["centres"], w["shape_ids"] = w["centres"][keep], w["shape_ids"][keep]
    c = Case(w)
    yield c
    smr.smr_destroy(c.ctx)


def test_tree_matches_oracle(c1, rnd):
    for c in (c1, rnd):
        t = c.M.tree
        assert c.info["n_levels"] == t.n_levels
        for s in range(t.n_levels):
            assert c.info["n_box"][s] == len(t.levels[s]["ij"])
            assert c.info["n_il"][s] == len(t.levels[s]["il"])
            assert c.info["L"][s] == c.M.grids[s].L


def test_patterns(c1, rnd):
    for c in (c1, rnd):
        for s in range(len(c.w["shapes"])):
            P = smr.smr_copy_pattern(c.ctx, s)
            assert rel(P, c.M.patterns[s]) < 1e-13


def test_translation_tables(c1, rnd):
    for c in (c1, rnd):
        for s, tab in enumerate(c.M.T):
            for (dx, dy), T0 in tab.items():
                T = smr.smr_copy_translation(c.ctx, s, dx, dy)
                assert np.max(np.abs(T - T0)) / np.max(np.abs(T0)) < 1e-12


def test_near_blocks(c1, rnd):
    for c in (c1, rnd):
        seen = set()
        for (mu, nu) in c.M.tree.near_pairs():
            sm, sn = c.sc.shape_ids[mu], c.sc.shape_ids[nu]
            d = tuple(int(v) for v in (c.M.tree.ij0[mu] - c.M.tree.ij0[nu]))
            key = (sm, sn) + d
            if key in seen:
                continue
            seen.add(key)
            B = smr.smr_copy_near_block(c.ctx, int(sm), int(sn), *d)
            assert rel(B, c.M.near_block(mu, nu)) < 1e-12, key


def test_level_spectra(c1, rnd):
    for c in (c1, rnd):
        x = crandn(c.info["n_unknowns"], 11)
        c.gpu_matvec(x)
        outs = [c.M.aggregate(x)]
        for s in range(c.M.tree.n_levels - 1):
            outs.append(c.M.upward(s, outs[s]))
        ins = [c.M.translate(s, outs[s]) for s in range(c.M.tree.n_levels)]
        for s in range(c.M.tree.n_levels - 2, -1, -1):
            ins[s] = ins[s] + c.M.downward(s, ins[s + 1])
        for s in range(c.M.tree.n_levels):
            go = smr.smr_copy_level(c.ctx, s, 0)[..., 0]
            gi = smr.smr_copy_level(c.ctx, s, 1)[..., 0]
            assert rel(go, outs[s]) < 1e-12, ("out", s)
            assert rel(gi, ins[s]) < 1e-12, ("in", s)


def test_matvec_fp64(c1, rnd):
    for c in (c1, rnd):
        for x in (crandn(c.info["n_unknowns"], 1), opm.rhs(c.sc, [0, 0, 1], [1, 0, 0])):
            y0 = c.M.matvec(x)
            assert rel(c.gpu_matvec(x), y0) < TOL64


def test_matvec_parts(c1):
    x = crandn(c1.info["n_unknowns"], 2)
    xd = torch.from_numpy(x).cuda()
    yn, yf = torch.empty_like(xd), torch.empty_like(xd)
    smr.smr_matvec_parts(c1.ctx, xd, yn, yf, smr.SMR_PREC_FP64)
    torch.cuda.synchronize()
    assert rel(yn.cpu().numpy(), c1.M.near(x)) < TOL64
    assert rel(yf.cpu().numpy(), c1.M.far(x)) < TOL64


def test_matvec_fp32(c1, rnd):
    for c in (c1, rnd):
        x = crandn(c.info["n_unknowns"], 3)
        err = rel(c.gpu_matvec(x, smr.SMR_PREC_FP32), c.M.matvec(x))
        assert err < 2e-5



def test_tensor_core_receive(c1, rnd):
    """The FP32 product with its receive step on the tensor cores (split TF32)
    matches the CUDA-core FP32 product to FP32 accuracy and the oracle to the
    FP32 bar, on 24- and 32-mode scenes; no pipeline wait ran out."""
    for case, seed in ((c1, 31), (rnd, 32)):
        x = crandn(case.info["n_unknowns"], seed)
        ref = case.M.matvec(x)
        smr.smr_set_tensor_cores(case.ctx, False)
        y0 = case.gpu_matvec(x, smr.SMR_PREC_FP32)
        smr.smr_set_tensor_cores(case.ctx, True)
        y1 = case.gpu_matvec(x, smr.SMR_PREC_FP32)
        smr.smr_sync(case.ctx)
        assert rel(y1, ref) < 2e-5, rel(y1, ref)
        assert rel(y1, y0) < 5e-6, rel(y1, y0)


def test_tensor_core_near(c1, rnd):
    """The FP32 near-field product on the tensor cores (pairs sharing a block
    as one split-TF32 GEMM, one launch per lattice offset) matches the FP64
    near product to the FP32 bar, and the CUDA-core FP32 near product."""
    for case, seed in ((c1, 33), (rnd, 34)):
        n = case.info["n_unknowns"]
        xd = torch.from_numpy(crandn(n, seed)).cuda()
        parts = {}
        for tc, prec in ((True, smr.SMR_PREC_FP32), (False, smr.SMR_PREC_FP32), (True, smr.SMR_PREC_FP64)):
            smr.smr_set_tensor_cores(case.ctx, tc)
            yn, yf = torch.empty_like(xd), torch.empty_like(xd)
            smr.smr_matvec_parts(case.ctx, xd, yn, yf, prec)
            torch.cuda.synchronize()
            parts[(tc, prec)] = yn.cpu().numpy()
        smr.smr_set_tensor_cores(case.ctx, True)
        smr.smr_sync(case.ctx)
        ref = parts[(True, smr.SMR_PREC_FP64)]
        assert rel(parts[(True, smr.SMR_PREC_FP32)], ref) < 2e-6
        assert rel(parts[(False, smr.SMR_PREC_FP32)], ref) < 2e-6
        assert rel(parts[(True, smr.SMR_PREC_FP32)], parts[(False, smr.SMR_PREC_FP32)]) < 2e-6


def test_autotuned_product_matches_oracle(rnd):
    """After smr_autotune picks launch variants, the FP64 and FP32 products
    still meet their bars against the oracle (every variant computes the
    same product)."""
    x = crandn(rnd.info["n_unknowns"], 41)
    ref = rnd.M.matvec(x)
    for prec, bar in ((smr.SMR_PREC_FP64, TOL64), (smr.SMR_PREC_FP32, 2e-5)):
        smr.smr_autotune(rnd.ctx, prec)
        assert rel(rnd.gpu_matvec(x, prec), ref) < bar


def test_sampled_shapes_match_oracle():
    """Shapes given as data (smr_add_shape_sampled): a sphere on a rotated
    16 x 32 rule, one on a rotated 12 x 24 rule (fewer points: padding) and
    a closed-form sphere in one 6 x 5 random lattice.  FP64 product, right-
    hand side and solve against the oracle with the same shape data; FP32
    (tensor cores) at the FP32 bar."""
    from tests.sampled import media, rotated_sphere
    md = media(4.0)
    shapes = [rotated_sphere(0.12, 8, 8, md, seed=1),
              rotated_sphere(0.17, 8, 8, md, n_theta=12, n_phi=24, seed=2), (0.15, 8, 8)]
    rng = np.random.default_rng(12)
    C = workloads.lattice(6, 5)
    w = dict(centres=C, shape_ids=rng.integers(0, 3, size=len(C)).astype(np.int32), shapes=shapes,
             eps_in=4.0, pitch=0.5)
    c = Case(w)
    x = crandn(c.info["n_unknowns"], 13)
    ref = c.M.matvec(x)
    assert rel(c.gpu_matvec(x), ref) < TOL64
    assert rel(c.gpu_matvec(x, smr.SMR_PREC_FP32), ref) < 2e-5
    b = opm.rhs(c.sc, [0, 0, 1], [1, 0, 0])
    bd = torch.empty_like(torch.from_numpy(b)).cuda()
    kh, pol = workloads.incidence(0, 0, "x")
    smr.smr_rhs_plane_waves(c.ctx, [kh], [pol], bd)
    torch.cuda.synchronize()
    assert rel(bd.cpu().numpy(), b) < 1e-12
    xd = torch.zeros_like(bd)
    rc, st = smr.smr_solve(c.ctx, bd, xd, tol=1e-6)
    assert rc == 0
    assert np.linalg.norm(b - c.M.matvec(xd.cpu().numpy())) / np.linalg.norm(b) <= 1.001e-6
    smr.smr_destroy(c.ctx)

@pytest.mark.parametrize("R", [5, 17, 64])
def test_batched_columns_match_single(rnd, R):
    """R right-hand sides in one product: every column equals the single
    product to rounding (the single right-hand-side kernels sum in their own
    order: staged conjugate-shifted parent rows in the anterpolation, tuned
    translation variants), in both precisions, and the FP64 columns match the
    oracle."""
    n = rnd.info["n_unknowns"]
    X = np.stack([crandn(n, 20 + r) for r in range(R)], axis=1)
    for prec, bar in ((smr.SMR_PREC_FP64, 1e-13), (smr.SMR_PREC_FP32, 1e-6)):
        Y = rnd.gpu_matvec(X, prec).reshape(n, R)
        for r in (0, R // 2, R - 1):
            y1 = rnd.gpu_matvec(np.ascontiguousarray(X[:, r]), prec)
            assert rel(Y[:, r], y1) < bar, (prec, r, rel(Y[:, r], y1))
    Y = rnd.gpu_matvec(X).reshape(n, R)
    for r in (1, R - 2):
        assert rel(Y[:, r], rnd.M.matvec(X[:, r])) < TOL64


def test_matvec_host_buffers(c1):
    x = crandn(c1.info["n_unknowns"], 4)
    y = smr.smr_matvec_host(c1.ctx, x)
    assert rel(y, c1.M.matvec(x)) < TOL64


def test_rhs(c1, rnd):
    for c in (c1, rnd):
        for (kh, pol) in workloads.incidence_grid64()[::13]:
            b = torch.empty(c.info["n_unknowns"], dtype=torch.complex128, device="cuda")
            smr.smr_rhs_plane_waves(c.ctx, [kh], [pol], b)
            torch.cuda.synchronize()
            assert rel(b.cpu().numpy(), opm.rhs(c.sc, kh, pol)) < 1e-13


def test_precond(c1):
    x = crandn(c1.info["n_unknowns"], 6)
    xd = torch.from_numpy(x).cuda()
    zd = torch.empty_like(xd)
    smr.smr_precond(c1.ctx, xd, zd)
    torch.cuda.synchronize()
    z0 = ogm.block_diag_precond(c1.sc)(x)
    assert rel(zd.cpu().numpy(), z0) < 1e-12


def test_single_particle_and_line():
    """Degenerate scenes: one particle (tensor-core tiles of one column, no
    interaction lists) and a 7-particle line; 8 + 8 and odd 5 + 4 modes (the
    odd count takes the CUDA-core aggregation).  FP64 at the parity bar,
    FP32 (tensor cores on and off) at the FP32 bar."""
    for C in ([[0.0, 0.0, 0.0]], [[0.5 * i, 0.0, 0.0] for i in range(7)]):
        for modes in ((8, 8), (5, 4)):
            w = dict(centres=np.array(C), shape_ids=np.zeros(len(C), dtype=np.int32),
                     shapes=[(0.15,) + modes], eps_in=4.0, pitch=0.5)
            c = Case(w)
            x = crandn(c.info["n_unknowns"], 8)
            ref = c.M.matvec(x)
            assert rel(c.gpu_matvec(x), ref) < TOL64
            for tc in (True, False):
                smr.smr_set_tensor_cores(c.ctx, tc)
                assert rel(c.gpu_matvec(x, smr.SMR_PREC_FP32), ref) < 2e-5, (len(C), modes, tc)
            smr.smr_sync(c.ctx)
            smr.smr_destroy(c.ctx)


def test_solve_fp64_and_mixed(c1):
    b = opm.rhs(c1.sc, [0, 0, 1], [1, 0, 0])
    bd = torch.from_numpy(b).cuda()
    for prec in (smr.SMR_PREC_FP64, smr.SMR_PREC_FP32):
        xd = torch.zeros_like(bd)
        rc, st = smr.smr_solve(c1.ctx, bd, xd, tol=1e-4, precision=prec)
        assert rc == 0
        x = xd.cpu().numpy()
        # the true residual of the FP64 oracle operator meets the tolerance
        r = np.linalg.norm(b - c1.M.matvec(x)) / np.linalg.norm(b)
        assert r <= 1.001e-4, (prec, r, st)
    # same iterations as the oracle GMRES on the same operator (within 1)
    x0, info = ogm.gmres(c1.M.matvec, b, precond=ogm.block_diag_precond(c1.sc), tol=1e-4)
    xd = torch.zeros_like(bd)
    rc, st = smr.smr_solve(c1.ctx, bd, xd, tol=1e-4, precision=smr.SMR_PREC_FP64)
    assert abs(st["iters"] - info["iters"]) <= 1


@pytest.mark.parametrize("prec", [smr.SMR_PREC_FP64, smr.SMR_PREC_FP32])
def test_solve_batched_columns(rnd, prec):
    """Three systems in lockstep ([N][R], R = 3): every column meets the
    tolerance on the oracle operator, and the lockstep run takes about as
    many Arnoldi steps as the slowest column solved alone."""
    n = rnd.info["n_unknowns"]
    incs = [workloads.incidence(0, 0, "x"), workloads.incidence(20, 45, "y"),
            workloads.incidence(35, 180, "x")]
    B = np.stack([opm.rhs(rnd.sc, k, e) for k, e in incs], axis=1)
    bd = torch.from_numpy(np.ascontiguousarray(B).reshape(-1)).cuda()
    xd = torch.zeros_like(bd)
    rc, st = smr.smr_solve(rnd.ctx, bd, xd, R=3, tol=1e-4, precision=prec)
    assert rc == 0, st
    X = xd.cpu().numpy().reshape(n, 3)
    singles = []
    for r in range(3):
        res = np.linalg.norm(B[:, r] - rnd.M.matvec(X[:, r])) / np.linalg.norm(B[:, r])
        assert res <= 1.001e-4, (r, res, st)
        b1 = torch.from_numpy(np.ascontiguousarray(B[:, r])).cuda()
        x1 = torch.zeros_like(b1)
        rc1, st1 = smr.smr_solve(rnd.ctx, b1, x1, tol=1e-4, precision=prec)
        assert rc1 == 0
        singles.append(st1["iters"])
    assert max(singles) - 2 <= st["iters"] <= max(singles) + 3, (singles, st)


@pytest.mark.parametrize("prec", [smr.SMR_PREC_FP64, smr.SMR_PREC_FP32])
def test_solve_restarted(rnd, prec):
    """Restarted GMRES (Krylov dimension 8) still reaches a tight tolerance
    on the oracle operator."""
    b = opm.rhs(rnd.sc, *workloads.incidence(10, 30, "x"))
    bd = torch.from_numpy(b).cuda()
    xd = torch.zeros_like(bd)
    rc, st = smr.smr_solve(rnd.ctx, bd, xd, tol=1e-5, restart=8, precision=prec)
    assert rc == 0, st
    res = np.linalg.norm(b - rnd.M.matvec(xd.cpu().numpy())) / np.linalg.norm(b)
    assert res <= 1.001e-5, (res, st)


def test_solve_rejects_nan_initial_guess(c1):
    """A NaN initial guess ends the solve with SMR_E_NAN (raised by the
    binding), in both precisions; it never reports convergence."""
    b = torch.from_numpy(opm.rhs(c1.sc, [0, 0, 1], [1, 0, 0])).cuda()
    for prec in (smr.SMR_PREC_FP64, smr.SMR_PREC_FP32):
        x = torch.full_like(b, float("nan"))
        with pytest.raises(smr.SmrError):
            smr.smr_solve(c1.ctx, b, x, tol=1e-4, precision=prec, use_x0=1)


def test_far_field_and_cross_sections(c1):
    b = opm.rhs(c1.sc, [0, 0, 1], [1, 0, 0])
    x, _ = ogm.gmres(c1.M.matvec, b, precond=ogm.block_diag_precond(c1.sc), tol=1e-8)
    rng = np.random.default_rng(9)
    d = rng.standard_normal((40, 3))
    d /= np.linalg.norm(d, axis=1)[:, None]
    xd = torch.from_numpy(x).cuda()
    F = torch.empty(40 * 3, dtype=torch.complex128, device="cuda")
    smr.smr_far_field(c1.ctx, xd, d, F)
    torch.cuda.synchronize()
    assert rel(F.cpu().numpy().reshape(40, 3), opm.far_field(c1.sc, x, d)) < 1e-12
    # Two columns: the converged scattering solution, and an arbitrary
    # coefficient vector with its own (unnormalised) direction and complex
    # polarisation, so both sums and the per-column forward direction count.
    y = crandn(c1.info["n_unknowns"], 12) * 0.3
    X = torch.from_numpy(np.ascontiguousarray(np.stack([x, y], axis=1))).cuda()
    khat = np.array([[0.0, 0.0, 1.0], [1.0, -2.0, 0.5]])
    pol = np.array([[1.0, 0, 0], [0.3 + 0.2j, 0.1j, -0.4]])
    for nt in (1, 9, 24):
        cs, ce = smr.smr_cross_sections(c1.ctx, X, khat, pol, n_theta=nt)
        for r, v in enumerate((x, y)):
            ws = opm.scattering_cross_section(c1.sc, v, nt)
            we = opm.extinction_cross_section(c1.sc, v, khat[r], pol[r])
            assert abs(cs[r] - ws) <= 1e-12 * abs(ws), (nt, r, cs[r], ws)
            assert abs(ce[r] - we) <= 1e-12 * max(abs(we), abs(ws)), (nt, r, ce[r], we)
    # Lossless particles at convergence: extinction equals scattering once
    # 24 x 48 directions resolve |F|^2.
    assert abs(cs[0] - ce[0]) < 1e-4 * cs[0]
    with pytest.raises(smr.SmrError):
        smr.smr_cross_sections(c1.ctx, X, khat, np.zeros((2, 3)), n_theta=8)
    with pytest.raises(smr.SmrError):
        smr.smr_cross_sections(c1.ctx, X, khat, pol, n_theta=0)


def test_near_field(c1):
    b = opm.rhs(c1.sc, [0, 0, 1], [1, 0, 0])
    x = crandn(c1.info["n_unknowns"], 10) + b
    pts = np.array([[0.0, 0.0, 2.0], [0.3, -0.2, 5.0], [3.0, 1.0, 0.4], [0.1, 0.1, 0.6]])
    xd = torch.from_numpy(x).cuda()
    EH = torch.empty(4 * 6, dtype=torch.complex128, device="cuda")
    smr.smr_near_field(c1.ctx, xd, pts, EH)
    torch.cuda.synchronize()
    E0, H0 = opm.near_field(c1.sc, x, pts)
    g = EH.cpu().numpy().reshape(4, 6)
    assert rel(g[:, :3], E0) < 1e-12 and rel(g[:, 3:], H0) < 1e-12


def test_invalid_arguments(c1):
    with pytest.raises(smr.SmrError):
        smr.smr_matvec(c1.ctx, 0, 0, R=1)
    ctx = smr.smr_create()
    with pytest.raises(smr.SmrError):
        smr.smr_set_scene(ctx, [[0, 0, 0]], [0], 4.0)      # no shapes
    smr.smr_add_sphere(ctx, 0.15, 4, 4)
    with pytest.raises(smr.SmrError):
        smr.smr_set_scene(ctx, [[0, 0, 0], [0.01, 0, 0]], [0, 0], 4.0)   # same cell
    with pytest.raises(smr.SmrError):
        smr.smr_set_scene(ctx, [[0, 0, 0]], [0], 4.0 + 0.1j)             # lossy
    xd = torch.zeros(16, dtype=torch.complex128, device="cuda")
    with pytest.raises(smr.SmrError):
        smr.smr_matvec(ctx, xd, xd, R=1)                   # no scene
    smr.smr_destroy(ctx)


def _oracle_cluster_apply(c, r):
    """The cluster block-Jacobi preconditioner from the oracle's blocks: 2 x 2
    clusters of lattice cells counted from the array's lower corner, each
    cluster's near matrix (self blocks and the blocks between its members)
    solved against its rows of r."""
    C = np.asarray(c.w["centres"])
    pitch = c.w["pitch"]
    ix = np.round((C[:, 0] - C[:, 0].min()) / pitch).astype(int)
    iy = np.round((C[:, 1] - C[:, 1].min()) / pitch).astype(int)
    m = 2 * c.sc.n_psi
    out = np.zeros_like(r)
    groups = {}
    for p in range(len(C)):
        groups.setdefault((ix[p] // 2, iy[p] // 2), []).append(p)
    for mem in groups.values():
        A = np.zeros((m * len(mem), m * len(mem)), dtype=complex)
        for a, pa in enumerate(mem):
            for b, pb in enumerate(mem):
                sa, sb = c.sc.shape_ids[pa], c.sc.shape_ids[pb]
                blk = (c.sc.self_block(sa) if pa == pb else
                       opm.exterior_block(c.sc, sa, C[pa] - C[pb], sb, np.zeros(3)))
                A[a * m:(a + 1) * m, b * m:(b + 1) * m] = blk
        rows = np.concatenate([np.arange(p * m, (p + 1) * m) for p in mem])
        out[rows] = np.linalg.solve(A, r[rows])
    return out


def test_cluster_preconditioner(rnd):
    """SMR_PRECOND_CLUSTER: the GPU's FP64 cluster inverses applied to r equal
    the oracle's cluster solves (holes and the ragged row leave partial
    clusters), FP32 within the FP32 bar; solves with it meet the tolerance on
    the oracle's operator in fewer iterations than block-diagonal GMRES."""
    n = rnd.info["n_unknowns"]
    r = crandn(n, 41)
    ref = _oracle_cluster_apply(rnd, r)
    rd = torch.from_numpy(r).cuda()
    zd = torch.empty_like(rd)
    smr.smr_precond_cluster(rnd.ctx, rd, zd, smr.SMR_PREC_FP64)
    torch.cuda.synchronize()
    assert rel(zd.cpu().numpy(), ref) < 1e-10
    smr.smr_precond_cluster(rnd.ctx, rd, zd, smr.SMR_PREC_FP32)
    torch.cuda.synchronize()
    assert rel(zd.cpu().numpy(), ref) < 1e-5
    b = opm.rhs(rnd.sc, [0, 0, 1.0], [1.0, 0, 0])
    bd = torch.from_numpy(b).cuda()
    its = {}
    for prec in (smr.SMR_PREC_FP64, smr.SMR_PREC_FP32):
        for pc in (smr.SMR_PRECOND_BLOCKDIAG, smr.SMR_PRECOND_CLUSTER):
            x = torch.zeros_like(bd)
            rc, st = smr.smr_solve(rnd.ctx, bd, x, tol=1e-6, maxit=500, precision=prec, precond=pc)
            assert rc == 0
            assert np.linalg.norm(b - rnd.M.matvec(x.cpu().numpy())) <= 1.001e-6 * np.linalg.norm(b)
            its[(prec, pc)] = st["iters"]
    assert its[(smr.SMR_PREC_FP64, smr.SMR_PRECOND_CLUSTER)] < its[(smr.SMR_PREC_FP64, smr.SMR_PRECOND_BLOCKDIAG)]


def test_polynomial_preconditioner(rnd):
    """poly_degree d: iterations on B p(B), p the GMRES residual polynomial's
    roots (harmonic Ritz values of d Arnoldi steps) in Leja order.  Solves in
    both precisions meet the tolerance on the oracle's operator, with fewer
    iterations than without the polynomial; a degree out of range is
    refused."""
    b = opm.rhs(rnd.sc, [0, 0, 1.0], [1.0, 0, 0])
    bd = torch.from_numpy(b).cuda()
    for prec in (smr.SMR_PREC_FP64, smr.SMR_PREC_FP32):
        x = torch.zeros_like(bd)
        rc, st0 = smr.smr_solve(rnd.ctx, bd, x, tol=1e-6, maxit=500, precision=prec)
        assert rc == 0
        for deg in (3, 6):
            x = torch.zeros_like(bd)
            rc, st = smr.smr_solve(rnd.ctx, bd, x, tol=1e-6, maxit=500, precision=prec, poly_degree=deg)
            assert rc == 0, (prec, deg)
            assert np.linalg.norm(b - rnd.M.matvec(x.cpu().numpy())) <= 1.001e-6 * np.linalg.norm(b)
            # the polynomial's own Arnoldi steps are counted in iters
            assert st["iters"] - deg < st0["iters"], (prec, deg, st["iters"], st0["iters"])
    with pytest.raises(smr.SmrError):
        smr.smr_solve(rnd.ctx, bd, torch.zeros_like(bd), poly_degree=1)


def test_overlap_is_bit_identical(rnd):
    """The overlapped product (near product and translations on side
    streams, ordered by events) gives bit for bit the ordered product, in
    both precisions, directly and through graphs, for one column and for
    several (column lanes)."""
    n = rnd.info["n_unknowns"]
    try:
        for R in (1, 5):
            x = np.stack([crandn(n, 60 + r) for r in range(R)], axis=1).reshape(-1)
            xd = torch.from_numpy(x).cuda()
            ref, y = torch.empty_like(xd), torch.empty_like(xd)
            for prec in (smr.SMR_PREC_FP64, smr.SMR_PREC_FP32):
                smr.smr_set_overlap(rnd.ctx, 0)
                smr.smr_matvec(rnd.ctx, xd, ref, prec, R=R)
                torch.cuda.synchronize()
                smr.smr_set_overlap(rnd.ctx, 1)
                for graph in (False, True, True):
                    y.fill_(float("nan"))
                    (smr.smr_matvec_graph if graph else smr.smr_matvec)(rnd.ctx, xd, y, prec, R=R)
                    torch.cuda.synchronize()
                    assert torch.equal(y, ref), (R, prec, graph)
    finally:
        smr.smr_set_overlap(rnd.ctx, 1)


def test_column_lanes_are_bit_identical(rnd):
    """FP32 products with R > 1 deal their columns to lanes with their own
    buffers and streams: any lane count gives bit for bit the product of one
    lane (the same kernels on the same data), directly and through a graph,
    and the lane count is checked."""
    n = rnd.info["n_unknowns"]
    R = 7
    x = np.stack([crandn(n, 90 + r) for r in range(R)], axis=1).reshape(-1)
    xd = torch.from_numpy(x).cuda()
    ref, y = torch.empty_like(xd), torch.empty_like(xd)
    try:
        smr.smr_set_column_lanes(rnd.ctx, 1)
        smr.smr_matvec(rnd.ctx, xd, ref, smr.SMR_PREC_FP32, R=R)
        torch.cuda.synchronize()
        for nl in (2, 3, 4, 16):
            smr.smr_set_column_lanes(rnd.ctx, nl)
            for graph in (False, True):
                for _ in range(2):
                    y.fill_(float("nan"))
                    f = smr.smr_matvec_graph if graph else smr.smr_matvec
                    f(rnd.ctx, xd, y, smr.SMR_PREC_FP32, R=R)
                    torch.cuda.synchronize()
                    assert torch.equal(y, ref), (nl, graph)
        for bad in (0, 17):
            with pytest.raises(smr.SmrError):
                smr.smr_set_column_lanes(rnd.ctx, bad)
    finally:
        smr.smr_set_column_lanes(rnd.ctx, 4)


def test_graph_product_matches_direct(c1, rnd):
    """The CUDA-graph replay launches the same kernels: bit-identical to
    smr_matvec, also on repeated replays and after a change of R."""
    for c in (c1, rnd):
        n = c.info["n_unknowns"]
        for R in (1, 3):
            x = np.stack([crandn(n, 70 + r) for r in range(R)], axis=1).reshape(-1)
            xd = torch.from_numpy(x).cuda()
            y0, y1 = torch.empty_like(xd), torch.empty_like(xd)
            for prec in (smr.SMR_PREC_FP64, smr.SMR_PREC_FP32):
                smr.smr_matvec(c.ctx, xd, y0, prec, R=R)
                for _ in range(3):
                    y1.zero_()
                    smr.smr_matvec_graph(c.ctx, xd, y1, prec, R=R)
                torch.cuda.synchronize()
                assert torch.equal(y0, y1)
