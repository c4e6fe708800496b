"""Particles off the lattice on the GPU against the FP64 oracle: a jittered
lattice of random-radius spheres, a sparse golden-angle spiral, jittered
meshed cylinders, and scenes with several particles per finest cell (the
paper's dense spiral spacing, a two-layer Moire lattice).  Displaced centres
keep their shift to the finest-group centre in aggregation and receive,
their exterior near blocks are computed for the exact offsets, and a cell's
particles sum into one box spectrum (Sec. V, non-lattice and 2.5D arrays).

Bars as for the lattice: <= 1e-10 relative per FP64 product, <= 2e-5 per
FP32 product, near blocks to 1e-12, solutions to their tolerance in the
oracle's true residual."""
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


def crandn(n, seed):
    rng = np.random.default_rng(seed)
    return (rng.standard_normal(n) + 1j * rng.standard_normal(n)) / math.sqrt(2)


class Case:
    def __init__(self, w):
        self.w = w
        self.ctx = smr.scene_from_workload(w)
        self.info = smr.smr_info(self.ctx)
        self.sc = opm.Scene(w["centres"], w["shape_ids"], w["shapes"], eps_in=w["eps_in"])
        self.M = oml.MLFMA(self.sc, w["pitch"], L0=w.get("L0", 10))

    def gpu_matvec(self, x, prec=smr.SMR_PREC_FP64):
        xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()
        yd = torch.empty_like(xd)
        smr.smr_matvec(self.ctx, xd, yd, prec)
        torch.cuda.synchronize()
        return yd.cpu().numpy()


@pytest.fixture(scope="module")
def jit():
    # 11 x 9 random radii, centres moved by up to 0.03 per axis, holes
    w = workloads.make("jittered", n=11, seed=9, modes=8, jitter=0.03)
    keep = np.ones(len(w["centres"]), dtype=bool)
    keep[[3, 30, 57]] = False
    keep[-11:-4] = False
    w["centres"], w["shape_ids"] = w["centres"][keep], w["shape_ids"][keep]
    c = Case(w)
    yield c
    smr.smr_destroy(c.ctx)


@pytest.fixture(scope="module")
def spiral():
    c = Case(workloads.make("spiral", n=160, modes=8))
    yield c
    smr.smr_destroy(c.ctx)


def test_tree_and_blocks(jit, spiral):
    for c in (jit, spiral):
        t = c.M.tree
        assert c.info["n_levels"] == t.n_levels
        for s in range(t.n_levels):
            assert c.info["n_box"][s] == len(t.levels[s]["ij"])
            assert c.info["n_il"][s] == len(t.levels[s]["il"])
        # one exterior block per displaced ordered pair (all offsets differ)
        n_ext = len([1 for (mu, nu) in t.near_pairs() if mu != nu])
        assert c.info["n_near_blocks"] == len(c.w["shapes"]) + n_ext


def test_pair_blocks_match_oracle(jit, spiral):
    for c in (jit, spiral):
        pairs = c.M.tree.near_pairs()
        rng = np.random.default_rng(1)
        for k in rng.choice(len(pairs), size=min(12, len(pairs)), replace=False):
            mu, nu = pairs[k]
            B = smr.smr_copy_pair_block(c.ctx, int(mu), int(nu))
            assert rel(B, c.M.near_block(mu, nu)) < 1e-12, (mu, nu)
    with pytest.raises(smr.SmrError):
        smr.smr_copy_pair_block(jit.ctx, 0, jit.sc.p - 1)


@pytest.mark.parametrize("which", ["jit", "spiral"])
def test_product_matches_oracle(jit, spiral, which):
    c = jit if which == "jit" else spiral
    x = crandn(c.info["n_unknowns"], 3)
    ref = c.M.matvec(x)
    assert rel(c.gpu_matvec(x), ref) < 1e-10
    assert rel(c.gpu_matvec(x, smr.SMR_PREC_FP32), ref) < 2e-5


def test_solved_far_field_matches_oracle(spiral):
    """Plane-wave scattering by the spiral: the GPU GMRES solution (FP64, and
    mixed precision) reaches its tolerance in the oracle's own true residual,
    and its far field equals the oracle's far field of the same solution."""
    c = spiral
    kh, pol = workloads.incidence(10, 40, "y")
    n = c.info["n_unknowns"]
    b = torch.empty(n, dtype=torch.complex128, device="cuda")
    smr.smr_rhs_plane_waves(c.ctx, [kh], [pol], b)
    torch.cuda.synchronize()
    bo = opm.rhs(c.sc, kh, pol)
    assert rel(b.cpu().numpy(), bo) < 1e-12
    dirs = np.array([[0, 0, 1.0], [0, 0, -1.0], [0.6, 0, 0.8], [0, 0.8, -0.6], [1.0, 0, 0]])
    for prec, tol in ((smr.SMR_PREC_FP64, 1e-10), (smr.SMR_PREC_FP32, 1e-6)):
        x = torch.zeros_like(b)
        rc, st = smr.smr_solve(c.ctx, b, x, tol=tol, maxit=400, precision=prec)
        assert rc == 0
        xh = x.cpu().numpy()
        assert np.linalg.norm(bo - c.M.matvec(xh)) / np.linalg.norm(bo) <= 1.01 * tol
        Fd = torch.empty(len(dirs) * 3, dtype=torch.complex128, device="cuda")
        smr.smr_far_field(c.ctx, x, dirs, Fd)
        torch.cuda.synchronize()
        assert rel(Fd.cpu().numpy().reshape(len(dirs), 3), opm.far_field(c.sc, xh, dirs)) < 1e-12


def test_jittered_meshed_cylinders():
    """4 x 3 jittered lattice of two meshed cylinders: the product lifted to
    RWG coefficients (the two sides' mode bases differ inside clusters of
    equal eigenvalues) matches the oracle."""
    from oracle import mesh as om
    NP = 6
    cyl = [(0.12, 0.6, 8, 3, 2), (0.18, 0.6, 8, 3, 2)]
    C = workloads.lattice(4, 3)
    C[:, :2] += np.random.default_rng(4).uniform(-0.04, 0.04, size=(len(C), 2))
    ids = np.array([0, 1, 1, 0, 1, 0, 0, 1, 0, 1, 1, 0], dtype=np.int32)
    ctx = smr.smr_create(pitch=workloads.PITCH)
    mms = []
    for args in cyl:
        V, T = workloads.cylinder_mesh(*args)
        smr.smr_add_shape_mesh(ctx, V, T, NP, NP)
        mms.append(om.MeshModes(om.Mesh(V, T), NP, NP))
    smr.smr_set_scene(ctx, C, ids, 4.0)
    outer, inner = opm.Medium(1.0), opm.Medium(4.0)
    sc = opm.Scene(C, ids, [mm.sampled(outer, inner) for mm in mms], eps_in=4.0)
    Ms = [smr.smr_shape_modes(ctx, s)[0] for s in range(2)]
    Mo = [mm.M for mm in mms]
    rng = np.random.default_rng(7)
    xg, xo = [], []
    for s in ids:
        cc = rng.standard_normal((2, Ms[s].shape[1])) + 1j * rng.standard_normal((2, Ms[s].shape[1]))
        xg.append((Ms[s] @ cc.T).T.ravel())
        xo.append((Mo[s] @ cc.T).T.ravel())
    xg, xo = np.concatenate(xg), np.concatenate(xo)

    n = 2 * NP

    def lifted(y, M):
        yy = y.reshape(len(ids), 2, n)
        return np.concatenate([(M[s].T @ yy[mu].T).ravel() for mu, s in enumerate(ids)])

    xd = torch.from_numpy(xg).cuda()
    yd = torch.empty_like(xd)
    smr.smr_matvec(ctx, xd, yd, smr.SMR_PREC_FP64)
    torch.cuda.synchronize()
    ref = lifted(oml.MLFMA(sc, workloads.PITCH).matvec(xo), Mo)
    got = lifted(yd.cpu().numpy(), Ms)
    assert np.max(np.abs(got - ref)) / np.max(np.abs(ref)) < 1e-10
    smr.smr_destroy(ctx)


def test_displaced_scenes_rejected():
    """Overlapping neighbours, a particle reaching a pitch from its cell
    centre (in the plane or, for a centre off the mean plane, in 3D) and two
    overlapping particles in one cell are refused with SMR_E_INVALID_ARG,
    and the context stays usable."""
    ctx = smr.smr_create(pitch=0.5)
    smr.smr_add_sphere(ctx, 0.15, 4, 4)
    ids = np.zeros(4, dtype=np.int32)
    good = workloads.lattice(2, 2)
    bad = []
    c = good.copy(); c[0, 0] += 0.24; c[1, 0] -= 0.2          # neighbours 0.06 apart
    bad.append(c)
    c = good.copy(); c[0, :2] += 0.249                          # 0.352 + 0.15 >= 0.5
    bad.append(c)
    c = good.copy(); c[1, :2] = c[0, :2] + [0.1, 0.0]          # overlapping, one cell
    bad.append(c)
    c = good.copy(); c[2, 2] += 0.6                             # 0.45 above the mean plane: 0.45 + 0.15
    bad.append(c)
    for cc in bad:
        with pytest.raises(smr.SmrError) as e:
            smr.smr_set_scene(ctx, cc, ids, 4.0)
        assert e.value.code == smr.SMR_E_INVALID_ARG
    c = good.copy(); c[:, :2] += np.array([[0.03, -0.02], [0.0, 0.04], [-0.05, 0.0], [0.01, 0.01]])
    smr.smr_set_scene(ctx, c, ids, 4.0)
    assert smr.smr_info(ctx)["n_near_blocks"] == 1 + 12
    smr.smr_destroy(ctx)


@pytest.fixture(scope="module")
def dense():
    # the paper's spiral spacing (c = sqrt(3) R): up to 4 centres per cell
    c = Case(workloads.make("spiral_dense", n=150, R=0.1, modes=8))
    yield c
    smr.smr_destroy(c.ctx)


@pytest.fixture(scope="module")
def moire():
    # two 4 x 4-cell honeycomb layers 0.5 apart, the upper turned by 5 deg
    c = Case(workloads.make("moire", m=4, shape="sphere", modes=6))
    yield c
    smr.smr_destroy(c.ctx)


@pytest.mark.parametrize("which", ["dense", "moire"])
def test_several_particles_per_cell(dense, moire, which):
    c = dense if which == "dense" else moire
    t = c.M.tree
    assert not t.one_per_cell
    assert c.info["n_box"][0] == len(t.levels[0]["ij"]) < c.sc.p
    for s in range(t.n_levels):
        assert c.info["n_box"][s] == len(t.levels[s]["ij"])
        assert c.info["n_il"][s] == len(t.levels[s]["il"])
    x = crandn(c.info["n_unknowns"], 8)
    ref = c.M.matvec(x)
    assert rel(c.gpu_matvec(x), ref) < 1e-10
    # the level-0 outgoing spectra of that product: each box the sum of its
    # particles' spectra, boxes in the oracle's order
    assert rel(smr.smr_copy_level(c.ctx, 0, 0)[..., 0], c.M.aggregate(x)) < 1e-12
    assert rel(c.gpu_matvec(x, smr.SMR_PREC_FP32), ref) < 2e-5
    # pair blocks, including pairs inside one cell
    same = [(mu, nu) for (mu, nu) in t.near_pairs() if mu != nu and t.cell[mu] == t.cell[nu]]
    assert same
    for mu, nu in same[:6]:
        assert rel(smr.smr_copy_pair_block(c.ctx, int(mu), int(nu)), c.M.near_block(mu, nu)) < 1e-12


def test_moire_solve(moire):
    c = moire
    kh, pol = workloads.incidence(0, 0, "x")
    n = c.info["n_unknowns"]
    b = torch.empty(n, dtype=torch.complex128, device="cuda")
    smr.smr_rhs_plane_waves(c.ctx, [kh], [pol], b)
    torch.cuda.synchronize()
    bo = opm.rhs(c.sc, kh, pol)
    assert rel(b.cpu().numpy(), bo) < 1e-12
    for prec, tol in ((smr.SMR_PREC_FP64, 1e-10), (smr.SMR_PREC_FP32, 1e-6)):
        x = torch.zeros_like(b)
        rc, st = smr.smr_solve(c.ctx, b, x, tol=tol, maxit=400, precision=prec)
        assert rc == 0
        assert np.linalg.norm(bo - c.M.matvec(x.cpu().numpy())) / np.linalg.norm(bo) <= 1.01 * tol
    # the cluster preconditioner needs one particle per cell
    z = torch.empty_like(b)
    with pytest.raises(smr.SmrError):
        smr.smr_precond_cluster(c.ctx, b, z)


@pytest.mark.parametrize("which", ["dense", "jit"])
def test_batched_columns_with_displaced_particles(dense, jit, which):
    """R = 3 right-hand sides in one product (FP64: the batched kernels with
    the per-particle spectra R wide; FP32: column by column) equal the
    single products column by column."""
    c = dense if which == "dense" else jit
    n = c.info["n_unknowns"]
    X = np.stack([crandn(n, 20 + j) for j in range(3)], axis=1)      # [n][R], R innermost
    for prec, tol in ((smr.SMR_PREC_FP64, 1e-13), (smr.SMR_PREC_FP32, 1e-6)):
        xd = torch.from_numpy(np.ascontiguousarray(X.ravel())).cuda()
        yd = torch.empty_like(xd)
        smr.smr_matvec(c.ctx, xd, yd, prec, R=3)
        torch.cuda.synchronize()
        Y = yd.cpu().numpy().reshape(n, 3)
        for j in range(3):
            assert rel(Y[:, j], c.gpu_matvec(X[:, j].copy(), prec)) < tol, (prec, j)
