"""Meshed particles on the GPU against the oracle (Sec. III static modes,
Sec. II self block with Eq. 20, the MLFMA product on their samples).

The two sides solve their own eigenproblems, so their modes agree only up to
an orthogonal change of basis inside each cluster of equal eigenvalues (the
cylinders have an 8-fold axis: most modes come in pairs).  The comparisons
are therefore of what the basis does not change, at mode counts whose cut
falls between clusters:
  * the kept eigenvalues;
  * the projector M^T M G onto the span of the modes (G the RWG Gram);
  * the self block lifted to RWG coefficients, M^T Z_s M, block by block;
  * products lifted the same way: x = M c for an RWG vector c per particle
    and current, y = Z x, compared as M^T y;
  * far fields of solved scattering problems.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from oracle import gmres as ogm
from oracle import mesh as om
from oracle import mlfma as oml
from oracle import pmchwt as pm
from paper_2407_21724_gb300 import smr, workloads

NP = 6                                            # modes per kind: cut between clusters
CYL = [(0.12, 0.6, 8, 3, 2), (0.18, 0.6, 8, 3, 2)]   # 96 triangles each


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


@pytest.fixture(scope="module")
def meshes():
    out = []
    for args in CYL:
        V, T = workloads.cylinder_mesh(*args)
        mm = om.MeshModes(om.Mesh(V, T), NP, NP)
        gp, gl = mm.gamma_perp_all, mm.gamma_par_all
        # the cut separates clusters on both sides
        assert (gp[NP - 1] - gp[NP]) > 1e-3 * gp[NP - 1] and (gl[NP] - gl[NP - 1]) > 1e-3 * gl[NP]
        out.append((V, T, mm))
    return out


@pytest.fixture(scope="module")
def scene(meshes):
    """3 x 3 lattice of the two cylinders, eps = 4 in vacuum."""
    C = workloads.lattice(3, 3)
    ids = np.array([0, 1, 0, 1, 1, 0, 0, 0, 1], dtype=np.int32)
    ctx = smr.smr_create(pitch=workloads.PITCH)
    for V, T, _ in meshes:
        smr.smr_add_shape_mesh(ctx, V, T, NP, NP)
    smr.smr_set_scene(ctx, C, ids, 4.0)
    outer, inner = pm.Medium(1.0), pm.Medium(4.0)
    shapes = [mm.sampled(outer, inner) for _, _, mm in meshes]
    sc = pm.Scene(C, ids, shapes, eps_in=4.0)
    yield ctx, sc, C, ids
    smr.smr_destroy(ctx)


def test_modes_match_oracle(meshes, scene):
    ctx = scene[0]
    for s, (_, _, mm) in enumerate(meshes):
        M, g = smr.smr_shape_modes(ctx, s)
        assert M.shape == mm.M.shape
        assert np.max(np.abs(g - np.r_[mm.gamma_perp, mm.gamma_par]) / np.abs(g)) < 1e-10
        for sl in (slice(0, NP), slice(NP, 2 * NP)):
            Pg = M[sl].T @ M[sl] @ mm.G
            Po = mm.M[sl].T @ mm.M[sl] @ mm.G
            assert np.max(np.abs(Pg - Po)) < 1e-9
            # G-orthonormal within each kind (loops and stars of a mesh are
            # not orthogonal to each other)
            assert np.max(np.abs(M[sl] @ mm.G @ M[sl].T - np.eye(NP))) < 1e-10


def test_host_mode_solve_equals_context(meshes, scene):
    ctx = scene[0]
    for s, (V, T, _) in enumerate(meshes):
        M0, g0 = smr.smr_shape_modes(ctx, s)
        M1, g1 = smr.smr_mesh_static_modes(V, T, NP, NP)
        assert np.array_equal(M0, M1) and np.array_equal(g0, g1)


def test_self_block_matches_oracle(meshes, scene):
    ctx, sc = scene[0], scene[1]
    n = 2 * NP
    for s, (_, _, mm) in enumerate(meshes):
        Zg = smr.smr_self_block(ctx, s)
        Zo = sc.shapes[s].Zs
        Mg, _ = smr.smr_shape_modes(ctx, s)
        for bi in range(2):
            for bj in range(2):
                Lg = Mg.T @ Zg[bi * n:(bi + 1) * n, bj * n:(bj + 1) * n] @ Mg
                Lo = mm.M.T @ Zo[bi * n:(bi + 1) * n, bj * n:(bj + 1) * n] @ mm.M
                assert _rel(Lg, Lo) < 1e-10, (s, bi, bj, _rel(Lg, Lo))


def _lifted_inputs(Ms, Mo, ids, rng):
    """x for the GPU (modes Ms per shape) and the oracle (Mo) from one random
    RWG vector per (particle, current): x = M c on each side."""
    xs_g, xs_o = [], []
    for s in ids:
        c = rng.standard_normal((2, Ms[s].shape[1])) + 1j * rng.standard_normal((2, Ms[s].shape[1]))
        xs_g.append((Ms[s] @ c.T).T.ravel())
        xs_o.append((Mo[s] @ c.T).T.ravel())
    return np.concatenate(xs_g), np.concatenate(xs_o)


def _lift(y, Ms, ids, n):
    """M^T y per (particle, current): the product in RWG coefficients."""
    yy = y.reshape(len(ids), 2, n)
    return np.concatenate([(Ms[s].T @ yy[mu].T).ravel() for mu, s in enumerate(ids)])


def test_product_matches_oracle(meshes, scene):
    ctx, sc, C, ids = scene
    Ms = [smr.smr_shape_modes(ctx, s)[0] for s in range(len(meshes))]
    Mo = [mm.M for _, _, mm in meshes]
    xg, xo = _lifted_inputs(Ms, Mo, ids, np.random.default_rng(7))
    xd = torch.from_numpy(xg).cuda()
    yd = torch.empty_like(xd)
    smr.smr_matvec(ctx, xd, yd, smr.SMR_PREC_FP64)
    torch.cuda.synchronize()
    yo = oml.MLFMA(sc, workloads.PITCH).matvec(xo)
    n = 2 * NP
    ref = _lift(yo, Mo, ids, n)
    assert _rel(_lift(yd.cpu().numpy(), Ms, ids, n), ref) < 1e-10
    # the FP32 product within the FP32 bar
    smr.smr_matvec(ctx, xd, yd, smr.SMR_PREC_FP32)
    torch.cuda.synchronize()
    assert _rel(_lift(yd.cpu().numpy(), Ms, ids, n), ref) < 2e-5


def test_solved_far_field_matches_oracle(scene):
    """Plane-wave scattering by the 3 x 3 array: GPU GMRES (FP64) against the
    oracle's GMRES on its MLFMA product; far fields do not depend on the mode
    basis."""
    ctx, sc, C, ids = scene
    kh, pol = workloads.incidence(20, 30, "x")
    n = smr.smr_info(ctx)["n_unknowns"]
    b = torch.empty(n, dtype=torch.complex128, device="cuda")
    smr.smr_rhs_plane_waves(ctx, [kh], [pol], b)
    x = torch.zeros_like(b)
    rc, st = smr.smr_solve(ctx, b, x, tol=1e-11, maxit=400, precision=smr.SMR_PREC_FP64)
    assert rc == 0
    xo, _ = ogm.gmres(oml.MLFMA(sc, workloads.PITCH).matvec, pm.rhs(sc, kh, pol), tol=1e-12)
    dirs = np.array([[0, 0, 1.0], [0, 0, -1.0], [0.6, 0, 0.8], [0, 0.8, -0.6], [1.0, 0, 0]])
    Fo = pm.far_field(sc, xo, dirs)
    Fd = torch.empty(len(dirs) * 3, dtype=torch.complex128, device="cuda")
    smr.smr_far_field(ctx, x, dirs, Fd)
    torch.cuda.synchronize()
    assert _rel(Fd.cpu().numpy().reshape(len(dirs), 3), Fo) < 1e-8


def test_rejected_meshes():
    ctx = smr.smr_create(pitch=0.5)
    try:
        V, T = workloads.cylinder_mesh(0.1, 0.3, 8, 2, 2)
        with pytest.raises(smr.SmrError) as e:
            smr.smr_add_shape_mesh(ctx, V, T[:-1], 2, 2)          # open
        assert e.value.code == smr.SMR_E_SHAPE
        with pytest.raises(smr.SmrError) as e:
            smr.smr_add_shape_mesh(ctx, V, T[:, ::-1], 2, 2)      # inward normals
        assert e.value.code == smr.SMR_E_SHAPE
        with pytest.raises(smr.SmrError) as e:
            smr.smr_add_shape_mesh(ctx, V, T, len(V), 2)         # more loops than the mesh has
        assert e.value.code == smr.SMR_E_SHAPE
    finally:
        smr.smr_destroy(ctx)


def test_near_sweep_preconditioner(scene):
    """SMR_PRECOND_NEAR (block-diagonal plus one or two Jacobi sweeps over the
    near field): the solve meets the tolerance on the oracle's operator, in
    fewer iterations than the block-diagonal preconditioner, and in as many as
    the oracle's GMRES with the same preconditioner built from its own near
    blocks (iteration counts do not depend on the mode basis)."""
    ctx, sc, C, ids = scene
    kh, pol = workloads.incidence(0, 0, "x")
    n = smr.smr_info(ctx)["n_unknowns"]
    b = torch.empty(n, dtype=torch.complex128, device="cuda")
    smr.smr_rhs_plane_waves(ctx, [kh], [pol], b)
    M = oml.MLFMA(sc, workloads.PITCH)
    bo = pm.rhs(sc, kh, pol)
    # the oracle's near matrix (self + the 8 lattice neighbours), split D + N
    Z = pm.dense_matrix(sc)
    m = 2 * sc.n_psi
    ij = np.round(np.asarray(C)[:, :2] / workloads.PITCH).astype(int)
    Dinv = np.zeros_like(Z)
    Zn = np.zeros_like(Z)
    for a in range(len(ids)):
        for c in range(len(ids)):
            if np.max(np.abs(ij[a] - ij[c])) <= 1:
                Zn[a * m:(a + 1) * m, c * m:(c + 1) * m] = Z[a * m:(a + 1) * m, c * m:(c + 1) * m]
        Dinv[a * m:(a + 1) * m, a * m:(a + 1) * m] = np.linalg.inv(Z[a * m:(a + 1) * m, a * m:(a + 1) * m])
    dirs = np.array([[0, 0, 1.0], [0, 0, -1.0], [0.6, 0, 0.8], [0, 0.8, -0.6]])
    iters = {}
    for sweeps in (1, 2):
        def pc(v, k=sweeps):
            t = Dinv @ v
            z = t.copy()
            for _ in range(k):
                z = z + t - Dinv @ (Zn @ z)
            return z
        xo, info = ogm.gmres(M.matvec, bo, precond=pc, tol=1e-6)
        Fo = pm.far_field(sc, xo, dirs)
        for prec in (smr.SMR_PREC_FP64, smr.SMR_PREC_FP32):
            x = torch.zeros_like(b)
            rc, st = smr.smr_solve(ctx, b, x, tol=1e-6, maxit=400, precision=prec,
                                   precond=smr.SMR_PRECOND_NEAR, near_sweeps=sweeps)
            # the library's true residual uses its FP64 product, which equals
            # the oracle's (lifted-product test); far fields are basis-free
            assert rc == 0 and st["resid_true"] <= 1e-6
            Fd = torch.empty(len(dirs) * 3, dtype=torch.complex128, device="cuda")
            smr.smr_far_field(ctx, x, dirs, Fd)
            torch.cuda.synchronize()
            assert _rel(Fd.cpu().numpy().reshape(len(dirs), 3), Fo) < 1e-4
            if prec == smr.SMR_PREC_FP64:
                assert abs(st["iters"] - info["iters"]) <= 1, (sweeps, st["iters"], info["iters"])
                iters[sweeps] = st["iters"]
    x = torch.zeros_like(b)
    rc, st = smr.smr_solve(ctx, b, x, tol=1e-6, maxit=400, precision=smr.SMR_PREC_FP64)
    assert rc == 0 and iters[1] < st["iters"]
    # the cluster block-Jacobi preconditioner on the pillars
    for prec in (smr.SMR_PREC_FP64, smr.SMR_PREC_FP32):
        x = torch.zeros_like(b)
        rc, sc_st = smr.smr_solve(ctx, b, x, tol=1e-6, maxit=400, precision=prec,
                                  precond=smr.SMR_PRECOND_CLUSTER)
        assert rc == 0 and sc_st["resid_true"] <= 1e-6
        Fd = torch.empty(len(dirs) * 3, dtype=torch.complex128, device="cuda")
        smr.smr_far_field(ctx, x, dirs, Fd)
        torch.cuda.synchronize()
        assert _rel(Fd.cpu().numpy().reshape(len(dirs), 3), Fo) < 1e-4
    with pytest.raises(smr.SmrError):
        smr.smr_solve(ctx, b, x, precond=smr.SMR_PRECOND_NEAR, near_sweeps=0)
