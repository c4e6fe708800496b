"""Rotated particles on the GPU against the FP64 oracle (the in-plane
rotations of Sec. V's brick and nanofin arrays): shapes made by
smr_add_shape_rotated from a fin given as data (element-wise parity) or as a
mesh (parity lifted to RWG coefficients), and a small geometric-phase lens
of fins solved to tolerance.

Bars: patterns <= 1e-13, FP64 product <= 1e-10, FP32 product <= 2e-5,
solutions to their tolerance in the oracle's true residual."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from oracle import mesh as om
from oracle import mlfma as oml
from oracle import pmchwt as opm
from paper_2407_21724_gb300 import smr, workloads

ANGLES = [0.0, 0.4, 1.3, 2.9]


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def crandn(n, seed):
    rng = np.random.default_rng(seed)
    return (rng.standard_normal(n) + 1j * rng.standard_normal(n)) / math.sqrt(2)


def matvec(ctx, x, prec):
    xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    yd = torch.empty_like(xd)
    smr.smr_matvec(ctx, xd, yd, prec)
    torch.cuda.synchronize()
    return yd.cpu().numpy()


@pytest.fixture(scope="module")
def fin():
    V, T = workloads.box_mesh(*workloads.FIN, 5, 1, 6)
    mm = om.MeshModes(om.Mesh(V, T), 6, 6)
    return V, T, mm, mm.sampled(opm.Medium(1.0), opm.Medium(4.0))


def _scene(n=5, seed=2):
    C = workloads.lattice(n, n)
    ids = np.random.default_rng(seed).integers(0, len(ANGLES), size=n * n).astype(np.int32)
    return C, ids


def test_sampled_fin_rotations_match_oracle(fin):
    _, _, _, sh = fin
    C, ids = _scene()
    ctx = smr.smr_create(pitch=workloads.PITCH)
    base = smr.smr_add_shape_sampled(ctx, sh.r, sh.w, sh.n_perp, sh.n_par, sh.psi, sh.div, sh.Zs)
    for a in ANGLES[1:]:
        smr.smr_add_shape_rotated(ctx, base, a)
    smr.smr_set_scene(ctx, C, ids, 4.0)
    shapes = [sh] + [dict(kind="rotated", base=0, angle=a) for a in ANGLES[1:]]
    sc = opm.Scene(C, ids, shapes, eps_in=4.0)
    M = oml.MLFMA(sc, workloads.PITCH)
    for s in range(len(ANGLES)):
        assert rel(smr.smr_copy_pattern(ctx, s), M.patterns[s]) < 1e-13
        assert np.array_equal(smr.smr_self_block(ctx, s), sh.Zs)
    x = crandn(smr.smr_info(ctx)["n_unknowns"], 5)
    ref = M.matvec(x)
    assert rel(matvec(ctx, x, smr.SMR_PREC_FP64), ref) < 1e-10
    assert rel(matvec(ctx, x, smr.SMR_PREC_FP32), ref) < 2e-5
    # rotating a rotated copy composes the angles
    s2 = smr.smr_add_shape_rotated(ctx, len(ANGLES) - 1, 0.5)
    smr.smr_set_scene(ctx, C, ids, 4.0)
    P2 = smr.smr_copy_pattern(ctx, s2)
    sc2 = opm.Scene(C, ids, shapes + [dict(kind="rotated", base=0, angle=ANGLES[-1] + 0.5)], eps_in=4.0)
    assert rel(P2, oml.MLFMA(sc2, workloads.PITCH).patterns[s2]) < 1e-12
    smr.smr_destroy(ctx)


def test_meshed_fin_rotations_match_oracle(fin):
    """The fin as a mesh on the GPU: its modes differ from the oracle's by
    a change of basis inside clusters of equal eigenvalues, so the product is
    compared lifted to RWG coefficients (x = M c per particle, y as M^T y);
    a rotated copy keeps the base's M and self block."""
    V, T, mm, sh = fin
    C, ids = _scene(4, 3)
    ctx = smr.smr_create(pitch=workloads.PITCH)
    base = smr.smr_add_shape_mesh(ctx, V, T, 6, 6)
    for a in ANGLES[1:]:
        smr.smr_add_shape_rotated(ctx, base, a)
    smr.smr_set_scene(ctx, C, ids, 4.0)
    Mg, g = smr.smr_shape_modes(ctx, base)
    for s in range(1, len(ANGLES)):
        Ms, gs = smr.smr_shape_modes(ctx, s)
        assert np.array_equal(Ms, Mg) and np.array_equal(gs, g)
        assert np.array_equal(smr.smr_self_block(ctx, s), smr.smr_self_block(ctx, base))
    shapes = [sh] + [dict(kind="rotated", base=0, angle=a) for a in ANGLES[1:]]
    sc = opm.Scene(C, ids, shapes, eps_in=4.0)
    n = 12
    rng = np.random.default_rng(9)
    cc = rng.standard_normal((len(ids), 2, Mg.shape[1])) + 1j * rng.standard_normal((len(ids), 2, Mg.shape[1]))
    xg = np.concatenate([(Mg @ cc[mu].T).T.ravel() for mu in range(len(ids))])
    xo = np.concatenate([(mm.M @ cc[mu].T).T.ravel() for mu in range(len(ids))])

    def lifted(y, M):
        yy = y.reshape(len(ids), 2, n)
        return np.concatenate([(M.T @ yy[mu].T).ravel() for mu in range(len(ids))])
    ref = lifted(oml.MLFMA(sc, workloads.PITCH).matvec(xo), mm.M)
    got = lifted(matvec(ctx, xg, smr.SMR_PREC_FP64), Mg)
    assert np.max(np.abs(got - ref)) / np.max(np.abs(ref)) < 1e-10
    smr.smr_destroy(ctx)


def test_pb_lens_solve(fin):
    """An 8 x 8 geometric-phase lens of coarse fins in 8 rotations, circular
    polarisation: GMRES (FP64 and mixed) reaches its tolerance in the
    oracle's true residual, and the far field is the oracle's."""
    _, _, _, sh = fin
    w = workloads.make("pbfins", n=8, bins=8)
    C, ids = w["centres"], w["shape_ids"]
    ctx = smr.smr_create(pitch=workloads.PITCH)
    base = smr.smr_add_shape_sampled(ctx, sh.r, sh.w, sh.n_perp, sh.n_par, sh.psi, sh.div, sh.Zs)
    shapes = [sh]
    for b in range(1, 8):
        smr.smr_add_shape_rotated(ctx, base, b * np.pi / 8)
        shapes.append(dict(kind="rotated", base=0, angle=b * np.pi / 8))
    smr.smr_set_scene(ctx, C, ids, 4.0)
    sc = opm.Scene(C, ids, shapes, eps_in=4.0)
    M = oml.MLFMA(sc, workloads.PITCH)
    kh, pol = w["incidences"][0]
    n = smr.smr_info(ctx)["n_unknowns"]
    b = torch.empty(n, dtype=torch.complex128, device="cuda")
    smr.smr_rhs_plane_waves(ctx, [kh], [pol], b)
    torch.cuda.synchronize()
    bo = opm.rhs(sc, kh, pol)
    assert rel(b.cpu().numpy(), bo) < 1e-12
    dirs = np.array([[0, 0, 1.0], [0, 0, -1.0], [0.6, 0, 0.8], [0, 0.8, -0.6], [1.0, 0, 0]])
    for prec, tol in ((smr.SMR_PREC_FP64, 1e-10), (smr.SMR_PREC_FP32, 1e-6)):
        x = torch.zeros_like(b)
        rc, st = smr.smr_solve(ctx, b, x, tol=tol, maxit=400, precision=prec)
        assert rc == 0
        xh = x.cpu().numpy()
        assert np.linalg.norm(bo - M.matvec(xh)) / np.linalg.norm(bo) <= 1.01 * tol
        Fd = torch.empty(len(dirs) * 3, dtype=torch.complex128, device="cuda")
        smr.smr_far_field(ctx, x, dirs, Fd)
        torch.cuda.synchronize()
        assert rel(Fd.cpu().numpy().reshape(len(dirs), 3), opm.far_field(sc, xh, dirs)) < 1e-12
    smr.smr_destroy(ctx)


def test_rotating_a_sphere_is_refused():
    ctx = smr.smr_create(pitch=0.5)
    s = smr.smr_add_sphere(ctx, 0.15, 4, 4)
    with pytest.raises(smr.SmrError) as e:
        smr.smr_add_shape_rotated(ctx, s, 0.3)
    assert e.value.code == smr.SMR_E_SHAPE
    with pytest.raises(smr.SmrError):
        smr.smr_add_shape_rotated(ctx, 5, 0.3)
    smr.smr_destroy(ctx)
