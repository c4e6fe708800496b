"""Failure handling on the GPU, driven without faulting anything.

* A bounded tensor-core wait is made to run out by setting the polling limit
  to zero rounds (every wait that has to wait gives up at once).  The product
  must report SMR_E_TIMEOUT through smr_sync, drain its own copies and MMAs,
  free its tensor memory and leave the context usable: the next product at
  the default limit must be correct.
* An Arnoldi breakdown: a single particle whose self block (given as data) is
  singular makes Z singular; GMRES without a preconditioner reaches an
  invariant Krylov space with the residual still large and must stop with
  SMR_E_BREAKDOWN instead of running to maxit.  The block-diagonal
  preconditioner is undefined for that scene and is refused.
* Checkpoint and resume of a solve: restarted GMRES carries nothing across
  a restart but the iterate x.  A solve stopped at maxit (a multiple of the
  restart length) saves x to a file; a fresh context on the same scene
  resumes from it (use_x0) and converges, with the interrupted and resumed
  iterations adding up to the uninterrupted solve's and the same solution.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2407_21724_gb300 import smr, workloads


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_tensor_core_wait_gives_up_and_context_recovers():
    w = workloads.make("random", n=9, seed=5, modes=16)
    ctx = smr.scene_from_workload(w)
    try:
        n = smr.smr_info(ctx)["n_unknowns"]
        rng = np.random.default_rng(1)
        x = torch.from_numpy(rng.standard_normal(n) + 1j * rng.standard_normal(n)).cuda()
        y = torch.empty_like(x)
        smr.smr_matvec(ctx, x, y, smr.SMR_PREC_FP64)
        y64 = y.cpu().numpy()
        smr.smr_set_tensor_cores(ctx, True)
        smr.smr_set_wait_limit(ctx, 0)
        smr.smr_matvec(ctx, x, y, smr.SMR_PREC_FP32)
        with pytest.raises(smr.SmrError) as e:
            smr.smr_sync(ctx)
        assert e.value.code == smr.SMR_E_TIMEOUT
        smr.smr_sync(ctx)                        # the flag was cleared by the report
        smr.smr_set_wait_limit(ctx, -1)
        for _ in range(2):
            y.fill_(float("nan"))
            smr.smr_matvec(ctx, x, y, smr.SMR_PREC_FP32)
            smr.smr_sync(ctx)
            assert _rel(y.cpu().numpy(), y64) < 2e-5
    finally:
        smr.smr_destroy(ctx)


def test_breakdown_on_singular_operator():
    from oracle import pmchwt as pm
    from tests.sampled import media, rotated_sphere
    sh = rotated_sphere(0.15, 8, 8, media(4.0), seed=3)
    n2 = 2 * sh.n_psi
    # the unknown the plane wave drives most is taken out of the range of Z
    sc = pm.Scene([[0.0, 0.0, 0.0]], [0], [sh], eps_in=4.0)
    kk = int(np.argmax(np.abs(pm.rhs(sc, [0, 0, 1], [1, 0, 0]))))
    Zs = np.eye(n2, dtype=complex)
    Zs[kk, kk] = 0.0                           # rank n2 - 1: Z of one particle is singular
    ctx = smr.smr_create(pitch=0.5)
    try:
        smr.smr_add_shape_sampled(ctx, sh.r, sh.w, sh.n_perp, sh.n_par, sh.psi, sh.div, Zs)
        smr.smr_set_scene(ctx, [[0.0, 0.0, 0.0]], [0], 4.0)
        n = smr.smr_info(ctx)["n_unknowns"]
        b = torch.empty(n, dtype=torch.complex128, device="cuda")
        smr.smr_rhs_plane_waves(ctx, [[0.0, 0.0, 1.0]], [[1.0, 0.0, 0.0]], b)
        bh = b.cpu().numpy()
        assert abs(bh[kk]) > 0.1 * np.linalg.norm(bh)    # b has a part outside the range of Z
        x = torch.zeros_like(b)
        with pytest.raises(smr.SmrError) as e:
            smr.smr_solve(ctx, b, x, tol=1e-8, maxit=200, precond=smr.SMR_PRECOND_NONE,
                          precision=smr.SMR_PREC_FP64)
        assert e.value.code == smr.SMR_E_BREAKDOWN
        with pytest.raises(smr.SmrError) as e:
            smr.smr_solve(ctx, b, x, tol=1e-8, maxit=200, precond=smr.SMR_PRECOND_BLOCKDIAG,
                          precision=smr.SMR_PREC_FP64)
        assert e.value.code == -1
    finally:
        smr.smr_destroy(ctx)


@pytest.mark.parametrize("prec", [smr.SMR_PREC_FP64, smr.SMR_PREC_FP32])
def test_solve_resumes_from_a_checkpoint(tmp_path, prec):
    w = workloads.make("random", n=12, seed=8, modes=8)
    kh, pol = workloads.incidence(0, 0, "x")
    tol, m = (1e-8 if prec == smr.SMR_PREC_FP64 else 1e-6), 10

    def start():
        ctx = smr.scene_from_workload(w)
        n = smr.smr_info(ctx)["n_unknowns"]
        b = torch.empty(n, dtype=torch.complex128, device="cuda")
        smr.smr_rhs_plane_waves(ctx, [kh], [pol], b)
        return ctx, b

    ctx, b = start()
    x = torch.zeros_like(b)
    rc, full = smr.smr_solve(ctx, b, x, tol=tol, restart=m, maxit=2000, precision=prec, max_outer=40)
    assert rc == 0 and full["iters"] > 2 * m
    x_full = x.cpu().numpy()
    # interrupted after two restart cycles; the iterate goes to a file
    x.zero_()
    rc, part = smr.smr_solve(ctx, b, x, tol=tol, restart=m, maxit=2 * m, precision=prec, max_outer=40)
    assert rc == smr.SMR_E_NOT_CONVERGED and part["iters"] <= 2 * m
    np.save(tmp_path / "x.npy", x.cpu().numpy())
    smr.smr_destroy(ctx)
    # a new context resumes
    ctx, b = start()
    x = torch.from_numpy(np.load(tmp_path / "x.npy")).cuda()
    rc, rest = smr.smr_solve(ctx, b, x, tol=tol, restart=m, maxit=2000, precision=prec, use_x0=1,
                             max_outer=40)
    assert rc == 0 and rest["resid_true"] <= tol
    if prec == smr.SMR_PREC_FP64:
        # restarted FP64 GMRES: the two halves add up to the whole
        assert abs(part["iters"] + rest["iters"] - full["iters"]) <= 2 * m // 5 + 2
    else:
        # iterative refinement restarts its inner solves at every outer step
        assert rest["iters"] < full["iters"]
    assert _rel(x.cpu().numpy(), x_full) < 100 * tol
    smr.smr_destroy(ctx)
