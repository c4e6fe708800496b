"""GMRES for the PMCHWT system (FP64), as used in Sec. V, stage v.

Test infrastructure only (see ``oracle/__init__``).

Right-preconditioned GMRES (Saad & Schultz 1986): minimise ||b - A M^{-1} u||
over the Krylov space of A M^{-1}, x = x0 + M^{-1} u, with modified
Gram-Schmidt Arnoldi and Givens rotations; the iteration stops when the
TRUE relative residual ||b - A x|| / ||b|| reaches ``tol`` (checked whenever
the Givens estimate does).  M^{-1} is the block-diagonal preconditioner built
from the self blocks Z_s (Sec. V, stage v).
"""
import numpy as np


def block_diag_precond(scene):
    """x -> blockdiag(Z_s^{-1}) x over particles."""
    n2 = 2 * scene.n_psi
    inv = {s: np.linalg.inv(scene.self_block(s)) for s in set(scene.shape_ids.tolist())}
    ids = scene.shape_ids

    def apply(r):
        rr = r.reshape(-1, n2)
        z = np.empty_like(rr)
        for mu in range(rr.shape[0]):
            z[mu] = inv[ids[mu]] @ rr[mu]
        return z.reshape(-1)
    return apply


def gmres(matvec, b, precond=None, x0=None, tol=1e-4, restart=None, maxit=2000):
    """Returns (x, info) with info = dict(iters, matvecs, resid_true, history)."""
    M = precond if precond is not None else (lambda v: v)
    b = np.asarray(b, dtype=complex)
    n = b.size
    bn = np.linalg.norm(b)
    x = np.zeros(n, dtype=complex) if x0 is None else np.array(x0, dtype=complex)
    m = restart or maxit
    hist, its, mvs = [], 0, 0
    r = b - matvec(x) if x0 is not None else b.copy()
    mvs += x0 is not None
    while True:
        beta = np.linalg.norm(r)
        if beta / bn <= tol or its >= maxit:
            return x, dict(iters=its, matvecs=mvs, resid_true=beta / bn, history=hist)
        V = np.zeros((m + 1, n), dtype=complex)
        H = np.zeros((m + 1, m), dtype=complex)
        cs = np.zeros(m, dtype=complex)
        sn = np.zeros(m, dtype=complex)
        g = np.zeros(m + 1, dtype=complex)
        g[0] = beta
        V[0] = r / beta
        j_end = 0
        for j in range(m):
            w = matvec(M(V[j]))
            mvs += 1
            its += 1
            for i in range(j + 1):                 # modified Gram-Schmidt
                H[i, j] = np.vdot(V[i], w)
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] != 0:
                V[j + 1] = w / H[j + 1, j]
            for i in range(j):                     # previous rotations
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -np.conj(sn[i]) * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            a, c = H[j, j], H[j + 1, j]
            den = np.sqrt(abs(a) ** 2 + abs(c) ** 2)
            cs[j] = abs(a) / den if a != 0 else 0.0
            sn[j] = (a / abs(a)) * np.conj(c) / den if a != 0 else 1.0
            H[j, j] = cs[j] * a + sn[j] * c
            H[j + 1, j] = 0.0
            g[j + 1] = -np.conj(sn[j]) * g[j]
            g[j] = cs[j] * g[j]
            hist.append(abs(g[j + 1]) / bn)
            j_end = j + 1
            if abs(g[j + 1]) / bn <= tol or its >= maxit or H[j, j] == 0:
                break
        y = np.linalg.solve(np.triu(H[:j_end, :j_end]), g[:j_end])
        x = x + M(V[:j_end].T @ y)
        r = b - matvec(x)
        mvs += 1
