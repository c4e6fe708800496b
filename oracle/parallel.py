"""The oracle's MLFMA product on every host core (FP64), for timing only.

Test infrastructure only (see ``oracle/__init__``): used by the CPU-baseline
and reference legs of ``bench.py``.

``ParallelMLFMA`` runs ``oracle.mlfma.MLFMA`` step by step, each step split
over disjoint subsets of the boxes (or particles) it writes, in worker
processes that write into level buffers held in shared memory.  Every entry
is computed by the same oracle code, with the same operations in the same
order, as the serial product, so the result is bit-identical to
``MLFMA.matvec`` (checked by tests/test_oracle_parallel.py).  Workers are
forked from a process that has not touched a GPU; the caller should pin the
BLAS pools to one thread (OMP_NUM_THREADS=1 and the like, before NumPy is
imported), or the workers oversubscribe the cores.
"""
import mmap
import multiprocessing as mp
import os

import numpy as np

from .mlfma import MLFMA
from .pmchwt import exterior_block

_G = {}        # state inherited by forked workers


def _shared(shape, dtype=complex):
    n = int(np.prod(shape)) * np.dtype(dtype).itemsize
    buf = mmap.mmap(-1, max(n, 1))
    return np.frombuffer(buf, dtype=dtype, count=int(np.prod(shape))).reshape(shape)


def _near_block_task(task):
    key, dc = task
    sc = _G["scene"]
    if key[0] == "self":
        return key, sc.self_block(key[1])
    return key, exterior_block(sc, key[0], dc, key[1], np.zeros(3))


def _step(task):
    M, B = _G["M"], _G["bufs"]
    kind, s, idx = task
    if kind == "near":
        M.near(B["x"], mus=idx, out=B["yn"])
    elif kind == "agg":
        M.aggregate(B["x"], mus=idx, out=B["out"][0])
    elif kind == "agg_box":
        M.aggregate(B["x"], out=B["out"][0], boxes=idx)
    elif kind == "up":
        M.upward(s, B["out"][s], parents=idx, out=B["out"][s + 1])
    elif kind == "tr":
        M.translate(s, B["out"][s], targets=idx, inc=B["in"][s])
    elif kind == "down":
        d = M.downward(s, B["in"][s + 1], children=idx, out=B["tmp"][s])
        B["in"][s][idx] = B["in"][s][idx] + d[idx]
    elif kind == "recv":
        M.receive(B["in"][0], mus=idx, out=B["yf"])
    return 0


class ParallelMLFMA:
    """Full oracle set-up and product over `workers` processes (default: all
    host cores).  Call close() when done."""

    def __init__(self, scene, pitch, workers=None, **kw):
        self.workers = workers or os.cpu_count() or 1
        ctx = mp.get_context("fork")
        _G["scene"] = scene
        with ctx.Pool(self.workers) as pool:
            M = MLFMA(scene, pitch, pmap=pool.map, **kw)
            # every distinct near block once (the keys MLFMA.near_block uses),
            # each computed for the exact offset of the first pair that
            # names it, as the serial product does
            keys = {}
            for mu, nu in M.tree.near_pairs():
                sm, sn = scene.shape_ids[mu], scene.shape_ids[nu]
                if mu == nu:
                    keys.setdefault(("self", sm), None)
                else:
                    d = tuple(M.tree.ij0[mu] - M.tree.ij0[nu])
                    dc = scene.centres[mu] - scene.centres[nu]
                    keys.setdefault((sm, sn, d) + tuple(np.round(dc, 12)), dc)
            tasks = sorted(keys.items(), key=lambda kv: str(kv[0]))
            for key, blk in pool.map(_near_block_task, tasks, chunksize=4):
                M._near_cache[key] = blk
        self.M = M
        p, n2 = scene.p, 2 * scene.n_psi
        t = M.tree
        self.bufs = dict(
            x=_shared((p * n2,)), yn=_shared((p * n2,)), yf=_shared((p * n2,)),
            out=[_shared((len(t.levels[s]["ij"]), M.grids[s].K, 4)) for s in range(t.n_levels)],
            tmp=[_shared((len(t.levels[s]["ij"]), M.grids[s].K, 4)) for s in range(t.n_levels)])
        self.bufs["in"] = [_shared((len(t.levels[s]["ij"]), M.grids[s].K, 4)) for s in range(t.n_levels)]
        _G["M"], _G["bufs"] = M, self.bufs
        self.pool = ctx.Pool(self.workers)

    def _chunks(self, n):
        parts = min(n, 4 * self.workers)
        return [c for c in np.array_split(np.arange(n), parts) if len(c)]

    def _run(self, kind, s, n):
        self.pool.map(_step, [(kind, s, c) for c in self._chunks(n)])

    def matvec(self, x):
        M, B, t = self.M, self.bufs, self.M.tree
        B["x"][:] = np.asarray(x, dtype=complex).reshape(-1)
        p = self.M.scene.p
        self._run("near", 0, p)
        if t.one_per_cell:
            self._run("agg", 0, p)
        else:
            # several particles per cell sum into one box: split by boxes
            self._run("agg_box", 0, len(t.levels[0]["ij"]))
        for s in range(t.n_levels - 1):
            self._run("up", s, len(t.levels[s + 1]["ij"]))
        for s in range(t.n_levels):
            self._run("tr", s, len(t.levels[s]["ij"]))
        for s in range(t.n_levels - 2, -1, -1):
            self._run("down", s, len(t.levels[s]["ij"]))
        self._run("recv", 0, p)
        return B["yn"] + B["yf"]

    def close(self):
        self.pool.close()
        self.pool.join()
