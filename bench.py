"""Benchmark of the MLFMA-SMR product and GMRES solve on one GB300.

Workload (default): the 200 x 200 hyperbolic metalens of 8 radius-quantised
dielectric spheres (eps_r = 4, pitch 0.5 wavelength, f = 50 wavelengths),
32 static modes per current: 2,560,000 complex unknowns, 7 interacting
levels.  A step is one MLFMA-SMR product y = Z x (near block-sparse product,
aggregation, interpolation, translation, anterpolation, receive) in the tuned
precision (FP32 arithmetic from FP64-generated tables, FP64 in and out).
The same line carries the plain-FP64 product rate and, measured after the
timed steps, the GMRES time to a 1e-4 true relative residual for the tuned
solver (FP64-outer iterative refinement over FP32-inner GMRES) and for plain
FP64 GMRES.

The reference arm (--impl reference) and the line's cpu_baseline time the
FP64 oracle's full product of the same workload on all host cores.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
       [--workload metalens200|random40|spheres8x8] [--no-solve]
For N > 1 launch with torch.distributed.run: every rank runs its own replica
(weak scaling, no collective on the data path).
"""
import argparse
import json
import os
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)
if "reference" in sys.argv:
    # the oracle runs single-threaded: pin every BLAS pool before NumPy loads
    for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[_v] = "1"

WORKLOADS = {
    "metalens200": ("metalens", dict(n=200, focal=50.0, shape="pillar")),
    "metalens150": ("metalens", dict(n=150, focal=40.0, shape="pillar")),
    "random40": ("random", dict(n=40, seed=21724, shape="pillar")),
    "batched100x64": ("random", dict(n=100, seed=21725, shape="pillar")),
    "random100": ("random", dict(n=100, seed=21725, shape="pillar")),
    "ragged16": ("ragged16", dict(shape="pillar")),
    "spheres8x8": ("spheres8x8", {}),
    # off-lattice scenes (spheres: one exterior near block per displaced pair)
    "jittered40": ("jittered", dict(n=40, seed=21728, jitter=0.02)),
    "lattice40": ("random", dict(n=40, seed=21728)),
    "spiral1600": ("spiral", dict(n=1600)),
    # rotated particles: 100 x 100 geometric-phase lens of nanofins, 16 rotations
    "pbfins100": ("pbfins", dict(n=100, bins=16)),
    # several particles per finest box: the paper's spiral spacing, and a
    # two-layer Moire lattice of meshed nanodisks
    "spiral_dense2000": ("spiral_dense", dict(n=2000)),
    "moire2k": ("moire", dict(m=22)),
    "moire20k": ("moire", dict(m=71)),            # the paper's 20,160-disk bilayer size
    # the paper's 40,000-brick golden-angle spiral, bricks turned in 64 steps
    "spiral_bricks40k": ("spiral_bricks", dict(n=40000, bins=64)),
}
METRIC = "MLFMA-SMR matvecs/s and GMRES time to 1e-4 residual, tuned vs plain FP64"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="metalens200", choices=sorted(WORKLOADS))
    ap.add_argument("--no-solve", action="store_true")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--train-arrays", type=int, default=None,
                    help="20x20 arrays solved to train the learned parts (0: skip); default 2000 on "
                         "metalens150, their evaluation scene, and 0 elsewhere")
    a = ap.parse_args()
    if a.train_arrays is None:
        a.train_arrays = 2000 if a.workload == "metalens150" else 0
    return a


# ------------------------------------------------------------------ reference arm (the oracle)
def oracle_rate(ws, steps, warmup):
    """Time the FP64 oracle's full MLFMA product of every scene in ws on all
    host cores (oracle.parallel: the oracle's own steps split over disjoint
    boxes in forked workers, bit-identical to the serial product).  A step is
    one product of each scene; returns (products per second per right-hand
    side, seconds per step, set-up seconds, workers)."""
    import numpy as np
    from oracle import pmchwt as opm
    from oracle.parallel import ParallelMLFMA
    from oracle.mesh import sampled_shapes
    t_step, t_setup, workers = 0.0, 0.0, 0
    built = {}
    for w in ws:
        t0 = time.perf_counter()
        # meshed shapes: the oracle's static modes and self blocks, each
        # distinct mesh once, the shapes in parallel (spawned processes)
        key = lambda s: s["verts"].tobytes() + s["tris"].tobytes() + bytes([s["n_perp"], s["n_par"]])
        mesh = lambda s: isinstance(s, dict) and s.get("kind") == "mesh"
        todo = {key(s): s for s in w["shapes"] if mesh(s) and key(s) not in built}
        if todo:
            for k, v in zip(todo, sampled_shapes(list(todo.values()), w["eps_in"], workers=os.cpu_count() or 1)):
                built[k] = v
        shapes = [built[key(s)] if mesh(s) else s for s in w["shapes"]]
        sc = opm.Scene(w["centres"], w["shape_ids"], shapes, eps_in=w["eps_in"])
        P = ParallelMLFMA(sc, w["pitch"], L0=w.get("L0", 10))
        t_setup += time.perf_counter() - t0
        workers = P.workers
        rng = np.random.default_rng(0)
        x = rng.standard_normal(sc.n_unknowns) + 1j * rng.standard_normal(sc.n_unknowns)
        try:
            for _ in range(warmup):
                P.matvec(x)
            t0 = time.perf_counter()
            for _ in range(steps):
                P.matvec(x)
            t_step += (time.perf_counter() - t0) / steps
        finally:
            P.close()
    return 1.0 / t_step, t_step, t_setup, workers


def run_reference(a):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_2407_21724_gb300 import workloads
    name, kw = WORKLOADS[a.workload]
    R = 64 if a.workload == "batched100x64" else 1
    if a.workload == "ragged16":
        ws = workloads.make(name, **kw)
        label = "ragged batch of 16 random arrays, 10x10 ... 60x60, one product"
    else:
        ws = [workloads.make(name, **kw)]
        label = ws[0]["label"]
    rate, t, t_setup, workers = oracle_rate(ws, a.steps, max(1, a.warmup))
    # the oracle applies one right-hand side per product: R columns cost R products
    sample = (f"the full workload: FP64 NumPy oracle MLFMA product of {sum(len(w['centres']) for w in ws)} "
              f"particles on {workers} worker processes (all host cores, BLAS single-threaded), "
              f"{t:.2f} s per product over {a.steps} timed products after {max(1, a.warmup)} warm-ups; "
              f"set-up (tables, near blocks) {t_setup:.1f} s, not timed"
              + (f"; {R} right-hand sides = {R} products" if R > 1 else ""))
    line = dict(metric=METRIC, value=rate, unit="matvecs/s", n_gpus=a.gpus, steps=a.steps,
                warmup=a.warmup, ms_per_step=1e3 * t, higher_is_better=True, scaling="weak",
                vs_baseline=None, dtype="f64", data="synthetic", impl="reference",
                config=dict(workload=label, rhs=R, l2="inputs larger than L2 (CPU run)"),
                cpu_baseline=dict(value=rate, unit="matvecs/s", cores=workers, kind="oracle", sample=sample,
                                  setup_seconds=t_setup),
                e2e=dict(value=rate, unit="matvecs/s", h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ our arm
def clocks_start(path):
    q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    try:
        f = open(path, "w")
        return subprocess.Popen(["nvidia-smi", "--query-gpu=" + q, "--format=csv,noheader,nounits",
                                 "-lms", "100"], stdout=f, stderr=subprocess.DEVNULL), f
    except (OSError, FileNotFoundError):
        return None, None


def clocks_stop(proc, f, path, dev):
    import statistics
    if proc is None:
        return None
    proc.terminate()
    proc.wait()
    f.close()
    sm, mx, reasons = [], None, set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in open(path):
        v = [s.strip() for s in line.split(",")]
        if len(v) < 9 or v[0] != str(dev):
            continue
        try:
            sm.append(float(v[1]))
            mx = float(v[2])
        except ValueError:
            continue
        for n, val in zip(names, v[5:9]):
            if val.lower() == "active":
                reasons.add(n)
    if not sm:
        return None
    return dict(sm_mhz=statistics.median(sm), sm_max_mhz=mx, reasons=sorted(reasons), samples=len(sm))


ALU_BOUND = ("near", "aggregate", "receive")
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12


def traffic_for(kernel):
    """DRAM bytes per launch of a kernel from the committed ncu summary, if
    it was taken on the current source of that kernel (else None)."""
    import hashlib
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    rec = json.load(open(p)).get(kernel)
    if not rec:
        return None
    src = os.path.join(ROOT, "paper_2407_21724_gb300", "csrc", rec["source"])
    h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    return rec["dram_bytes_per_launch"] if h == rec["sha"] else None


def train_learned(smr, workloads, n_arrays, dev, n_side=20, width=256, steps=1500, batch=4096, modes=16):
    """Solve n_arrays random n_side x n_side pillar arrays (ragged batches of
    up to 400, one incidence each, FP32-inner refinement to 1e-4), then train the
    MLP on their de-phased coefficients.  Returns parameters and timings."""
    import numpy as np
    import torch
    t0 = time.perf_counter()
    feats, tgts, xs = [], [], []
    arrays = workloads.training_arrays(n_arrays, n=n_side, seed0=100000, modes=modes, shape="pillar")
    chunks = [arrays[i:i + 400] for i in range(0, n_arrays, 400)]
    sols = []
    for ch in chunks:
        ctx = smr.scene_from_arrays(ch)
        nn_ = smr.smr_info(ctx)["n_unknowns"]
        kh = [w["incidences"][0][0] for w in ch]
        pol = [w["incidences"][0][1] for w in ch]
        b = torch.empty(nn_, dtype=torch.complex128, device=dev)
        smr.smr_rhs_plane_waves_arrays(ctx, kh, pol, b)
        x = torch.zeros_like(b)
        smr.smr_solve(ctx, b, x, tol=1e-4, precision=smr.SMR_PREC_FP32, maxit=3000)
        sols.append((ctx, kh, pol, x))
    t_data = time.perf_counter() - t0
    scale = float(torch.sqrt(torch.mean(torch.cat([torch.abs(s[3]) ** 2 for s in sols]))))
    for ctx, kh, pol, x in sols:
        p = smr.smr_info(ctx)["p"]
        smr.smr_nn_init(ctx, width=8, seed=0)          # features need an initialised network
        f = torch.empty((p, 448), dtype=torch.float32, device=dev)
        t = torch.empty((p, 4 * smr.smr_info(ctx)["n_psi"]), dtype=torch.float32, device=dev)
        smr.smr_nn_features(ctx, kh, pol, f)
        smr.smr_nn_targets(ctx, kh, x, scale, t)
        feats.append(f)
        tgts.append(t)
    F = torch.cat(feats)
    T = torch.cat(tgts)
    for ctx, *_ in sols[1:]:
        smr.smr_destroy(ctx)
    ctx = sols[0][0]
    smr.smr_nn_init(ctx, width=width, seed=1)
    rng = np.random.default_rng(0)
    N = F.shape[0]
    torch.cuda.synchronize(dev)
    t1 = time.perf_counter()
    losses = []
    for it in range(steps):
        idx = torch.from_numpy(rng.integers(0, N, size=batch).astype(np.int32)).to(dev)
        lr = 2e-3 if it < steps * 2 // 3 else 5e-4
        losses.append(smr.smr_nn_train_step(ctx, batch, F, T, lr, idx=idx))
    t_train = time.perf_counter() - t1
    params = smr.smr_nn_get_params(ctx)
    smr.smr_destroy(ctx)
    return dict(params=params, scale=scale, width=width, arrays=n_arrays, samples=int(N),
                data_seconds=t_data, train_seconds=t_train, steps=steps, batch=batch,
                loss_first=float(np.mean(losses[:20])), loss_last=float(np.mean(losses[-20:])))


def focal_report(smr, ctx, x, w, dev):
    """Total-field intensity |E_inc + E_s|^2 of the solved lens on its axis,
    z in [0.2 f, 1.8 f] (161 points), and on the line x in [-5, 5] at the
    intended focal plane z = f (201 points); near field by direct surface
    quadrature of the solved currents."""
    import numpy as np
    import torch
    f = w["focal"]
    z = np.linspace(0.2 * f, 1.8 * f, 161)
    xs = np.linspace(-5.0, 5.0, 201)
    pts = np.concatenate([np.stack([0 * z, 0 * z, z], 1), np.stack([xs, 0 * xs, f + 0 * xs], 1)])
    EH = torch.empty(len(pts) * 6, dtype=torch.complex128, device=dev)
    t0 = time.perf_counter()
    smr.smr_near_field(ctx, x, pts, EH)
    torch.cuda.synchronize(dev)
    t = time.perf_counter() - t0
    E = EH.cpu().numpy().reshape(-1, 6)[:, :3]
    k = 2 * np.pi
    kh, pol = w["incidences"][0]
    E = E + np.outer(np.exp(-1j * k * (pts @ kh)), pol)
    I = np.sum(np.abs(E) ** 2, axis=1)
    Iz, Ix = I[:161], I[161:]
    half = Ix >= 0.5 * Ix.max()
    return dict(z_peak=float(z[np.argmax(Iz)]), focal_length=f, peak_intensity=float(Iz.max()),
                fwhm_x=float(xs[half].max() - xs[half].min()), points=int(len(pts)), seconds=t)


def combine_ranks(ms_total, world, R, steps, device):
    """Replicas: the slowest rank's time over the units all ranks processed.
    Returns (max over ranks of ms_total, whole-job products per second)."""
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([ms_total], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_total = float(t.item())
        dist.barrier()
    return ms_total, world * R * steps / (ms_total / 1e3)


def run_ours(a):
    import numpy as np
    import torch
    import torch.distributed as dist
    from paper_2407_21724_gb300 import smr, workloads

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    name, kw = WORKLOADS[a.workload]
    t0 = time.perf_counter()
    if a.workload == "ragged16":
        ws = workloads.make(name, **kw)
        w = dict(label="ragged batch of 16 random arrays, 10x10 ... 60x60, one product",
                 pitch=ws[0]["pitch"])
        ctx = smr.scene_from_arrays(ws, device=local)
        incs = [(v["incidences"][0][0], v["incidences"][0][1]) for v in ws]
    else:
        w = workloads.make(name, **kw)
        ctx = smr.scene_from_workload(w, device=local)
        incs = [w["incidences"][0]]
    setup_s = time.perf_counter() - t0
    R = 64 if a.workload == "batched100x64" else 1
    t1 = time.perf_counter()
    # launch variants for this scene, timed on single-column products (columns
    # of a batched FP32 product run through the same kernels), and for R > 1
    # the number of columns in flight
    smr.smr_autotune(ctx, smr.SMR_PREC_FP32, R=R)
    tune_s = time.perf_counter() - t1
    info = smr.smr_info(ctx)
    n = info["n_unknowns"]
    st = torch.cuda.current_stream(dev)
    if R > 1:
        grid = workloads.incidence_grid64()
        b = torch.empty(n * R, dtype=torch.complex128, device=dev)
        smr.smr_rhs_plane_waves(ctx, [k for k, _ in grid], [q for _, q in grid], b)
    else:
        b = torch.empty(n, dtype=torch.complex128, device=dev)
        smr.smr_rhs_plane_waves_arrays(ctx, [k for k, _ in incs], [q for _, q in incs], b)
    rng = np.random.default_rng(rank)
    x = torch.from_numpy(rng.standard_normal(n * R) + 1j * rng.standard_normal(n * R)).to(dev)
    y = torch.empty_like(x)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)   # 256 MB > 129 MB L2
    P32 = smr.SMR_PREC_FP32

    def timed(prec, steps, warmup, graph=True):
        mv = smr.smr_matvec_graph if graph else smr.smr_matvec
        for _ in range(warmup):
            mv(ctx, x, y, prec)
        torch.cuda.synchronize(dev)
        evs = []
        for _ in range(steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            mv(ctx, x, y, prec)
            e1.record(st)
            evs.append((e0, e1))
        torch.cuda.synchronize(dev)
        return sum(e0.elapsed_time(e1) for e0, e1 in evs)

    # ---- timed region: K tuned products
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    cproc, cf = clocks_start(os.path.join(ROOT, f".clocks_{rank}.csv")) if rank == 0 else (None, None)
    ms_total = timed(P32, a.steps, max(3, a.warmup))
    clocks = clocks_stop(cproc, cf, os.path.join(ROOT, f".clocks_{rank}.csv"), local) if rank == 0 else None
    if cf is not None and os.path.exists(os.path.join(ROOT, f".clocks_{rank}.csv")):
        os.remove(os.path.join(ROOT, f".clocks_{rank}.csv"))
    torch.cuda.synchronize(dev)
    ms_total, value = combine_ranks(ms_total, world, R, a.steps, dev)
    ms_step = ms_total / a.steps

    # ---- the same products launched kernel by kernel (no graph)
    ms_direct = timed(P32, max(3, a.steps // 4), 2, graph=False) / max(3, a.steps // 4)

    # ---- plain FP64 products (same protocol, fewer steps)
    k64 = max(3, a.steps // 4)
    ms64 = timed(smr.SMR_PREC_FP64, k64, 2) / k64 / R

    # ---- error of the tuned (FP32) product against the FP64 product, whose
    # agreement with the FP64 oracle is the tested parity bar (<= 1e-10)
    def prod(v, prec):
        out = torch.empty_like(v)
        smr.smr_matvec(ctx, v, out, prec)
        torch.cuda.synchronize(dev)
        return out

    def relerr(u, v):
        return float(torch.linalg.vector_norm(u - v) / torch.linalg.vector_norm(v))

    errors = dict(reference="the FP64 GPU product / solution (the FP64 product equals the FP64 "
                            "oracle's to <= 1e-10 in the parity tests)",
                  product_random_x=relerr(prod(x, P32), prod(x, smr.SMR_PREC_FP64)),
                  product_x_eq_b=relerr(prod(b, P32), prod(b, smr.SMR_PREC_FP64)))

    # ---- per-launch profile of the tuned product (CUDA events around every launch)
    prof_runs = [smr.smr_profile_matvec(ctx, x, y, P32) for _ in range(max(3, a.steps // 4))]
    nr = len(prof_runs)
    names, launch = {}, {}
    for run in prof_runs:
        for rec in run:
            for key, tab in ((rec["name"], names), ("%s:%d" % (rec["name"], rec["level"]), launch)):
                d = tab.setdefault(key, dict(ms=0.0, bytes=0.0, flops=0.0, launches=0.0))
                d["ms"] += rec["ms"] / nr
                d["bytes"] += rec["bytes"] / nr
                d["flops"] += rec["flops"] / nr
                d["launches"] += 1.0 / nr
    tot = sum(d["ms"] for d in names.values())
    # dominant kernel launch: the (kernel, level) with the largest share of the step
    top = max(launch, key=lambda k: launch[k]["ms"])
    d = launch[top]
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) \
        if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    hbm = peaks.get("hbm_gbs", 6800.0)
    # CUDA-core peaks measured on this device (FP32 scalar and packed FMA, FP64 FMA)
    alu_peaks = {}
    for kind, key in ((0, "fp32_fma"), (1, "fp32x2_fma"), (2, "fp64_fma")):
        try:
            alu_peaks[key] = round(smr.smr_measure_peak(kind), 2)
        except smr.SmrError:
            pass
    fp32_peak = max(alu_peaks.get("fp32_fma", 0.0), alu_peaks.get("fp32x2_fma", 0.0))
    # the bound is the roof the launch would hit first: its FP32 flops at the
    # FP32 peak against its bytes at the HBM peak (the per-pair near blocks
    # of displaced scenes make the near product HBM-bound)
    alu_first = (top.split(":")[0] in ALU_BOUND and
                 d["flops"] / ((fp32_peak or FP32_PEAK_TFLOPS) * 1e12) > d["bytes"] / (hbm * 1e9))
    if alu_first:
        # dense per-particle contractions on the FP32 pipes: against the
        # measured FP32 CUDA-core peak (else 152 SMs x 128 lanes x 2 flop x 2.07 GHz)
        ach = d["flops"] / d["ms"] / 1e9
        pk = fp32_peak or FP32_PEAK_TFLOPS
        roofline = dict(kernel=top, bound="alu", achieved=ach, peak=pk, unit="TFLOP/s", frac=ach / pk,
                        peak_source="measured (smr_measure_peak, FP32 FMA)" if fp32_peak else
                        "derived: 152 SMs x 128 FP32 lanes x 2 flop x 2070 MHz",
                        hbm_GBps=d["bytes"] / d["ms"] / 1e6)
    else:
        ach = d["bytes"] / d["ms"] / 1e6
        roofline = dict(kernel=top, bound="hbm", achieved=ach, peak=hbm, unit="GB/s", frac=ach / hbm,
                        peak_source="measured (MEASURED_PEAKS.json hbm_gbs)" if "hbm_gbs" in peaks
                        else "fallback 6800 GB/s")
    roofline.update(traffic=traffic_for(top), algorithmic_bytes_per_launch=d["bytes"],
                    algorithmic_flops_per_launch=d["flops"], launch_ms=d["ms"], share_of_step=d["ms"] / tot,
                    alu_peaks_measured_tflops=alu_peaks)
    breakdown = {k: dict(ms=round(v["ms"], 4), share=round(v["ms"] / tot, 4), launches=round(v["launches"]),
                         GBps=round(v["bytes"] / v["ms"] / 1e6, 1),
                         TFLOPs=round(v["flops"] / v["ms"] / 1e9, 2)) for k, v in names.items()}
    launches = len(prof_runs[0])

    # ---- end to end through the C ABI with host buffers (copies timed)
    xh = torch.from_numpy(rng.standard_normal(n * R) + 1j * rng.standard_normal(n * R)).pin_memory()
    yh = torch.empty_like(xh).pin_memory()
    xa, ya = xh.numpy(), yh.numpy()
    lib = smr.lib()
    import ctypes as C
    D = C.POINTER(C.c_double)
    px, py = xa.ctypes.data_as(D), ya.ctypes.data_as(D)
    for _ in range(2):
        lib.smr_matvec_host(ctx, R, px, py, P32, st.cuda_stream)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    ke = max(3, a.steps // 2)
    for _ in range(ke):
        rc = lib.smr_matvec_host(ctx, R, px, py, P32, st.cuda_stream)
        assert rc == 0
    e2e_s = (time.perf_counter() - t0) / ke / R

    # ---- GMRES to 1e-4 (tuned, tuned + learned initial guess, plain FP64)
    gm = None
    if not a.no_solve:
        gm = {}
        learned = None
        if a.train_arrays > 0 and R == 1:
            # training arrays carry the workload's modes per current (N_perp = N_par)
            learned = train_learned(smr, workloads, a.train_arrays, dev, modes=info["n_psi"] // 2)

        def solve(label, prec, x0=None, lpc=False, extra_opts=None):
            xs = torch.zeros_like(b) if x0 is None else x0.clone()
            torch.cuda.synchronize(dev)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            extra = dict(extra_opts or {})
            if x0 is not None:
                # the guess is part of the solve: features + network + re-phasing
                smr.smr_nn_predict(ctx, [k for k, _ in incs], [q for _, q in incs], learned["scale"], xs)
                extra["use_x0"] = 1
            if lpc:
                # learned local-coupling preconditioner, built inside the timed solve
                smr.smr_nn_precond(ctx, [k for k, _ in incs], [q for _, q in incs], learned["scale"], b)
                extra["precond"] = smr.SMR_PRECOND_LEARNED
            # the learned preconditioner is an ablation arm; if it has not cut
            # the residual tenfold in 40 iterations the solver falls back to
            # the block-diagonal one (reported as fallback_precond)
            rc, stt = smr.smr_solve(ctx, b, xs, R=R, tol=1e-4, precision=prec, maxit=3000, **extra)
            e1.record(st)
            torch.cuda.synchronize(dev)
            stt["solver_seconds"] = stt.pop("seconds")
            gm[label] = dict(seconds=e0.elapsed_time(e1) / 1e3, converged=(rc == 0), **stt)
            return xs

        xt = solve("tuned_fp32_inner_fp64_outer", P32)
        sols = dict(tuned=xt)
        # the tuned solver restarted every 200 iterations: more iterations, far
        # less Gram-Schmidt (the unrestarted basis costs as much as the products)
        sols["tuned_restart"] = solve("tuned_restart200", P32, extra_opts=dict(restart=200))
        if "focal" in w and R == 1:
            gm["focal"] = focal_report(smr, ctx, xt, w, dev)
        if learned is not None:
            smr.smr_nn_init(ctx, width=learned["width"], seed=0)
            smr.smr_nn_set_params(ctx, learned["params"])
            solve("tuned_plus_learned_x0", P32, x0=torch.zeros_like(b))
            solve("tuned_plus_learned_x0_and_precond", P32, x0=torch.zeros_like(b), lpc=True)
            gm["learned_training"] = {k: v for k, v in learned.items() if k not in ("params",)}
        sols["fp64"] = solve("plain_fp64", smr.SMR_PREC_FP64)
        # the tuned solution and its far field against the plain FP64 solve
        errors["solution_tuned_vs_fp64"] = relerr(sols["tuned"], sols["fp64"])
        errors["solution_tuned_restart_vs_fp64"] = relerr(sols["tuned_restart"], sols["fp64"])
        th, ph = np.meshgrid(np.radians(np.linspace(5.0, 175.0, 8)), np.radians(np.arange(8) * 45.0),
                             indexing="ij")
        dirs = np.stack([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)], -1).reshape(-1, 3)
        ff = {}
        for key, v in sols.items():
            F = torch.empty(len(dirs) * 3 * R, dtype=torch.complex128, device=dev)
            smr.smr_far_field(ctx, v, dirs, F, R=R)
            torch.cuda.synchronize(dev)
            ff[key] = F
        errors["far_field_tuned_vs_fp64"] = relerr(ff["tuned"], ff["fp64"])
        errors["far_field_directions"] = "64: theta in linspace(5, 175 deg, 8) x phi in 0, 45, ..., 315 deg"
        errors["solve_tolerance"] = "both solves stop at a true FP64 relative residual of 1e-4"
        best = min(v["seconds"] for k, v in gm.items() if k.startswith("tuned") and isinstance(v, dict)
                   and "seconds" in v)
        gm["speedup_tuned_vs_plain"] = gm["plain_fp64"]["seconds"] / best

    # ---- CPU oracle baseline on a bounded sample (rank 0, N = 1 only)
    cpu = None
    if rank == 0 and world == 1 and not a.no_cpu:
        env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
        cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "2",
               "--warmup", "1", "--workload", a.workload]
        r = subprocess.run(cmd, capture_output=True, text=True, env=env)
        for line in r.stdout.splitlines():
            if line.startswith("{"):
                cpu = json.loads(line)["cpu_baseline"]
        if cpu and gm and "plain_fp64" in gm and cpu.get("value"):
            # the oracle cannot run the full solve here: its GMRES time is the
            # extrapolation (plain GPU iteration count + 1) x oracle time per product
            it = gm["plain_fp64"]["iters"] + 1
            cpu["gmres_seconds_extrapolated"] = it * R / cpu["value"]
            cpu["gmres_extrapolation"] = f"{it} products (the plain FP64 solve's count) x oracle seconds per product"
    smr.smr_destroy(ctx)
    if rank == 0:
        line = dict(metric=METRIC, value=value, unit="matvecs/s", n_gpus=world, steps=a.steps,
                    warmup=a.warmup, ms_per_step=ms_step, higher_is_better=True, scaling="weak",
                    vs_baseline=None, dtype="f32", data="synthetic",
                    config=dict(workload=w["label"], rhs=R, precision="FP32 product, FP64 tables/IO",
                                l2="L2 flushed (256 MB write) before every timed step",
                                parallelism="replicas" if world > 1 else "single GPU",
                                levels=info["n_levels"], L=info["L"], unknowns=n,
                                column_lanes=info["column_lanes"] if R > 1 else 1),
                    fp64_matvecs_per_s=1e3 / ms64, fp64_ms_per_matvec=ms64,
                    ms_per_step_without_graph=ms_direct / R,
                    gmres=gm, errors_vs_fp64=errors, setup_s=setup_s, autotune_s=tune_s,
                    e2e=dict(value=1.0 / e2e_s, unit="matvecs/s", h2d_bytes_per_step=16 * n * R,
                             d2h_bytes_per_step=16 * n * R),
                    gpu_launches=launches * a.steps, roofline=roofline, kernels=breakdown,
                    launches_ms={k: round(v["ms"], 4) for k, v in launch.items()},
                    clocks=clocks, cpu_baseline=cpu)
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)
