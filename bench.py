"""SRWCR value+gradient throughput on B300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--config c2|c1|c3|c5] [--storage f32|bf16]

A step is one full value+gradient pass (fused warp/statistics kernel,
FP64 finalisation, adjoint) over the 256x256x96 CT-shaped pair (default),
inputs resident in HBM, through srwcr_value_and_grad_async with the same
buffers every step (the library replays the call from its CUDA graph).  The
L2 is flushed (256 MB write) between steps, outside the timed events.  Under torchrun every rank runs its own replica
(weak scaling, no collective on the data path); the timed region is
bracketed by a barrier and synchronisation and the max over ranks is used.

--impl reference times the FP64 CPU oracle on the host cores on a bounded
sample of the same workload (a slab of the volume).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

CONFIG_NAMES = {"c1": "c1_2d_128", "c2": "c2_ct_256x256x96", "c3": "c3_oct_160",
                "c5": "c5_ct_512x512x300"}
METRIC = "SRWCR value+grad Gvoxel/s & HBM-roofline % at 256²×96; batched vs plain pairs/s"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
# The sources of the row kernels the committed ncu counters describe (the
# counters are used only while these files hash the same).
KERNEL_SOURCES = ["paper_1804_05061_b300/csrc/kernels_rows.cuh",
                  "paper_1804_05061_b300/csrc/device_math.cuh"]


def kernel_hash() -> str:
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def hbm_peak():
    try:
        with open(PEAKS_FILE) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(t: float, dist, device) -> float:
    """The slowest rank's time (every rank gets it); t itself without a
    process group.  device: where the collective's tensor lives (a CUDA
    device under NCCL, "cpu" under gloo)."""
    if dist is None:
        return t
    import torch
    tt = torch.tensor([t], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


def whole_job_rate(ws: int, units_per_rank: float, seconds: float) -> float:
    """Replicas: every rank processes the same units, so the job's rate is
    ws * units / (the slowest rank's time)."""
    return ws * units_per_rank / seconds


class Clocks:
    """nvidia-smi sampling of SM clock and throttle reasons during a region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["active", "hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown",
                 "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names[1:], parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


def host_info():
    """Host cores and CPU model (the CPU baseline runs here)."""
    model = None
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    return {"nproc": os.cpu_count(), "cpu_model": model}


def oracle_full_eval(pair, c, storage="f32"):
    """FP64 oracle value+gradient of the whole workload at c on one host
    core: seconds, D, gradient, and the degenerate regions (count, summed
    p(r))."""
    import oracle
    prob = pair.prob
    geo = oracle.Geometry.from_problem(prob)
    A, M = oracle.prepare(pair.fixed, pair.moving, prob.n_bins, storage)
    t = time.perf_counter()
    st = oracle.value(geo, A, M, c)
    g = oracle.gradient(geo, A, M, c, st)
    dt = time.perf_counter() - t
    deg = st.valid == 0
    return {"seconds": dt, "D": float(st.D), "g": np.asarray(g, np.float64).ravel(),
            "n_degenerate": int(st.n_degenerate), "degenerate_p_mass": float(st.pr[deg].sum())}


def workload_text(pair):
    """What the workload is: image shape, content, FFD spacing, spatial and
    intensity bins."""
    prob = pair.prob
    kind = {"c1": "2-D ellipse phantom pair", "c2": "CT-shaped pair", "c3": "OCT-shaped pair (speckled layers)",
            "c5": "CT-shaped pair"}.get(pair.name[:2], "pair")
    shape = "x".join(str(d) for d in prob.dims[:prob.ndim])
    sb = prob.sbin_intervals[:prob.ndim]
    bins = "spatial bins on the FFD grid" if not any(sb) else f"spatial bins {tuple(sb)} intervals"
    return (f"{shape} {kind}, FFD spacing {prob.ffd_spacing[0]}, {bins}, "
            f"{prob.n_bins} intensity bins")


def slab(pair, nz):
    """Sub-volume (the middle nz slices) as a bounded sample of a 3-D
    workload."""
    prob = pair.prob
    if prob.ndim == 2:
        return pair
    z0 = (prob.dims[2] - nz) // 2
    p2 = synth.problem(3, (prob.dims[0], prob.dims[1], nz), prob.ffd_spacing,
                       prob.sbin_intervals, prob.n_bins)
    return synth.PairSpec(pair.name + f"_slab{nz}", p2,
                          np.ascontiguousarray(pair.fixed[z0:z0 + nz]),
                          np.ascontiguousarray(pair.moving[z0:z0 + nz]))


def _oracle_slab_job(job):
    """One oracle value+gradient of a slab sample (worker process)."""
    fixed, moving, dims, spacing, sbins, nbins, storage, seed = job
    import oracle
    prob = synth.problem(3, dims, spacing, sbins, nbins)
    c = synth.coefficients(prob, seed, 2.0)
    geo = oracle.Geometry.from_problem(prob)
    A, M = oracle.prepare(fixed, moving, nbins, storage)
    t = time.perf_counter()
    st = oracle.value(geo, A, M, c)
    oracle.gradient(geo, A, M, c, st)
    return time.perf_counter() - t


class OraclePool:
    """All host cores: one spawned process per core, each evaluating the
    same bounded slab sample with the unchanged single-threaded oracle."""

    def __init__(self, sample, storage, procs=None):
        import multiprocessing as mp
        import oracle
        oracle.build()
        self.procs = procs or os.cpu_count() or 1
        prob = sample.prob
        self.job = (sample.fixed, sample.moving, tuple(prob.dims), tuple(prob.ffd_spacing),
                    tuple(prob.sbin_intervals), prob.n_bins, storage, 2001)
        self.voxels = prob.n_voxels
        self.pool = mp.get_context("spawn").Pool(self.procs)

    def step(self):
        """Wall seconds of one round: every process evaluates the sample once."""
        t = time.perf_counter()
        self.pool.map(_oracle_slab_job, [self.job] * self.procs, chunksize=1)
        return time.perf_counter() - t

    def close(self):
        self.pool.close()
        self.pool.join()


def accuracy(D, g, D_ref, g_ref):
    """Relative errors of a GPU result against the FP64 oracle's."""
    g = np.asarray(g, np.float64).ravel()
    gn, gn_ref = float(np.linalg.norm(g)), float(np.linalg.norm(g_ref))
    return {"D_rel": abs(D - D_ref) / abs(D_ref), "gnorm_rel": abs(gn - gn_ref) / gn_ref,
            "g_max_elem_rel": float(np.abs(g - g_ref).max() / np.abs(g_ref).max()),
            "D": D, "D_oracle": D_ref}


def run_reference(args, pair, c_full):
    """The oracle on every host core: each step is one round in which every
    process evaluates value+gradient of the same 256x256x8 slab sample."""
    ws, rank, _ = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
        if rank != 0:
            dist.barrier()
            return
    sample = slab(pair, 8)
    prob = sample.prob
    pool = OraclePool(sample, args.storage)
    for _ in range(args.warmup):
        pool.step()
    dt = sum(pool.step() for _ in range(args.steps))
    pool.close()
    v = pool.procs * prob.n_voxels * args.steps / dt / 1e9
    host = host_info()
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "Gvoxel/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"{pair.name} ({pair.prob.dims[0]}x{pair.prob.dims[1]}x"
                       f"{pair.prob.dims[2]}, {pair.prob.n_bins} bins); reference steps run on "
                       f"a {prob.dims[0]}x{prob.dims[1]}x{prob.dims[2]} slab",
                       "storage": args.storage},
            "cpu_baseline": {"value": v, "unit": "Gvoxel/s", "cores": pool.procs, "kind": "oracle",
                             "host": host,
                             "sample": f"{pool.procs} processes (one per host core), each one "
                             f"value+gradient of the {prob.dims} slab per step, {args.steps} steps"},
            "e2e": {"value": v, "unit": "Gvoxel/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def bench_batch(args, eng, torch, dist, ws):
    """Batched form on the 32-pair PET/CT-shaped batch (BF16 storage): pairs/s
    of value+gradient for the plain per-pair loop, one launch per phase over
    all (pair, tile) items, and the same replayed from a CUDA graph; then
    L-BFGS iterations/s of the per-pair driver against the batched,
    graph-replayed one.  The batch's images (about 350 MB in BF16) exceed
    the L2, so no flush is needed between steps."""
    specs = synth.batch_specs(args.batch_pairs)
    engines = [eng.from_problem(s.prob, s.fixed, s.moving, storage="bf16") for s in specs]
    cs = [torch.from_numpy(synth.coefficients(s.prob, 7000 + i, 2.0)).cuda()
          for i, s in enumerate(specs)]
    tiles = [e.autotune(c, reps=2) for e, c in zip(engines, cs)]
    b = eng.Batch(engines)
    for i, c in enumerate(cs):
        b.coef(i).copy_(c)
    n = len(engines)
    gs = [torch.empty_like(c) for c in cs]
    Ds = torch.empty(n, dtype=torch.float64, device=cs[0].device)
    cur = torch.cuda.current_stream()
    steps = max(3, min(args.steps, 20))

    def timed(fn, stream):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        s0 = torch.cuda.Event(enable_timing=True)
        s1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.profiler.start()
        s0.record(stream)
        for _ in range(steps):
            fn()
        s1.record(stream)
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
        return max_over_ranks(s0.elapsed_time(s1) / 1e3, dist, cs[0].device)

    def plain():
        for i, e in enumerate(engines):
            e.value_and_grad_async(cs[i], Ds[i], gs[i])

    t_plain = timed(plain, cur)
    D_plain = Ds.cpu().numpy().copy()
    # The batch stream is ordered after the current stream on entry; its
    # events are recorded on the batch stream itself.
    t_eager = timed(lambda: b.value_and_grad_async(use_graph=False), b.stream)
    t_graph = timed(lambda: b.value_and_grad_async(use_graph=True), b.stream)
    D_batch = b.values()
    launches = b.info().launches_per_eval
    # Error of every pair's batched result against the FP64 oracle values
    # stored for these pairs and coefficients (tests/golden, written from the
    # oracle alone); the worst pair is reported.
    worst = None
    gold_path = os.path.join(ROOT, "tests", "golden", "full_size_oracle.json")
    if os.path.exists(gold_path):
        gold = json.load(open(gold_path))["cases"]
        errs = []
        for i in range(n):
            ref = gold.get(f"c4_pair{i:02d}")
            if ref is None or ref.get("coef_seed") != 7000 + i or list(specs[i].prob.dims) != ref["dims"]:
                continue
            gi = b.grad(i).detach().cpu().numpy().ravel().astype(np.float64)
            errs.append({"pair": i, "D_rel": abs(D_batch[i] - ref["D"]) / abs(ref["D"]),
                         "gnorm_rel": abs(float(np.linalg.norm(gi)) - ref["gnorm"]) / ref["gnorm"]})
        if errs:
            worst = {"pairs_checked": len(errs),
                     "worst_D_rel": max(errs, key=lambda r: r["D_rel"]),
                     "worst_gnorm_rel": max(errs, key=lambda r: r["gnorm_rel"]),
                     "reference": "FP64 oracle on the BF16-rounded inputs (stored)"}

    # L-BFGS: per-pair host-driven driver vs batched, graph-replayed rounds.
    o = eng.SRWCR.default_opts()
    o.max_iter[0] = args.batch_lbfgs_iters
    o.stable_window = 0
    x0 = [torch.zeros_like(c) for c in cs]
    torch.cuda.synchronize()
    tp = time.perf_counter()
    it_plain = 0
    f_plain = []
    for e, x in zip(engines, x0):
        r = e.register(x, 1, o)
        it_plain += r.iterations[0]
        f_plain.append(r.final_value[0])
    torch.cuda.synchronize()
    tp = time.perf_counter() - tp
    for i in range(n):
        b.coef(i).zero_()
    b.register(o, use_graph=True)            # captures the round graph
    for i in range(n):
        b.coef(i).zero_()
    torch.cuda.synchronize()
    tb = time.perf_counter()
    rep = b.register(o, use_graph=True)
    tb = time.perf_counter() - tb
    it_b = int(rep["iterations"].sum())
    f_b = rep["final_value"]
    rel = [abs(a - c) / abs(c) for a, c in zip(f_b, f_plain)]
    vox = sum(s.prob.n_voxels for s in specs)
    return {
        "workload": f"{n} PET/CT-shaped pairs, cube edges "
                    f"{sorted(set(s.prob.dims[0] for s in specs))} (counts "
                    f"{[sum(1 for s in specs if s.prob.dims[0] == e) for e in sorted(set(s.prob.dims[0] for s in specs))]}), "
                    f"{vox} voxels in all, FFD spacing 8, spatial bins on the FFD grid, 32 "
                    "intensity bins, BF16 storage, autotuned tiles",
        "metric": "pairs/s (value+gradient of every pair)",
        "plain_pairs_per_s": whole_job_rate(ws, n * steps, t_plain),
        "batched_pairs_per_s": whole_job_rate(ws, n * steps, t_eager),
        "graph_pairs_per_s": whole_job_rate(ws, n * steps, t_graph),
        "graph_vs_plain": t_plain / t_graph,
        "batched_gvoxel_per_s": whole_job_rate(ws, vox * steps, t_graph) / 1e9,
        "launches_per_eval_batched": launches,
        "launches_per_eval_plain": 6 * n,
        "max_abs_D_diff_batched_vs_plain": float(np.abs(D_batch - D_plain).max()),
        "accuracy_vs_oracle": worst,
        "tiles": sorted(set(tuple(t) for t in tiles)),
        "steps": steps,
        "lbfgs": {"iterations_per_pair": args.batch_lbfgs_iters,
                  "plain_iters_per_s": it_plain / tp, "batched_graph_iters_per_s": it_b / tb,
                  "speedup": (it_b / tb) / (it_plain / tp) if it_plain else None,
                  "max_rel_final_value_diff": float(max(rel)),
                  "note": "plain = srwcr_register per pair (host-driven line search); "
                          "batched = device-resident L-BFGS rounds replayed from a CUDA graph; "
                          "wall clock including host checks"},
    }


def bench_registration(eng, torch, pair):
    """The 256x256x96 pair registered coarse to fine over a 3-level pyramid
    (levels 64x64x24, 128x128x48, 256x256x96; default L-BFGS options: at most
    200/200/120 iterations, stop when D is stable over 20 steps), from zero
    coefficients.  Wall clock of srwcr_register (host-driven line search)."""
    prob = pair.prob
    e = eng.from_problem(prob, pair.fixed, pair.moving, storage="f32", pyramid_levels=3)
    for lvl in range(3):
        e.autotune(e.zeros(lvl), level=lvl, reps=2)
    c = e.zeros()
    D0 = e.value(c)
    o = e.default_opts()
    torch.cuda.synchronize()
    t = time.perf_counter()
    rep = e.register(c, 3, o)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t
    its = [int(rep.iterations[l]) for l in (2, 1, 0)]
    evs = [int(rep.evaluations[l]) for l in (2, 1, 0)]
    names = {0: "SRWCR_OK", 5: "SRWCR_ELINESEARCH", 7: "SRWCR_ENOTCONVERGED"}
    return {"workload": f"{pair.name}, 3-level pyramid, coarse to fine, from zero coefficients",
            "levels": [list(e.levels[l].dims) for l in (2, 1, 0)],
            "iterations": its, "evaluations": evs,
            "final_value": [float(rep.final_value[l]) for l in (2, 1, 0)],
            "status": [names.get(int(rep.status[l]), int(rep.status[l])) for l in (2, 1, 0)],
            "D_start_finest": D0, "D_end_finest": e.value(c), "wall_s": wall,
            "iterations_per_s": sum(its) / wall}


def bench_accuracy(eng, torch):
    """Synthetic-grid accuracy run (Sec. III-A, Table II): a 128^3 binary grid O
    and a warped copy W(x) = O(x + v(x)) under a smooth bias field, v a cubic
    B-spline field with control displacements uniform in [-15, 15] voxels
    (spacing 16).  3-level pyramid, FFD spacing 5, spatial bins on the FFD
    grid, 32 bins, default L-BFGS options with the coarsest level started
    off the lattice (start_jitter 0.5 voxel: the identity samples the binary
    moving image at the lattice, where every voxel sits at a kink of the
    Parzen window).  The four combinations of Table II (paper: its means over
    ten cases, its own warp spacing and bias field), plus the paper's best
    one started at the identity.  RMSE over the whole volume; the recovered
    displacement is v when O moves and the inverse of v when W moves."""
    import numpy as np
    g = synth.grid_pair(seed=0)
    n = g.original.shape[0]
    prob = synth.problem(3, (n, n, n), (5, 5, 5), (0, 0, 0), 32)
    v = synth.displacement_field(g.original.shape, g.true_spacing, g.true_coef)
    w = synth.inverse_displacement(v)
    rms = lambda a: float(np.sqrt(np.mean(np.sum(a ** 2, axis=0))))
    out = {"workload": "128^3 binary grid vs. its B-spline-warped, bias-field copy (seed 0)",
           "start_jitter_voxels": 0.5}
    for key, role, fixed, moving, truth, paper, jitter in (
            ("m_as_b_w_as_moving", "mas_b", g.original, g.warped, w, 1.89, 0.5),
            ("m_as_b_o_as_moving", "mas_b", g.warped, g.original, v, 1.00, 0.5),
            ("m_as_a_w_as_moving", "mas_a", g.original, g.warped, w, 1.70, 0.5),
            ("m_as_a_o_as_moving", "mas_a", g.warped, g.original, v, 0.78, 0.5),
            ("m_as_a_o_as_moving_identity_start", "mas_a", g.warped, g.original, v, 0.78, 0.0)):
        e = eng.from_problem(prob, fixed, moving, role=role, pyramid_levels=3)
        c = e.zeros()
        o = e.default_opts()
        o.start_jitter = jitter
        o.seed = 1
        torch.cuda.synchronize()
        t = time.perf_counter()
        rep = e.register(c, 3, o)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t
        u = synth.displacement_field(g.original.shape, (5, 5, 5), c.cpu().numpy())
        out[key] = {"rmse_initial_voxels": rms(truth), "rmse_final_voxels": rms(u - truth),
                    "paper_table_ii_final": paper,
                    "iterations": [int(rep.iterations[l]) for l in (2, 1, 0)],
                    "kernel_path": [int(e.levels[l].kernel_path) for l in (2, 1, 0)],
                    "wall_s": wall}
        e.close()
    return out


def bench_rigid(eng, torch, prob):
    """Rigid pre-alignment (Sec. III-D): a 256x256x96 CT-shaped phantom and a
    copy moved by a known rigid transform (translation in voxels, extrinsic
    x-y-z Euler angles in radians) with inverted contrast (a multi-modal
    pair), the workload's bins and FFD spacing, 3 pyramid levels.  Reports
    the device time of one rigid value+gradient at the finest level (general
    per-voxel kernels), the 3-level rigid L-BFGS wall time and the parameter
    errors."""
    import numpy as np
    mu_true = [4.0, -3.0, 2.0, 0.04, -0.03, 0.07]
    dims = tuple(prob.dims[:prob.ndim])
    f, m = synth.rigid_pair("ct", dims, mu_true, 11)
    e = eng.from_problem(prob, f, m, pyramid_levels=3)
    mu = torch.zeros(6, dtype=torch.float32, device=e.device)
    for _ in range(3):
        e.rigid_value_and_grad(mu)
    reps = 10
    torch.cuda.synchronize()
    s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s0.record(e.stream)
    for _ in range(reps):
        e.rigid_value_and_grad(mu)
    s1.record(e.stream)
    torch.cuda.synchronize()
    ms = s0.elapsed_time(s1) / reps
    o = e.default_opts()
    torch.cuda.synchronize()
    t = time.perf_counter()
    mu_est, rep = e.rigid_register(mu, 3, o)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t
    mu_est = mu_est.cpu().numpy()
    return {"workload": f"{dims[0]}x{dims[1]}x{dims[2]} CT phantom vs. rigidly moved, "
                        "contrast-inverted copy (seed 11)",
            "mu_true": mu_true, "mu_found": [float(v) for v in mu_est],
            "translation_error_voxels": float(np.abs(mu_est[:3] - mu_true[:3]).max()),
            "angle_error_rad": float(np.abs(mu_est[3:] - mu_true[3:]).max()),
            "iterations": [int(rep.iterations[l]) for l in (2, 1, 0)],
            "D_final": float(rep.final_value[0]),
            "value_and_grad_ms": ms, "gvoxel_per_s": prob.n_voxels / ms / 1e6,
            "register_wall_s": wall}


def row_skips(e, c, level=0):
    """Shares of the row kernels' 32-voxel x-rows that skip work at c: the
    value pass skips rows whose warped intensities are all 0 (no moment to
    add), the adjoint rows where the moving image's interpolated gradient is
    0 at every voxel (computed from srwcr_debug_warp_grad)."""
    import torch
    lv = e.levels[level]
    nx, ny, nz = lv.dims
    out = e.debug_warp_grad(c, level).view(nz, ny, nx, 4)
    nxb = (nx + 31) // 32
    pad = torch.zeros((nz, ny, nxb * 32, 4), dtype=out.dtype, device=out.device)
    pad[:, :, :nx] = out
    rows = pad.view(nz, ny, nxb, 32, 4)
    val = (rows[..., 0] == 0).all(-1)
    adj = (rows[..., 1:] == 0).all(-1).all(-1)
    return {"value": float(val.float().mean()), "adjoint": float(adj.float().mean()),
            "rows": int(val.numel())}


def degenerate(e, level=0):
    """Regions the value leaves out (sigma_r^2 at the degenerate threshold or
    p(r) = 0): their count and summed share p(r)."""
    st, nd = e.region_stats(level)
    deg = st[:, 1] == 0.0
    return {"regions": int(nd), "of": int(st.shape[0]), "p_mass": float(st[deg, 0].sum())}


def time_steps(e, c, D, g, steps, warmup, flush, dist, dev, clocks=None):
    """CUDA-event time of `steps` value+gradient calls through
    srwcr_value_and_grad_async with the same buffers (the library replays its
    graph), the L2 flushed before each outside the events; then the
    per-kernel split from a separate pass with the library's events on.
    Returns (slowest rank's seconds, per-kernel ms, launches, wall, clocks)."""
    import torch
    stream = e.stream
    for _ in range(warmup):
        e.value_and_grad_async(c, D, g)
    torch.cuda.synchronize()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    e.profile_read(reset=True)
    if clocks is not None:
        clocks.start()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    torch.cuda.profiler.start()     # no-op unless a profiler waits for it
    t0 = time.perf_counter()
    for k in range(steps):
        flush.zero_()
        starts[k].record(stream)
        e.value_and_grad_async(c, D, g)
        ends[k].record(stream)
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    if dist is not None:
        dist.barrier()
    wall = time.perf_counter() - t0
    clk = clocks.stop() if clocks is not None else None
    _, _, launches = e.profile_read(reset=True)
    step_ms = sum(s_.elapsed_time(t_) for s_, t_ in zip(starts, ends))
    t_dev = max_over_ranks(step_ms / 1e3, dist, dev)
    e.set_profiling(True)
    for _ in range(min(steps, 20)):
        flush.zero_()
        e.value_and_grad_async(c, D, g)
    torch.cuda.synchronize()
    e.set_profiling(False)
    kms, kcnt, _ = e.profile_read(reset=True)
    names = ["accumulate", "finalize", "adjoint"]
    avg = {names[i]: (kms[i] / kcnt[i] if kcnt[i] else 0.0) for i in range(3)}
    return t_dev, avg, launches, wall, clk


def bench_pair_section(eng, torch, pair, storage, c_np, args, flush, dist, dev, ws, oracle_ref):
    """Device-timed value+gradient of another workload or storage type, with
    its error against the FP64 oracle (oracle_ref: a finished
    oracle_full_eval of the same pair, storage and coefficients)."""
    prob = pair.prob
    e = eng.from_problem(prob, pair.fixed, pair.moving, storage=storage)
    c = torch.from_numpy(c_np).to(dev)
    tile = e.autotune(c, reps=5)
    g = torch.empty_like(c)
    D = torch.empty((), dtype=torch.float64, device=dev)
    steps = max(3, min(args.steps, 20))
    t_dev, avg, _, _, _ = time_steps(e, c, D, g, steps, args.warmup, flush, dist, dev)
    out = {"workload": f"{pair.name}: {prob.dims[0]}x{prob.dims[1]}x{prob.dims[2]}, FFD spacing "
                       f"{prob.ffd_spacing[0]}, spatial bins "
                       f"{list(prob.sbin_intervals[:prob.ndim]) if any(prob.sbin_intervals) else 'on the FFD grid'}, "
                       f"{prob.n_bins} intensity bins",
           "storage": storage, "tile": list(tile),
           "value": whole_job_rate(ws, prob.n_voxels * steps, t_dev) / 1e9, "unit": "Gvoxel/s",
           "ms_per_step": t_dev * 1e3 / steps,
           "kernel_ms": {k: round(v, 4) for k, v in avg.items()},
           "rows_skipped": row_skips(e, c), "degenerate": degenerate(e)}
    if oracle_ref is not None:
        Dv, gv = e.value_and_grad(c)
        out["accuracy_vs_oracle"] = accuracy(Dv, gv.cpu().numpy(), oracle_ref["D"], oracle_ref["g"])
        out["degenerate"]["oracle_regions"] = oracle_ref["n_degenerate"]
        out["degenerate"]["oracle_p_mass"] = oracle_ref["degenerate_p_mass"]
    e.close()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="c2", choices=sorted(CONFIG_NAMES))
    ap.add_argument("--storage", default="f32", choices=["f32", "bf16"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-form section")
    ap.add_argument("--batch-pairs", type=int, default=32)
    ap.add_argument("--batch-lbfgs-iters", type=int, default=10)
    ap.add_argument("--no-registration", action="store_true",
                    help="skip the 3-level pyramid registration run")
    ap.add_argument("--no-accuracy", action="store_true",
                    help="skip the synthetic-grid accuracy run")
    ap.add_argument("--no-rigid", action="store_true", help="skip the rigid pre-alignment run")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the other-storage and dense-content (OCT) lines")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    pair = synth.make_pair(CONFIG_NAMES[args.config])
    prob = pair.prob
    c_np = synth.coefficients(prob, 2001, 2.0)
    if args.impl == "reference":
        run_reference(args, pair, c_np)
        return

    ws, rank, local = dist_env()
    # The FP64 oracle evaluations (the CPU baseline and the error of each GPU
    # result) run in spawned worker processes beside the GPU sections; the
    # pool is started before the first CUDA call.
    cpu_jobs = {}
    executor = None
    other = "bf16" if args.storage == "f32" else "f32"
    dense = synth.make_pair(CONFIG_NAMES["c3"]) if args.config != "c3" else None
    c_dense = synth.coefficients(dense.prob, 2003, 2.0) if dense is not None else None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        import concurrent.futures as cf
        import multiprocessing as mp
        import oracle
        oracle.build()
        executor = cf.ProcessPoolExecutor(max_workers=3, mp_context=mp.get_context("spawn"))
        cpu_jobs["main"] = executor.submit(oracle_full_eval, pair, c_np, args.storage)
        if not args.no_extra:
            cpu_jobs["other"] = executor.submit(oracle_full_eval, pair, c_np, other)
            if dense is not None:
                cpu_jobs["dense"] = executor.submit(oracle_full_eval, dense, c_dense, "f32")

    import torch
    import paper_1804_05061_b300 as eng

    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    e = eng.from_problem(prob, pair.fixed, pair.moving, storage=args.storage)
    stream = e.stream
    c = torch.from_numpy(c_np).to(dev)
    tile = e.autotune(c, reps=10)    # more repetitions: a steadier choice between close tiles
    g = torch.empty_like(c)
    D = torch.empty((), dtype=torch.float64, device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MB > L2

    clocks = Clocks(local)
    t_dev, avg, launches, wall, clk = time_steps(e, c, D, g, args.steps, args.warmup, flush,
                                                 dist, dev, clocks)
    step_ms = t_dev * 1e3
    value = whole_job_rate(ws, prob.n_voxels * args.steps, t_dev) / 1e9
    D_gpu = float(D.item())
    g_gpu = g.cpu().numpy().ravel()
    # The same steps with the L2 warm (no flush between them).
    warm0 = torch.cuda.Event(enable_timing=True)
    warm1 = torch.cuda.Event(enable_timing=True)
    warm0.record(stream)
    for _ in range(args.steps):
        e.value_and_grad_async(c, D, g)
    warm1.record(stream)
    torch.cuda.synchronize()
    t_warm = max_over_ranks(warm0.elapsed_time(warm1) / 1e3, dist, dev)
    l2_warm = {"value": whole_job_rate(ws, prob.n_voxels * args.steps, t_warm) / 1e9,
               "unit": "Gvoxel/s", "ms_per_step": t_warm * 1e3 / args.steps}
    e.profile_read(reset=True)
    skips = row_skips(e, c)
    deg = degenerate(e)

    # End to end through the host-buffer entry point: H2D c from pinned host
    # memory, compute, D2H g and D into pinned host memory.
    c_pin = torch.from_numpy(np.ascontiguousarray(c_np.ravel())).pin_memory()
    g_pin = torch.zeros_like(c_pin).pin_memory()
    c_host, g_host = c_pin.numpy(), g_pin.numpy()
    for _ in range(2):
        e.value_and_grad_host(c_host, g_host)
    # Five batches of 40 synchronising calls (about 10 ms each at the
    # 256x256x96 workload).  With a few milliseconds of timed work, a single
    # stall of the machine's host would dominate a batch.  So `value` comes from
    # the median batch, and `mean_value` from all the calls together.
    n_batch, n_call = 5, max(40, args.steps)
    tb = []
    for _ in range(n_batch):
        t0 = time.perf_counter()
        for _ in range(n_call):
            e.value_and_grad_host(c_host, g_host)
        tb.append(time.perf_counter() - t0)
    t_med = max_over_ranks(sorted(tb)[n_batch // 2], dist, dev)
    t_all = max_over_ranks(sum(tb), dist, dev)
    e2e = {"value": whole_job_rate(ws, prob.n_voxels * n_call, t_med) / 1e9, "unit": "Gvoxel/s",
           "h2d_bytes_per_step": int(c_host.nbytes), "d2h_bytes_per_step": int(g_host.nbytes + 8),
           "steps": n_batch * n_call, "batches": n_batch, "calls_per_batch": n_call,
           "mean_value": whole_job_rate(ws, prob.n_voxels * n_batch * n_call, t_all) / 1e9,
           "batch_ms": [round(t * 1e3, 3) for t in tb]}

    # Roofline of the dominant kernel (algorithmic bytes / CUDA-event time).
    esz = 2 if args.storage == "bf16" else 4
    lv = e.levels[0]
    bytes_alg = {
        "accumulate": 2 * esz * lv.n_voxels + 4 * lv.n_params + 16 * lv.n_regions * prob.n_bins,
        "adjoint": 2 * esz * lv.n_voxels + 4 * lv.n_params * 2
                   + 4 * lv.n_regions * (prob.n_bins + 2),
    }
    dom = max(("accumulate", "adjoint"), key=lambda k: avg[k])
    peak, peak_kind = hbm_peak()
    achieved = bytes_alg[dom] / (avg[dom] / 1e3) / 1e9 if avg[dom] > 0 else 0.0
    traffic = None
    warp_inst = None
    prof_file = os.path.join(ROOT, "profiles", f"{dom}_{args.config}_{args.storage}_traffic.json")
    if os.path.exists(prof_file):
        try:
            pj = json.load(open(prof_file))
            if pj.get("kernel_hash") == kernel_hash():
                traffic = pj.get("dram_bytes_per_launch")
                warp_inst = pj.get("warp_instructions")
        except Exception:
            traffic = None
    # The kernel's real limiter is instruction issue (no dense contraction;
    # HBM-light): executed warp-instructions per launch (ncu, same kernel
    # source) over its event time, against 4 schedulers x SMs x max SM clock.
    try:
        sm_mhz = float(json.load(open(PEAKS_FILE))["sm_max_mhz"])
    except Exception:
        sm_mhz = 2032.0
    issue_peak = 4 * torch.cuda.get_device_properties(dev).multi_processor_count * sm_mhz * 1e6
    issue = None
    if warp_inst and avg[dom] > 0:
        rate = warp_inst / (avg[dom] / 1e3)
        issue = {"warp_instructions_per_launch": warp_inst, "achieved_per_s": rate,
                 "peak_per_s": issue_peak, "frac": rate / issue_peak,
                 "source": os.path.relpath(prof_file, ROOT)}
    roofline = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak,
                "peak_source": peak_kind, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic, "algorithmic_bytes": bytes_alg[dom],
                "dram_frac": (traffic / (avg[dom] / 1e3) / 1e9 / peak
                              if traffic and avg[dom] > 0 else None),
                "kernel_ms": {k: round(v, 4) for k, v in avg.items()},
                "algorithmic_bytes_per_voxel_step": 4 * esz, "issue": issue,
                "rows_skipped_frac": {"value": skips["value"], "adjoint": skips["adjoint"]}}
    e.close()
    del e

    def oracle_result(key):
        if key not in cpu_jobs:
            return None
        return cpu_jobs[key].result()

    extra = {}
    if not args.no_extra:
        extra[f"{other}_storage"] = bench_pair_section(
            eng, torch, pair, other, c_np, args, flush, dist, dev, ws, oracle_result("other"))
        if dense is not None:
            extra["dense_oct"] = bench_pair_section(
                eng, torch, dense, "f32", c_dense, args, flush, dist, dev, ws,
                oracle_result("dense"))

    reg = None
    if not args.no_registration and args.config == "c2":
        reg = bench_registration(eng, torch, pair)
    acc = None if args.no_accuracy else bench_accuracy(eng, torch)
    rig = None
    if not args.no_rigid and args.config == "c2":
        rig = bench_rigid(eng, torch, prob)

    batch = None
    if not args.no_batch:
        del flush
        batch = bench_batch(args, eng, torch, dist, ws)

    cpu = None
    acc_main = None
    main_ref = oracle_result("main")
    if main_ref is not None:
        acc_main = accuracy(D_gpu, g_gpu, main_ref["D"], main_ref["g"])
        deg["oracle_regions"] = main_ref["n_degenerate"]
        deg["oracle_p_mass"] = main_ref["degenerate_p_mass"]
        cpu = {"value": prob.n_voxels / main_ref["seconds"] / 1e9, "unit": "Gvoxel/s", "cores": 1,
               "kind": "oracle", "host": host_info(),
               "sample": f"one full value+gradient of {prob.dims} ({prob.n_voxels} voxels) on "
                         f"one core, {main_ref['seconds']:.1f} s"}
        executor.shutdown()
        # Every host core: one process per core on the 256x256x8 slab.
        sample = slab(pair, 8)
        pool = OraclePool(sample, args.storage)
        pool.step()
        rounds = 2
        dt = sum(pool.step() for _ in range(rounds))
        pool.close()
        cpu["all_cores"] = {"value": pool.procs * sample.prob.n_voxels * rounds / dt / 1e9,
                            "unit": "Gvoxel/s", "cores": pool.procs,
                            "sample": f"{pool.procs} processes, each one value+gradient of the "
                                      f"{sample.prob.dims} slab per round, {rounds} rounds"}

    line = {"metric": METRIC, "value": value, "unit": "Gvoxel/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": step_ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": args.storage, "data": "synthetic",
            "config": {"workload": f"{pair.name}: {workload_text(pair)}, M as B, finest level",
                       "storage": args.storage, "tile": list(tile),
                       "kernel_path": "row-parallel" if lv.kernel_path else "general",
                       "n_voxels": prob.n_voxels,
                       "n_params": prob.n_params, "parallelism": f"replicas x{ws}",
                       "l2": "flushed between steps (256 MB write, outside the timed events)",
                       "wall_ms_per_step_incl_flush": wall / args.steps * 1e3},
            "accuracy_vs_oracle": acc_main, "degenerate": deg,
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "l2_warm": l2_warm,
            "clocks": clk,
            "gpu_launches": launches, **extra, "batched": batch, "registration": reg,
            "accuracy": acc, "rigid": rig}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
