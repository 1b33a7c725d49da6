#!/usr/bin/env python
"""Benchmark: Strang steps per second of the FitzHugh-Nagumo bidomain model on
the 256^3 prolate-shell workload, each diffusion solve converged to a 1e-8
GMRES residual, through the KFBI library's C ABI on one GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl kfbi|reference]
    python bench.py --workload star-sweep|shell-large|heldout|stiff|stimulus|coupled|neumann|mesh

One JSON line on rank 0.  Multi-GPU runs are independent replicas (one
stimulus location per rank, no data-path collective); `value` sums the ranks.
The reference arm times the CPU oracle on the host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Strang steps/s at 256^3 to 1e-8 residual (mixed/learned vs FP64); FFT HBM GB/s"
UNIT = "steps/s"


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


# FP64 arithmetic peak of a GB300 from its unit counts and clock: 152 SMs x
# 2 FP64 FMA/clk/SM (4 flop) x 2.07 GHz, the 1.25 TFLOP/s class figure.
FP64_PEAK_TFLOPS = 152 * 4 * 2.070e9 / 1e12


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax = float(p[2])
            except ValueError:
                continue
            for n, v in zip(names, p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def replica_time(ms_step, world, dist=None, device=None):
    """Slowest rank's time per step and the whole job's steps/s: every rank
    advances its own replica by one step per step time, so the job runs
    world / max_rank(ms) * 1000 steps per second."""
    if dist is not None:
        import torch
        t = torch.tensor([ms_step], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_step = float(t.item())
    return ms_step, world * 1000.0 / ms_step


def workload(N, rank):
    from kfbi_workloads import configs as C
    geom, grid, cfg, V0, w0 = C.config2(N=N)
    if rank > 0:
        c = C.midwall_centers([rank - 1])[0]
        V0 = C.ball_stimulus(grid, c, 0.1)
    return geom, grid, cfg, V0, w0


# ----------------------------------------------------------------- GPU arm

def run_gpu(args):
    import torch

    import paper_2104_05024_gb300.kfbi as K
    from kfbi_workloads import configs as C

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    precision = {"fp64": K.FP64, "mixed": K.MIXED, "projection": K.MIXED, "learned": K.MIXED_LEARNED}[args.precision]
    warm = K.WARM_PROJECTION if args.precision == "projection" else K.WARM_PREVIOUS

    geom, grid, cfg, V0, w0 = workload(args.N, rank)
    t0 = time.time()
    h = K.KFBI(geom, grid, sigma_i=cfg.sigma_i, sigma_e=cfg.sigma_e, dt=cfg.dt, tol=cfg.tol, precision=precision,
               restart=50, max_iter=400, warm=warm)
    torch.cuda.synchronize()
    setup_s = time.time() - t0
    fhn = C.FHN_CONFIG
    learn_info = None
    if precision == K.MIXED_LEARNED:
        learn_info, mlp = train_warmstart(args, geom, grid, cfg, dev)
        h.set_warmstart(mlp)
    V = torch.tensor(V0, device=dev)
    w = torch.tensor(w0, device=dev)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        h.bidomain_step(fhn, V, w, None, nsteps=1)
    barrier()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    l0 = K.launch_count()
    with ClockSampler(local) as clk:
        barrier()
        torch.cuda.nvtx.range_push("timed")     # lets a profiler select the timed launches
        # the K steps in up to five equal segments (events between them, no
        # synchronisation inside the timed region) for a median per step
        nseg = 5 if args.steps % 5 == 0 else 1
        seg_ev = [torch.cuda.Event(enable_timing=True) for _ in range(nseg - 1)]
        stats = []
        e0.record(stream)
        for sgi in range(nseg):
            stats += h.bidomain_step(fhn, V, w, None, nsteps=args.steps // nseg)
            if sgi < nseg - 1:
                seg_ev[sgi].record(stream)
        e1.record(stream)
        torch.cuda.nvtx.range_pop()
        barrier()
    launches = K.launch_count() - l0
    V_main, w_main = V.clone(), w.clone()
    ue_main = torch.empty_like(V)
    h.bidomain_step(fhn, V_main, w_main, ue_main, nsteps=0)     # u_e of the final state only
    ms = e0.elapsed_time(e1)
    marks = [e0] + seg_ev + [e1]
    seg_ms = [marks[i].elapsed_time(marks[i + 1]) / (args.steps // nseg) for i in range(nseg)]
    ms_step, value = replica_time(ms / args.steps, world, dist, dev)
    iters = [s["iters"] for s in stats]

    # ---- roofline of the hot path's transform solve (the unit of the
    # algorithmic bytes: one box solve, 2 G s bytes, G = (N-1)^3 unknowns)
    pk, kind = peaks()
    prec_pass = K.FP64 if precision == K.FP64 else K.MIXED
    lam = h.info["lambda"]
    N = args.N
    roof = box_solve_roofline(h, N, prec_pass, lam, pk, kind, dev)
    roof_512 = None
    if precision != K.FP64 and not args.no_large:
        # the same float32 solve at 512^3, where the grid (512 MB) leaves L2
        from kfbi_workloads import geometry as G
        h512 = K.KFBI(G.shell_config2(C.surface_res(512)), C.Grid(3, 512), tol=cfg.tol)
        roof_512 = box_solve_roofline(h512, 512, K.MIXED, lam, pk, kind, dev)
        h512.close()
        torch.cuda.empty_cache()

    # ---- end to end through the C ABI with host buffers: the same steps as
    # `value` (a second run from the same initial state, W warm-up steps, then
    # K timed steps), V and w copied in from pinned host memory and back out
    # every step
    he = K.KFBI(geom, grid, sigma_i=cfg.sigma_i, sigma_e=cfg.sigma_e, dt=cfg.dt, tol=cfg.tol, precision=precision,
                restart=50, max_iter=400, warm=warm)
    if precision == K.MIXED_LEARNED:
        he.set_warmstart(mlp)
    Vh = torch.tensor(V0, dtype=torch.float64).pin_memory()
    wh = torch.tensor(w0, dtype=torch.float64).pin_memory()
    Ve, we = torch.empty_like(V), torch.empty_like(w)
    Ve.copy_(Vh)
    we.copy_(wh)
    for _ in range(args.warmup):
        he.bidomain_step(fhn, Ve, we, None, nsteps=1)
    Vh.copy_(Ve)
    wh.copy_(we)
    barrier()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(args.steps):
        Ve.copy_(Vh, non_blocking=True)
        we.copy_(wh, non_blocking=True)
        he.bidomain_step(fhn, Ve, we, None, nsteps=1)
        Vh.copy_(Ve, non_blocking=True)
        wh.copy_(we, non_blocking=True)
    b.record(stream)
    barrier()
    he.close()
    e2e_ms, e2e_value = replica_time(a.elapsed_time(b) / args.steps, world, dist, dev)
    nbytes = V.numel() * 8 * 2

    # the other forms on the same workload and protocol (plain float64, mixed)
    forms = {args.precision: {"steps_per_s": 1000.0 / ms_step, "gmres_iters_per_step": float(np.mean(iters))}}
    if args.compare:
        for name, p, wm in (("fp64", K.FP64, K.WARM_PREVIOUS), ("mixed", K.MIXED, K.WARM_PREVIOUS),
                            ("projection", K.MIXED, K.WARM_PROJECTION), ("learned", K.MIXED_LEARNED, None)):
            if name in forms or (p == K.MIXED_LEARNED and learn_info is None):
                continue
            h2 = K.KFBI(geom, grid, sigma_i=cfg.sigma_i, sigma_e=cfg.sigma_e, dt=cfg.dt, tol=cfg.tol, precision=p,
                        restart=50, max_iter=400, warm=wm or K.WARM_PREVIOUS)
            if p == K.MIXED_LEARNED:
                h2.set_warmstart(mlp)
            V2, w2 = torch.tensor(V0, device=dev), torch.tensor(w0, device=dev)
            for _ in range(args.warmup):
                h2.bidomain_step(fhn, V2, w2, None, nsteps=1)
            barrier()
            a2, b2 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a2.record(stream)
            st2 = h2.bidomain_step(fhn, V2, w2, None, nsteps=args.steps)
            b2.record(stream)
            barrier()
            forms[name] = {"steps_per_s": 1000.0 * args.steps / a2.elapsed_time(b2),
                           "gmres_iters_per_step": float(np.mean([s["iters"] for s in st2]))}
            if name == "fp64":
                # field differences of this form's state against the float64 state after the same steps
                ue2 = torch.empty_like(V2)
                h2.bidomain_step(fhn, V2, w2, ue2, nsteps=0)
                forms["max_abs_diff_vs_fp64"] = {"V": float((V_main - V2).abs().max()),
                                                 "w": float((w_main - w2).abs().max()),
                                                 "ue": float((ue_main - ue2).abs().max()),
                                                 "V_max": float(V2.abs().max()),
                                                 "ue_max": float(ue2.abs().max())}
            h2.close()
    if "fp64" in forms:
        for name in ("mixed", "projection", "learned"):
            if name in forms:
                forms[name]["speedup_vs_fp64"] = forms[name]["steps_per_s"] / forms["fp64"]["steps_per_s"]

    result = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if precision == K.FP64 else "f32+f64", "data": "synthetic",
        "config": {"workload": f"config 2: FHN bidomain, prolate shell, {N}^3 grid, dt 0.05, GMRES tol 1e-8",
                   "timed_steps": f"steps {args.warmup + 1}..{args.warmup + args.steps} of the run "
                                  "(iterations per step fall as the projection history fills)",
                   "N": N, "M": geom.M, "precision": args.precision, "parallelism": "replicas" if world > 1 else "1gpu",
                   "l2": "inputs larger than L2 (V and w: %.0f MB each)" % (V.numel() * 8 / 1e6),
                   "setup_s": round(setup_s, 2), "n_irregular": h.info["n_irregular"],
                   "n_crossings": h.info["n_crossings"]},
        "ms_per_step_segments": [round(x, 4) for x in seg_ms],
        "ms_per_step_median": float(np.median(seg_ms)),
        "gmres_iters_per_step": float(np.mean(iters)),
        "outer_per_step": float(np.mean([s["outer"] for s in stats])),
        "forms": forms,
        "learned": learn_info if learn_info is None else dict(learn_info, used=int(sum(s["warmstart"] for s in stats))),
        "roofline": roof,
        "roofline_512": roof_512,
        "clocks": clk.summary(),
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": nbytes,
                "d2h_bytes_per_step": nbytes},
        "gpu_launches": int(launches),
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        result["cpu_baseline"] = cpu_baseline(args.N, steps=1)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    h.close()
    if rank == 0:
        print(json.dumps(result), flush=True)


def _pass_times(h, prec, lam, reps, flush=None):
    """Mean CUDA-event time (ms) of each transform pass of the box solver on
    the handle's padded work grid (pass 0 x forward, 1 y, 2 z solve, 3 x
    inverse).  flush: a tensor larger than L2 written before every launch
    (cold-cache times), else back-to-back launches."""
    import torch
    stream = torch.cuda.current_stream()
    out = {}
    for p in ((0, 1, 2, 3, 4, 5) if h.info["xy_fused"] and prec != 0 else (0, 1, 2, 3)):
        for _ in range(3):
            h.transform_pass(p, lam, prec)
        tot = 0.0
        if flush is None:
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(reps):
                h.transform_pass(p, lam, prec)
            b.record(stream)
            torch.cuda.synchronize()
            tot = a.elapsed_time(b)
        else:
            for _ in range(reps):
                flush.add_(1.0)
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                h.transform_pass(p, lam, prec)
                b.record(stream)
                torch.cuda.synchronize()
                tot += a.elapsed_time(b)
        out[p] = tot / reps
    return out


def _chain_time(h, prec, lam, reps):
    """Mean CUDA-event time (ms) of one box solve as the hot path runs it:
    its passes (x forward, y, z solve, y, x inverse; with the fused x-y
    passes x-y forward, z solve, x-y inverse) launched back to back, `reps`
    solves in a row."""
    import torch
    stream = torch.cuda.current_stream()
    seq = (4, 2, 5) if h.info["xy_fused"] and prec != 0 else (0, 1, 2, 1, 3)
    for _ in range(3):
        for p in seq:
            h.transform_pass(p, lam, prec)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(reps):
        for p in seq:
            h.transform_pass(p, lam, prec)
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


# DRAM bytes (ncu dram__bytes_read.sum + dram__bytes_write.sum, caches flushed
# before each launch) per launch of each transform pass of the current
# kernels, by (N, element size, fused x-y passes) and pass 0..5; the
# five-pass solve runs pass 1 twice.  Kernels changed since the capture must
# drop their entry.
NCU_DRAM_BYTES = {
    # ncu captures each launch cold (caches flushed before it), so at 256^3
    # every pass reads the grid from DRAM once; back-to-back passes in the
    # timed region find it in L2 (the cold-capture bytes go with solve_ms_cold)
    (256, 4, False): {0: 4.62e6, 1: 70.2e6, 2: 70.65e6, 3: 71.3e6},
    (512, 4, False): {0: 473.1e6, 1: 1007.06e6, 2: 1007.27e6, 3: 1006.37e6},
}


def box_solve_roofline(h, N, prec, lam, pk, kind, dev):
    """Roofline line of one box solve: algorithmic bytes 2 G s (G = (N-1)^3
    unknowns, s the element size: the right-hand side read once and the
    solution written once) over the time of its five passes (x forward, y,
    z solve, y, x inverse) run back to back as the hot path runs them,
    against the measured HBM copy bandwidth.  Float64 solves are also
    reported against the FP64 pipe."""
    import torch
    import paper_2104_05024_gb300.kfbi as K
    esize = 8 if prec == K.FP64 else 4
    G = (N - 1) ** 3
    alg = 2.0 * G * esize
    warm = _pass_times(h, prec, lam, 20)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)   # 256 MB > 129 MB L2
    cold = _pass_times(h, prec, lam, 5, flush)
    del flush
    fused = 4 in warm
    # five passes (x forward, y, z solve, y, x inverse) or, with the fused x-y
    # passes, three (x-y forward, z solve, x-y inverse)
    solve = (lambda t: t[4] + t[2] + t[5]) if fused else (lambda t: t[0] + 2.0 * t[1] + t[2] + t[3])  # noqa: E731
    grid_mb = N ** 3 * esize / 1e6
    resident = grid_mb < 129.0
    # back-to-back passes (the hot path's GMRES iterations run them so); a
    # grid that fits the L2 stays resident between them, which the label says
    t = warm
    chain = _chain_time(h, prec, lam, 20)
    achieved = alg / (chain / 1e3) / 1e9
    kern = "k_xy_fwd, k_strided_tma (z), k_xy_inv" if fused else "k_xfwd, k_strided*, k_xinv"
    roof = {"kernel": f"box solve {N}^3 {'float64' if esize == 8 else 'float32'} ({kern})",
            "unit_of_work": "one box solve: 2 G s bytes, G = (N-1)^3", "bound": "hbm",
            "achieved": achieved, "peak": pk["hbm_gbs"], "unit": "GB/s", "peak_source": kind,
            "frac": achieved / pk["hbm_gbs"],
            "algorithmic_bytes": alg, "solve_ms": chain, "solve_ms_sum_of_passes": solve(t),
            "passes": 3 if fused else 5,
            "l2": (f"L2-resident: the {grid_mb:.0f} MB grid fits the 129 MB L2 and stays there between "
                   "back-to-back passes; solve_ms_cold has a 256 MB L2 flush before each pass" if resident else
                   f"grid {grid_mb:.0f} MB exceeds the 129 MB L2: back-to-back passes"),
            "pass_ms": {k: round(v, 4) for k, v in t.items()},
            "pass_ms_cold": {k: round(v, 4) for k, v in cold.items()},
            "solve_ms_cold": solve(cold),
            "pass_gbs": {k: round(2.0 * N ** 3 * esize / (v / 1e3) / 1e9, 1) for k, v in t.items()}}
    nb = NCU_DRAM_BYTES.get((N, esize, fused))
    if nb is not None:
        tr = (nb[4] + nb[2] + nb[5]) if fused else (nb[0] + 2 * nb[1] + nb[2] + nb[3])
        roof["traffic"] = tr
        roof["traffic_unit"] = "ncu dram read + write bytes of the five passes of one solve"
        # an L2-resident grid: the cold capture's bytes over the cold solve time
        tt = solve(cold) if resident else chain
        roof["dram_gbs"] = tr / (tt / 1e3) / 1e9
        roof["dram_frac"] = roof["dram_gbs"] / pk["hbm_gbs"]
        if resident:
            roof["traffic_note"] = "cold capture; dram_gbs uses solve_ms_cold"
    else:
        roof["traffic"] = None
    if esize == 8:
        lines = (N - 1) * (N - 1)
        fl_dst = 2.5 * N * np.log2(N)            # real-FFT flop count of one DST-I line
        flops = 6 * lines * fl_dst + 3.0 * G
        roof["fp64_tflops"] = flops / (chain / 1e3) / 1e12
        roof["fp64_peak_tflops"] = FP64_PEAK_TFLOPS
    return roof


def train_warmstart(args, geom, grid, cfg, dev):
    """Train the warm-start network on densities of runs with the 8 training
    stimulus locations (untimed); the timed run's stimulus is held out."""
    import torch

    import paper_2104_05024_gb300.kfbi as K
    from paper_2104_05024_gb300 import warmstart as WS
    from kfbi_workloads import configs as C

    t0 = time.time()
    Fs, Ts = [], []
    for c in C.midwall_centers(C.TRAIN_SEEDS):
        h = K.KFBI(geom, grid, sigma_i=cfg.sigma_i, sigma_e=cfg.sigma_e, dt=cfg.dt, tol=cfg.tol, precision=K.MIXED,
                   restart=50, max_iter=400)
        V = torch.tensor(C.ball_stimulus(grid, c, 0.1), device=dev)
        w = torch.zeros_like(V)
        F, T = WS.collect(h, C.FHN_CONFIG, V, w, args.train_steps)
        Fs.append(F)
        Ts.append(T)
        h.close()
    F, T = torch.cat(Fs), torch.cat(Ts)
    norm = WS.fit_norm(F, T)
    mlp = K.MLP(WS.init_params(0), norm, max(8192, geom.M))
    losses = WS.train(mlp, F, T, epochs=args.train_epochs, batch=4096, lr=2e-3)
    torch.cuda.synchronize()
    info = {"train_rows": int(F.shape[0]), "train_seeds": len(C.TRAIN_SEEDS), "steps_per_seed": args.train_steps,
            "epochs": args.train_epochs, "loss_first_last": [round(losses[0], 5), round(losses[-1], 5)],
            "train_s": round(time.time() - t0, 1)}
    return info, mlp


# ------------------------------------------------- single-solve workloads

def _event_ms(fn, reps=1):
    import torch
    stream = torch.cuda.current_stream()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(stream)
    out = None
    for _ in range(reps):
        out = fn()
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps, out


def run_star_sweep(args):
    """Config 1: Neumann modified-Helmholtz solve (lambda = 2/dt = 40) on the
    star body with u = prod cos(pi x_a), GMRES to 1e-10, N = 32 ... 256:
    max / rms / off-axis max error over the interior nodes, observed orders,
    iterations, time, float64 and float32 transforms with refinement."""
    import torch

    import paper_2104_05024_gb300.kfbi as K
    from kfbi_workloads import configs as C
    dev = torch.device("cuda", 0)
    rows, prev = [], None
    for N in (32, 64, 128, 256):
        geom, grid, lam, tol = C.config1(N)
        t0 = time.time()
        h = K.KFBI(geom, grid, tol=tol, restart=50, max_iter=400)
        torch.cuda.synchronize()
        setup_s = time.time() - t0
        f, u_ex, gN = C.manufactured(geom, grid, lam)
        inside = h.export_setup()["inside"]
        # the star surface has conical points where it meets the z axis (the
        # radius varies linearly with the polar angle there); errors are also
        # reported away from them
        X = grid.coords()
        off_axis = np.broadcast_to(X[0] ** 2 + X[1] ** 2, grid.shape) > 0.15 ** 2
        fd, gd = torch.tensor(f, device=dev), torch.tensor(gN, device=dev)
        u = torch.empty(grid.shape, dtype=torch.float64, device=dev)
        psi = torch.zeros(geom.M, dtype=torch.float64, device=dev)
        row = {"N": N, "M": geom.M, "setup_s": round(setup_s, 3)}
        for name, prec in (("fp64", K.FP64), ("mixed", K.MIXED)):
            def solve():
                psi.zero_()
                return h.solve_neumann(fd, gd, u, psi, lam, tol=tol, precision=prec)
            solve()
            ms, st = _event_ms(solve, reps=3)
            e = np.abs(u.cpu().numpy() - u_ex)
            row[name] = {"ms": round(ms, 3), "iters": st["iters"], "true_rel_res": st["true_rel_res"],
                         "max_err": float(e[inside].max()), "rms_err": float(np.sqrt((e[inside] ** 2).mean())),
                         "max_err_off_axis": float(e[inside & off_axis].max())}
        if prev is not None:
            row["order"] = {k: float(np.log2(prev["fp64"][k] / row["fp64"][k]))
                            for k in ("max_err", "rms_err", "max_err_off_axis")}
        rows.append(row)
        prev = row
        h.close()
    # the stated node count (cube-sphere resolution n = N: about 6 N^2 nodes,
    # spacing about 0.47 h), float64, 300 iterations at most
    from kfbi_workloads import geometry as G
    dense = []
    for N in (32, 64):
        geom, grid = G.star_config1(N), C.Grid(3, N)
        lam, tol = 40.0, 1e-10
        h = K.KFBI(geom, grid, tol=tol, restart=50, max_iter=300)
        f, u_ex, gN = C.manufactured(geom, grid, lam)
        inside = h.export_setup()["inside"]
        u = torch.empty(grid.shape, dtype=torch.float64, device=dev)
        psi = torch.zeros(geom.M, dtype=torch.float64, device=dev)
        st = h.solve_neumann(torch.tensor(f, device=dev), torch.tensor(gN, device=dev), u, psi, lam, tol=tol,
                             max_iter=300)
        e = np.abs(u.cpu().numpy() - u_ex)
        dense.append({"N": N, "M": geom.M, "iters": st["iters"], "rel_res": st["rel_res"],
                      "converged": st["rel_res"] <= tol, "max_err": float(e[inside].max())})
        h.close()
    print(json.dumps({"metric": "star-body Neumann solve: max error, observed order, time", "workload":
                      "config 1: star r = 0.6 + 0.1 sin(3 theta) cos(2 phi), lambda 40, tol 1e-10",
                      "unit": "ms", "rows": rows, "rows_6N2_nodes": dense}), flush=True)


def run_shell_large(args):
    """Config 3: single Neumann solve on the shell at 384^3 and 512^3, Gaussian
    bump right-hand side, GMRES to 1e-8, float64 against float32 transforms
    with float64 refinement: iterations, solve time, box-solve GB/s."""
    import torch

    import paper_2104_05024_gb300.kfbi as K
    from kfbi_workloads import configs as C, geometry as G
    dev = torch.device("cuda", 0)
    pk, kind = peaks()
    rows = []
    for N in (384, 512):
        geom, grid, lam, tol = G.shell_config2(C.surface_res(N)), C.Grid(3, N), 40.0, 1e-8
        t0 = time.time()
        h = K.KFBI(geom, grid, tol=tol, restart=50, max_iter=400)
        torch.cuda.synchronize()
        row = {"N": N, "M": geom.M, "setup_s": round(time.time() - t0, 2), "n_irregular": h.info["n_irregular"]}
        fd = torch.tensor(C.gaussian_rhs(grid, seed=0), device=dev)
        gd = torch.zeros(geom.M, dtype=torch.float64, device=dev)
        u = torch.empty(grid.shape, dtype=torch.float64, device=dev)
        u64 = torch.empty_like(u)
        psi = torch.zeros(geom.M, dtype=torch.float64, device=dev)
        for name, prec, esize in (("fp64", K.FP64, 8), ("fp32+refine", K.MIXED, 4)):
            def solve():
                psi.zero_()
                return h.solve_neumann(fd, gd, u, psi, lam, tol=tol, precision=prec)
            solve()
            ms, st = _event_ms(solve, reps=2)
            box_prec = K.FP64 if prec == K.FP64 else K.FP32
            h.box_solve(fd, u, lam, precision=box_prec)
            box_ms, _ = _event_ms(lambda: h.box_solve(fd, u, lam, precision=box_prec), reps=5)
            # five transform passes, each reading and writing the padded grid
            gbs = 5 * 2.0 * N ** 3 * esize / (box_ms / 1e3) / 1e9
            row[name] = {"solve_ms": round(ms, 2), "iters": st["iters"], "outer": st["outer"],
                         "rel_res": st["rel_res"], "true_rel_res": st["true_rel_res"],
                         "box_solve_ms": round(box_ms, 3), "box_solve_gbs": round(gbs, 1),
                         "box_solve_frac_hbm": round(gbs / pk["hbm_gbs"], 3)}
        # field agreement of the two forms
        h.solve_neumann(fd, gd, u64, psi.zero_(), lam, tol=tol, precision=K.FP64)
        h.solve_neumann(fd, gd, u, psi.zero_(), lam, tol=tol, precision=K.MIXED)
        row["max_abs_diff_u_vs_fp64"] = float((u - u64).abs().max())
        row["u_max"] = float(u64.abs().max())
        rows.append(row)
        del fd, u, u64, psi
        h.close()
    print(json.dumps({"metric": "shell Neumann solve at 384^3 / 512^3: time, iterations, box-solve GB/s",
                      "workload": "config 3: prolate shell, 32 Gaussian bumps (seed 0), lambda 40, tol 1e-8",
                      "unit": "ms", "peak_hbm_gbs": pk["hbm_gbs"], "peak_source": kind, "rows": rows}), flush=True)


def run_heldout(args):
    """Config 4: the warm-start network trained on the 8 training stimulus
    locations, then runs from the 4 held-out locations with the plain
    previous-density guess and with the learned guess, same steps each."""
    import torch

    import paper_2104_05024_gb300.kfbi as K
    from kfbi_workloads import configs as C
    dev = torch.device("cuda", 0)
    geom, grid, cfg, _, _ = C.config2(N=args.N)
    info, mlp = train_warmstart(args, geom, grid, cfg, dev)
    rows = []
    for seed, c in zip(C.HELDOUT_SEEDS, C.midwall_centers(C.HELDOUT_SEEDS)):
        V0 = torch.tensor(C.ball_stimulus(grid, c, 0.1), device=dev)
        row = {"seed": seed, "center": [round(x, 4) for x in c]}
        out = {}
        for name, prec, wm in (("previous", K.MIXED, K.WARM_PREVIOUS), ("projection", K.MIXED, K.WARM_PROJECTION),
                               ("learned", K.MIXED_LEARNED, K.WARM_PREVIOUS)):
            h = K.KFBI(geom, grid, sigma_i=cfg.sigma_i, sigma_e=cfg.sigma_e, dt=cfg.dt, tol=cfg.tol, precision=prec,
                       restart=50, max_iter=400, warm=wm)
            if prec == K.MIXED_LEARNED:
                h.set_warmstart(mlp)
            V, w = V0.clone(), torch.zeros_like(V0)
            ms, st = _event_ms(lambda: h.bidomain_step(C.FHN_CONFIG, V, w, None, nsteps=args.steps))
            row[name] = {"steps_per_s": round(1000.0 * args.steps / ms, 3),
                         "gmres_iters": int(sum(s["iters"] for s in st)),
                         "guess_used": int(sum(s["warmstart"] for s in st))}
            out[name] = V
            h.close()
        row["speedup_vs_previous"] = {k: round(row[k]["steps_per_s"] / row["previous"]["steps_per_s"], 3)
                                      for k in ("projection", "learned")}
        row["max_abs_diff_V_vs_previous"] = {k: float((out[k] - out["previous"]).abs().max())
                                             for k in ("projection", "learned")}
        rows.append(row)
    mlp.close()
    print(json.dumps({"metric": "held-out stimuli: GMRES iterations and Strang steps/s, learned vs previous guess",
                      "workload": f"config 4: shell {args.N}^3, {args.steps} Strang steps from each held-out "
                                  "stimulus, tol 1e-8, float32 transforms with float64 refinement",
                      "unit": "steps/s", "training": info, "rows": rows}), flush=True)


def run_stiff(args):
    """The paper's stiff FitzHugh-Nagumo parameters (H 100, theta 0.25,
    alpha 0.25, zeta 1, beta 1000) with dt = h on the shell at N^3, GMRES and
    the simple iteration (gamma 0.8), float64 and float32 transforms with
    refinement, tol 1e-8: Strang steps/s and iterations per step."""
    import torch

    import paper_2104_05024_gb300.kfbi as K
    from kfbi_workloads import configs as C
    dev = torch.device("cuda", 0)
    geom, grid, cfg0, V0, w0 = C.config2(N=args.N)
    dt = grid.h
    rows = {}
    for name, prec, solver, warm in (("fp64_gmres", K.FP64, K.GMRES, K.WARM_PREVIOUS),
                                     ("fp64_simple", K.FP64, K.RICHARDSON, K.WARM_PREVIOUS),
                                     ("mixed_gmres_projection", K.MIXED, K.GMRES, K.WARM_PROJECTION),
                                     ("mixed_simple", K.MIXED, K.RICHARDSON, K.WARM_PREVIOUS)):
        h = K.KFBI(geom, grid, sigma_i=1.0, sigma_e=2.0, dt=dt, tol=1e-8, precision=prec, solver=solver,
                   restart=50, max_iter=2000, warm=warm)
        V, w = torch.tensor(V0, device=dev), torch.tensor(w0, device=dev)
        h.bidomain_step(C.FHN_PAPER, V, w, None, nsteps=2)
        ms, st = _event_ms(lambda: h.bidomain_step(C.FHN_PAPER, V, w, None, nsteps=args.steps))
        rows[name] = {"steps_per_s": round(1000.0 * args.steps / ms, 3),
                      "iters_per_step": float(np.mean([s["iters"] for s in st]))}
        h.close()
    print(json.dumps({"metric": "stiff FHN Strang steps/s, GMRES vs simple iteration",
                      "workload": f"shell {args.N}^3, FHN H 100 theta 0.25 alpha 0.25 zeta 1 beta 1000, "
                                  f"dt = h = {dt:.5f}, tol 1e-8, {args.steps} steps after 2",
                      "unit": "steps/s", "rows": rows}), flush=True)


def run_stimulus(args):
    """Virtual electrode (Section 7: +-10 in balls of radius 0.25 at
    (-+0.3, 0, 0)) on a sphere of radius 0.6 at N^3 with the paper's
    FitzHugh-Nagumo parameters, dt = h, tol 1e-8: the S Poisson problem
    (solved once per call) and Strang steps/s, float64 and float32 transforms
    with refinement and the history projection."""
    import torch

    import paper_2104_05024_gb300.kfbi as K
    from kfbi_workloads import configs as C, geometry as G
    dev = torch.device("cuda", 0)
    N = args.N
    geom, grid = G.sphere3(0.6, C.surface_res(N)), C.Grid(3, N)
    I = torch.tensor(C.virtual_electrode(grid), device=dev)
    rows = {}
    for name, prec, warm in (("fp64", K.FP64, K.WARM_PREVIOUS), ("mixed_projection", K.MIXED, K.WARM_PROJECTION)):
        h = K.KFBI(geom, grid, sigma_i=1.0, sigma_e=2.0, dt=grid.h, tol=1e-8, precision=prec, warm=warm,
                   restart=50, max_iter=400)
        V = torch.zeros(grid.shape, dtype=torch.float64, device=dev)
        w = torch.zeros_like(V)
        ue = torch.empty_like(V)
        ms0, _ = _event_ms(lambda: h.bidomain_step(C.FHN_PAPER, V, w, ue, nsteps=1, istim=I))
        ms, st = _event_ms(lambda: h.bidomain_step(C.FHN_PAPER, V, w, ue, nsteps=args.steps, istim=I))
        ms_s = ms0 - ms / args.steps   # the S solve of a call, less one step
        rows[name] = {"steps_per_s": round(1000.0 * args.steps / ms, 3),
                      "iters_per_step": float(np.mean([s["iters"] for s in st])),
                      "S_solve_ms": round(ms_s, 2), "V_max": float(V.abs().max()), "ue_max": float(ue.abs().max())}
        h.close()
    print(json.dumps({"metric": "virtual-electrode Strang steps/s and S Poisson solve",
                      "workload": f"sphere r 0.6, {N}^3, FHN H 100 theta 0.25 alpha 0.25 zeta 1 beta 1000, "
                                  f"dt = h, tol 1e-8, {args.steps} steps (one call)",
                      "unit": "steps/s", "rows": rows}), flush=True)


def run_coupled(args):
    """The anisotropic coupled system (Eq. pde1) with the paper's conductivity
    tensors D_i = diag(30, 5, 5), D_e = diag(20, 10, 10) in the sphere of
    Example 3 (radius 0.9: the paper leaves it unstated and observes up to
    x = 0.875) at N^3, FitzHugh-Nagumo of the workloads with the stimulus ball
    at (0.8, 0, 0), dt 0.05, GMRES to 1e-8: Strang steps/s and iterations per
    step in float64, with float32 transforms (GMRES-IR) and with the history
    projection as well, and the coupled box solve (two fields, per-mode 2 x 2
    solve) against the scalar float64 one."""
    import torch

    import paper_2104_05024_gb300.kfbi as K
    from kfbi_workloads import configs as C, geometry as G
    dev = torch.device("cuda", 0)
    N = args.N
    geom, grid = G.sphere3(0.9, C.surface_res(N)), C.Grid(3, N)
    V0 = C.ball_stimulus(grid, (0.8, 0.0, 0.0), 0.1)
    Di, De = (30.0, 5.0, 5.0), (20.0, 10.0, 10.0)
    forms, fields = {}, {}
    for name, prec, warm in (("fp64", K.FP64, K.WARM_PREVIOUS), ("mixed", K.MIXED, K.WARM_PREVIOUS),
                             ("mixed_projection", K.MIXED, K.WARM_PROJECTION)):
        h = K.KFBI(geom, grid, D_i=Di, D_e=De, dt=0.05, tol=1e-8, restart=50, max_iter=600, precision=prec,
                   warm=warm)
        V = torch.tensor(V0, device=dev)
        w = torch.zeros_like(V)
        ue = torch.empty_like(V)
        h.bidomain_step(C.FHN_CONFIG, V, w, None, nsteps=2)
        ms, st = _event_ms(lambda: h.bidomain_step(C.FHN_CONFIG, V, w, ue, nsteps=args.steps))
        forms[name] = {"steps_per_s": round(1000.0 * args.steps / ms, 3),
                       "iters_per_step": float(np.mean([s["iters"] for s in st])),
                       "outer_per_step": float(np.mean([s["outer"] for s in st])),
                       "true_rel_res_max": float(max(s["true_rel_res"] for s in st)),
                       "V_max": float(V.abs().max()), "ue_max": float(ue.abs().max())}
        fields[name] = (V, ue)
        if name == "fp64":
            r = torch.randn(grid.shape, dtype=torch.float64, device=dev)
            vi, ve = torch.empty_like(r), torch.empty_like(r)
            h.box_solve_coupled(r, r, vi, ve, 40.0)
            box_ms, _ = _event_ms(lambda: h.box_solve_coupled(r, r, vi, ve, 40.0), reps=5)
        h.close()
    for name in ("mixed", "mixed_projection"):
        forms[name]["speedup_vs_fp64"] = round(forms[name]["steps_per_s"] / forms["fp64"]["steps_per_s"], 2)
    diff = {name: {"V": float((fields[name][0] - fields["fp64"][0]).abs().max()),
                   "ue": float((fields[name][1] - fields["fp64"][1]).abs().max())}
            for name in ("mixed", "mixed_projection")}
    hs = K.KFBI(geom, grid, tol=1e-8)
    hs.box_solve(r, vi, 60.0, precision=K.FP64)
    box1_ms, _ = _event_ms(lambda: hs.box_solve(r, vi, 60.0, precision=K.FP64), reps=5)
    hs.close()
    print(json.dumps({"metric": "anisotropic coupled Strang steps/s (float64 and float32 transforms with refinement)",
                      "workload": f"sphere r 0.9 at {N}^3, D_i diag(30, 5, 5), D_e diag(20, 10, 10), FHN of the "
                                  f"workloads, dt 0.05, tol 1e-8, {args.steps} steps after 2",
                      "unit": "steps/s", "forms": forms, "max_abs_diff_vs_fp64": diff,
                      "coupled_box_solve_ms": round(box_ms, 3), "scalar_box_solve_ms": round(box1_ms, 3)}),
          flush=True)


def run_neumann(args):
    """The Neumann box (zero normal derivative on the box boundary, the box
    Green's function of Section 4; all (N+1)^3 nodes, cosine transforms)
    against the Dirichlet box on the shell workload at N^3, in float64 and
    with float32 transforms (GMRES-IR), projection warm start, tol 1e-8:
    Strang steps/s, iterations per step, the box solve time (float64, or
    plain float32) and its algorithmic bytes (read r, write v) per second."""
    import torch

    import paper_2104_05024_gb300.kfbi as K
    from kfbi_workloads import configs as C
    dev = torch.device("cuda", 0)
    N = args.N
    rows = {}
    for bc, prec in (("dirichlet", K.FP64), ("neumann", K.FP64), ("dirichlet", K.MIXED), ("neumann", K.MIXED)):
        geom, grid, cfg, V0, w0 = C.config2(N=N, bc=bc)
        h = K.KFBI(geom, grid, sigma_i=cfg.sigma_i, sigma_e=cfg.sigma_e, dt=cfg.dt, tol=cfg.tol, precision=prec,
                   warm=K.WARM_PROJECTION, restart=50, max_iter=500)
        V, w = torch.tensor(V0, device=dev), torch.tensor(w0, device=dev)
        ue = torch.empty_like(V)
        h.bidomain_step(C.FHN_CONFIG, V, w, None, nsteps=3)
        ms, st = _event_ms(lambda: h.bidomain_step(C.FHN_CONFIG, V, w, ue, nsteps=args.steps))
        r = torch.randn(grid.shape, dtype=torch.float64, device=dev)
        v = torch.empty_like(r)
        bprec = K.FP64 if prec == K.FP64 else K.FP32
        h.box_solve(r, v, h.info["lambda"], precision=bprec)
        box_ms, _ = _event_ms(lambda: h.box_solve(r, v, h.info["lambda"], precision=bprec), reps=5)
        pts = int(np.prod(grid.shape))
        key = bc + ("_fp64" if prec == K.FP64 else "_mixed")
        rows[key] = {"field_nodes": pts, "steps_per_s": round(1000.0 * args.steps / ms, 3),
                    "iters_per_step": float(np.mean([s["iters"] for s in st])),
                    "true_rel_res_max": float(max(s["true_rel_res"] for s in st)),
                    "V_max": float(V.abs().max()), "ue_max": float(ue.abs().max()),
                    "box_solve_ms": round(box_ms, 3),
                    "box_solve_algorithmic_GBs": round(2 * 8 * pts / (box_ms * 1e-3) / 1e9, 1)}
        h.close()
    print(json.dumps({"metric": "Neumann-box Strang steps/s and box solve (vs the Dirichlet box)",
                      "workload": f"shell {N}^3, FHN of the workloads, dt 0.05, tol 1e-8, float64 and float32 "
                                  f"transforms, projection warm start, {args.steps} steps after 3",
                      "unit": "steps/s", "rows": rows}), flush=True)


def run_mesh(args):
    """A domain given only by its boundary triangle mesh (Section 5.3,
    Example 4; the left ventricle of the paper is not available, a smooth
    non-convex geodesic mesh with valence-5 vertices stands in): setup time
    of the mesh classification, crossings and local surfaces on the GPU, and
    Strang steps/s at N^3 in float64 and in the float32-transform form with
    the history projection, tol 1e-8."""
    import time

    import torch

    import paper_2104_05024_gb300.kfbi as K
    from kfbi_workloads import configs as C, geometry as G
    dev = torch.device("cuda", 0)
    N = args.N
    geom, grid = G.bean_mesh(max(4, N // 4)), C.Grid(3, N)
    V0 = C.ball_stimulus(grid, (0.45, 0.0, 0.0), 0.15)
    rows = {}
    for name, prec in (("fp64", K.FP64), ("mixed_projection", K.MIXED)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h = K.KFBI(geom, grid, sigma_i=1.0, sigma_e=2.0, dt=0.05, tol=1e-8, precision=prec,
                   warm=K.WARM_PROJECTION, restart=50, max_iter=500)
        torch.cuda.synchronize()
        setup_s = time.perf_counter() - t0
        V = torch.tensor(V0, device=dev)
        w = torch.zeros_like(V)
        h.bidomain_step(C.FHN_CONFIG, V, w, None, nsteps=3)
        ms, st = _event_ms(lambda: h.bidomain_step(C.FHN_CONFIG, V, w, None, nsteps=args.steps))
        rows[name] = {"setup_s": round(setup_s, 3), "steps_per_s": round(1000.0 * args.steps / ms, 3),
                      "iters_per_step": float(np.mean([s["iters"] for s in st])),
                      "true_rel_res_max": float(max(s["true_rel_res"] for s in st)),
                      "V_max": float(V.abs().max()), "n_irregular": h.info["n_irregular"],
                      "n_crossings": h.info["n_crossings"]}
        h.close()
    print(json.dumps({"metric": "mesh-only domain: setup and Strang steps/s",
                      "workload": f"geodesic bean mesh, {geom.M} vertices / {geom.tri.shape[0]} triangles, {N}^3, "
                                  f"FHN of the workloads, dt 0.05, tol 1e-8, {args.steps} steps after 3",
                      "unit": "steps/s", "rows": rows}), flush=True)


# -------------------------------------------------------------- CPU oracle

def cpu_baseline(N, steps=1):
    """Oracle Strang steps on the host cores (setup excluded from the time)."""
    from kfbi_workloads import configs as C
    from oracle.bidomain import Bidomain
    geom, grid, cfg, V0, w0 = workload(N, 0)
    t0 = time.time()
    bd = Bidomain(geom, grid, cfg, C.FHN_CONFIG)
    setup = time.time() - t0
    V, w = V0.copy(), w0.copy()
    t0 = time.time()
    for _ in range(steps):
        V, w, _ = bd.step(V, w)
    dt = time.time() - t0
    return {"value": steps / dt, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"{steps} Strang step(s) of the {N}^3 workload after a {setup:.0f} s oracle setup "
                      "(numpy/scipy FP64, scipy.fft workers = all cores)"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    steps = max(1, min(args.steps, 2))
    cb = cpu_baseline(args.N, steps=steps)
    cb["sample"] += f"; timed {steps} of the requested {args.steps} steps"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": cb["value"], "unit": UNIT, "n_gpus": 0, "steps": steps,
        "warmup": 0, "ms_per_step": 1000.0 / cb["value"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"config 2: FHN bidomain, prolate shell, {args.N}^3 grid, dt 0.05, GMRES tol 1e-8",
                   "N": args.N, "precision": "fp64"},
        "cpu_baseline": cb,
        "e2e": {"value": cb["value"], "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed Strang steps (default: 200, the length of the config-2 run, for the strang "
                         "workload; 40 for the others)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="kfbi", choices=["kfbi", "reference"])
    ap.add_argument("--precision", default="learned", choices=["fp64", "mixed", "projection", "learned"],
                    help="fp64 / mixed: previous-density start; projection: mixed with the history projection; "
                         "learned: projection corrected by the network")
    ap.add_argument("--no-compare", dest="compare", action="store_false",
                    help="skip timing the other precision forms on the same workload")
    ap.add_argument("--N", type=int, default=256)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-large", action="store_true", help="skip the 512^3 box-solve roofline line")
    ap.add_argument("--train-steps", type=int, default=12, help="Strang steps per training stimulus (learned form)")
    ap.add_argument("--train-epochs", type=int, default=8)
    ap.add_argument("--workload", default="strang",
                    choices=["strang", "star-sweep", "shell-large", "heldout", "stiff", "stimulus", "coupled", "neumann", "mesh"],
                    help="strang: the timed benchmark; the others print one result line each")
    args = ap.parse_args()
    if args.steps is None:
        args.steps = 200 if args.workload == "strang" and args.impl == "kfbi" else 40
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "star-sweep":
        run_star_sweep(args)
    elif args.workload == "shell-large":
        run_shell_large(args)
    elif args.workload == "heldout":
        run_heldout(args)
    elif args.workload == "stiff":
        run_stiff(args)
    elif args.workload == "stimulus":
        run_stimulus(args)
    elif args.workload == "coupled":
        run_coupled(args)
    elif args.workload == "neumann":
        run_neumann(args)
    elif args.workload == "mesh":
        run_mesh(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
