#!/usr/bin/env python
"""Benchmark: BODex coarse-stage synthesis on GB300.

One bench step = one 200-upper-iteration synthesis run (FK -> SDF query ->
G -> 12 batched QPs x 50 ADMM iterations -> energy + envelope gradient ->
Adam + clamp, every iteration) over 4096 grasps of the paper-scale
workload: Shadow-like 5-finger hand (22 joints, 5 contacts), 64^3 SDF grid
(2 mm) of a seeded union of 8 primitives, 12 desired wrenches.  Inputs are
resident in HBM when the timed region starts; L2 (129 MB) is flushed by a
256 MB write before every timed step (the working set is smaller than L2).

Prints ONE JSON line (rank 0).  `--impl reference` times the FP64 CPU
oracle on a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import bodex_inputs as I  # noqa: E402

METRIC = "grasps/s (200-step runs) & QP solves/s at 1e-5 residual; p50/p99 job latency"
WORKLOAD = "paper-scale: 4096 grasps, 5-finger 22-joint hand, 5 contacts, 64^3 SDF grid (2 mm), " \
           "12 wrenches, 200 upper steps x 50 ADMM iterations, fp32"
N_STEPS, ADMM_ITERS, B_PER_GPU, S = 200, 50, 4096, 12
FP32_LANES = 128  # FP32 FMA lanes per SM (Blackwell)
# dram__bytes_read.sum + dram__bytes_write.sum of one fused_kernel<5, step> launch on this
# workload, from an ncu capture of a 5-step launch of the same kernel (the state is read once
# per launch and the grid stays in L2, so the bytes do not grow with the steps)
TRAFFIC_BYTES = 14_563_072 + 4_864
TRAFFIC_SOURCE = "ncu dram__bytes_read.sum + dram__bytes_write.sum of one fused_kernel<5, step> launch (5 steps)"


def admm_iter_flops(m: int) -> int:
    """Algorithmic FLOPs of one ADMM iteration of one QP (see below)."""
    nv, nc, nnz = 3 * m, 9 * m + 1, 26 * m
    return 4 * nnz + 2 * nv * nv + 6 * nv + 10 * nc


def flops_per_grasp_step(m: int, n_joints: int, s: int, iters: int) -> float:
    """Algorithmic FLOPs of one upper iteration of one grasp (FMA = 2).

    ADMM iteration of one QP:  F_it = 4 nnz(A) + 2 nv^2 + 6 nv + 10 nc,
    nnz(A) = 26 m, nv = 3m, nc = 9m + 1.
    Per grasp and iteration: G^T G 6 nv (nv+1), Cholesky + inverse 2 nv^3,
    FK 72 (6+n), SDF + G 150 m, adjoint 1000, per wrench q, Q and r 24 nv."""
    nv = 3 * m
    f_it = admm_iter_flops(m)
    setup = 6 * nv * (nv + 1) + 2 * nv ** 3 + 72 * (6 + n_joints) + 150 * m + 1000 + s * 24 * nv
    return s * iters * f_it + setup


def sm_count() -> int:
    """Streaming multiprocessors of the current device (152 on a GB300)."""
    import torch
    return int(torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count)


def fp32_peak_tflops(sm_mhz: float) -> float:
    return sm_count() * FP32_LANES * 2 * sm_mhz * 1e6 / 1e12


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (FileNotFoundError, OSError):
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
        sm, mx, reasons = [], None, set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


# ---------------------------------------------------------------------------- CPU oracle
def oracle_run(wl: str, grasps: int, steps: int, grad_mode: str = "analytic", threads: int | None = None):
    """One measured run of the FP64 oracle's coarse-stage loop (exact
    active-set QPs; the analytic envelope gradient, or central differences):
    the first `grasps` grasps of workload `wl` for `steps` upper iterations.
    Returns (grasps/s for runs of that length, seconds, threads)."""
    import oracle as O
    hand, obj, x0, T, P, _, _ = I.workload(wl, batch=grasps)
    th = threads or O.default_threads()
    H, Ob = O.Hand(hand), O.Object(obj)
    t0 = time.perf_counter()
    O.run(H, Ob, x0, T, P, n_steps=steps, grad_mode=grad_mode, threads=th)
    dt = time.perf_counter() - t0
    return grasps / dt, dt, th


def paper_sample_size(budget_s: float, threads: int, cap: int = 256) -> int:
    """Grasps of the paper workload whose 200-step oracle run takes about
    `budget_s` on `threads` threads (a multiple of the threads, at most
    `cap`), from a 2-step probe."""
    rate, _, _ = oracle_run("paper", threads, 2, threads=threads)  # grasps/s for 2-step runs
    g = int(budget_s * rate * 2 / N_STEPS)
    return max(threads, min(cap, g // threads * threads))


def cpu_baseline(budget_s: float):
    """The oracle on the host cores: the paper-scale workload (4096 grasps,
    5-finger hand) as one measured 200-step run of up to 256 of its grasps;
    the tiny workload in full, 64 grasps x 50 steps; the differentiation
    workload in full: the evaluation of its 1024 grasps plus central
    differences (h = 1e-6) on its 64 sampled instances; and the paper-scale
    workload on one core."""
    import oracle as O
    th = O.default_threads()
    g = paper_sample_size(budget_s, th)
    rate, dt, _ = oracle_run("paper", g, N_STEPS, threads=th)
    r1, dt1, _ = oracle_run("tiny", 64, 50, threads=th)
    hand, obj, x0, T, P, _, _ = I.workload("grad")
    idx = np.random.default_rng(3).choice(1024, 64, replace=False)
    t0 = time.perf_counter()
    O.evaluate(O.Hand(hand), O.Object(obj), x0, T, P, threads=th)
    O.grad_fd(O.Hand(hand), O.Object(obj), x0[idx], T, P, step=1e-6, threads=th)
    dt3 = time.perf_counter() - t0
    g1 = 2
    rate_1, dt_1, _ = oracle_run("paper", g1, N_STEPS, threads=1)
    return {"value": rate, "unit": "grasps/s", "cores": th, "kind": "oracle",
            "sample": f"paper workload, {g} grasps x {N_STEPS} upper steps (one measured run, exact active-set QPs, "
                      f"analytic envelope gradient), {dt:.1f} s on {th} threads",
            "single_core": {"value": rate_1, "unit": "grasps/s", "cores": 1,
                            "sample": f"{g1} grasps x {N_STEPS} upper steps, {dt_1:.1f} s"},
            "tiny_config_full": {"value": r1, "unit": "grasps/s", "sample": f"64 grasps x 50 upper steps, {dt1:.1f} s"},
            "differentiation_config_full": {"seconds": dt3,
                                            "sample": "1024-grasp evaluation + central differences (h = 1e-6) on 64 "
                                                      "sampled grasps"},
            "paper_context": "49.8 grasps/s for the whole pipeline on one RTX 3090 (Shadow hand, Table 3); "
                             "context only, another machine and pipeline"}


def run_reference(args, rank, world):
    if rank != 0:
        return
    import oracle as O
    th = O.default_threads()
    g = paper_sample_size(6.0, th, cap=128)
    rates, secs = [], []
    for k in range(args.warmup + args.steps):
        rate, dt, _ = oracle_run("paper", g, N_STEPS, threads=th)
        if k >= args.warmup:
            rates.append(rate)
            secs.append(dt)
    value = float(np.mean(rates))
    ms = float(np.mean(secs) * 1e3)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "grasps/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample": f"{g} grasps x {N_STEPS} upper steps per bench step"},
        "cpu_baseline": {"value": value, "unit": "grasps/s", "cores": th, "kind": "oracle",
                         "sample": f"paper workload, {g} grasps x {N_STEPS} upper steps per bench step (measured "
                                   f"200-step runs, exact active-set QPs, analytic envelope gradient)"},
        "e2e": {"value": value, "unit": "grasps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------- GPU path
def run_ours(args, rank, world, local_rank):
    import torch

    import paper_2412_16490_gb300 as bx

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))

    def barrier():
        if dist is not None:
            dist.barrier()

    hand = I.hand_template("hand5")
    obj = I.grid_object(2)
    B = B_PER_GPU
    x0 = I.initial_poses(hand, obj, B, seed=2 + 1000 * rank)
    T = I.wrench_set(S)
    P = I.default_params()
    H, Ob = bx.Hand(hand), bx.Object(obj)
    sp = bx.step_params(P, qp=bx.qp_params(max_iter=ADMM_ITERS, eps_abs=0.0))
    st = bx.State(H, B, S)
    x_dev = torch.as_tensor(x0).cuda()
    T_dev = torch.as_tensor(T).cuda()
    E_dev = torch.empty(B, device="cuda")
    stat_dev = torch.empty(B, dtype=torch.int32, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()

    n_up = args.upper_steps
    if args.mixed_only:  # one persistent launch of the mixed-template batch (profiler captures)
        jobs, T = I.mixed_workload(seed=4)
        Tt = torch.as_tensor(T).cuda()
        sp_m = bx.step_params(P, qp=bx.qp_params(max_iter=ADMM_ITERS), work_pulling=int(args.work_pulling))
        hands, table = {}, []
        for hand_t, obj_t, xj in jobs:
            Hj = hands.setdefault(hand_t.name, bx.Hand(hand_t))
            stj = bx.State(Hj, xj.shape[0], T.shape[0])
            stj.set_pose(torch.as_tensor(xj).cuda())
            table.append(dict(hand=Hj, obj=bx.Object(obj_t), state=stj, T=Tt, n_steps=n_up))
        for _ in range(2):  # warm-up, then the launch a capture skips to
            bx.bodex_step_multi(table, sp_m)
        torch.cuda.synchronize()
        if rank == 0:
            print(json.dumps({"workload": f"mixed templates, {sum(j.shape[0] for _, _, j in jobs)} grasps, "
                                          f"{n_up} upper steps per launch", "launches": 2}))
        return
    if args.exact_step_only:  # two fused runs with exact QPs (a small command for profiler captures)
        sp_x = bx.step_params(P, qp=bx.qp_params(max_iter=64, solver=bx.QP_EXACT))
        for _ in range(2):
            st.set_pose(x_dev)
            bx.bodex_step(H, Ob, st, T_dev, n_up, sp_x, E_last=E_dev, status=stat_dev)
        torch.cuda.synchronize()
        if rank == 0:
            print(json.dumps({"workload": f"paper workload, {n_up} upper steps with exact QPs", "launches": 2}))
        return
    if args.setup_only:  # the fused step's set-up phases alone (a small command for profiler captures)
        sp_0 = bx.step_params(P, qp=bx.qp_params(max_iter=0, eps_abs=0.0))
        for _ in range(2):
            st.set_pose(x_dev)
            bx.bodex_step(H, Ob, st, T_dev, n_up, sp_0, E_last=E_dev, status=stat_dev)
        torch.cuda.synchronize()
        if rank == 0:
            print(json.dumps({"workload": f"paper workload, {n_up} upper steps at 0 ADMM iterations", "launches": 2}))
        return
    if args.qp_exact_only:  # the exact QP solver alone (a small command for profiler captures)
        line = qp_exact_rate(bx, torch, H, Ob, x_dev, T_dev)
        if rank == 0:
            print(json.dumps(dict(line, workload="49152 QPs at the paper geometry, exact solver")))
        return
    if args.qp_only:  # the standalone batched QPs alone (a small command for profiler captures)
        line = qp_solve_rate(bx, torch, H, Ob, x_dev, T_dev)
        if rank == 0:
            print(json.dumps(dict(line, workload="49152 cold-start QPs at the paper geometry, to 1e-5, cap 5000")))
        return

    def one_run():
        st.set_pose(x_dev)
        bx.bodex_step(H, Ob, st, T_dev, n_up, sp, E_last=E_dev, status=stat_dev)

    for _ in range(args.warmup):
        one_run()
    torch.cuda.synchronize()

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    barrier()
    torch.cuda.synchronize()
    with ClockSampler(local_rank) as clk:
        for k in range(args.steps):
            flush.zero_()  # L2 flush between timed steps (outside the events)
            a, k0, k1, b = ev[k]
            a.record(stream)
            st.set_pose(x_dev)
            k0.record(stream)
            bx.bodex_step(H, Ob, st, T_dev, n_up, sp, E_last=E_dev, status=stat_dev)
            k1.record(stream)
            b.record(stream)
        torch.cuda.synchronize()
    barrier()
    step_ms = [a.elapsed_time(b) for a, _, _, b in ev]
    kern_ms = [k0.elapsed_time(k1) for _, k0, k1, _ in ev]
    mean_step = float(np.mean(step_ms))
    if dist is not None:
        t = torch.tensor([mean_step], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        mean_step = float(t.item())
    value = world * B / (mean_step / 1e3) * (n_up / N_STEPS)

    # roofline of the fused step kernel (the only kernel of the timed step)
    fl = flops_per_grasp_step(hand.n_contacts, hand.n_joints, S, ADMM_ITERS) * B * n_up
    kern_s = float(np.mean(kern_ms)) / 1e3
    clocks = clk.summary()
    peaks = measured_peaks()
    sm_max = (clocks or {}).get("sm_max_mhz") or peaks.get("sm_max_mhz") or 2070.0
    peak = fp32_peak_tflops(sm_max)
    achieved = fl / kern_s / 1e12

    # E at the last evaluated pose must have dropped for the run to count
    E_init = bx.bodex_energy_grad(H, Ob, x_dev, T_dev, sp)["E"]
    e_drop = float(torch.median(E_dev / E_init).item())
    nonfinite = int(((stat_dev & bx.ST_NONFINITE) != 0).sum().item())

    extra = {}
    if rank == 0 and not args.quick:
        extra["admm_sweep"] = admm_sweep(bx, torch, H, Ob, x_dev, T_dev, P, B)
        extra["cta_sweep"] = cta_sweep(bx, torch, H, Ob, T_dev, P)
        extra["synthesis"] = synthesis_rate(bx, torch, H, Ob, x_dev, T_dev, sp)
        extra["energies"] = energy_variants(bx, torch, H, Ob, x_dev, T_dev, P)
        extra["exact_qps_200_steps"] = exact_run_rate(bx, torch, H, Ob, x_dev, T_dev, P)
        # the pyramid's QPs with the default fixed penalty; adaptive rho beside it
        extra["qp_solves"] = qp_solve_rate(bx, torch, H, Ob, x_dev, T_dev)
        extra["qp_solves"]["adaptive_rho"] = qp_solve_rate(bx, torch, H, Ob, x_dev, T_dev, adaptive_rho=1)
        extra["qp_solves_elliptic_cone"] = qp_solve_rate(bx, torch, H, Ob, x_dev, T_dev, cone=bx.CONE_ELLIPTIC)
        extra["qp_solves_exact"] = qp_exact_rate(bx, torch, H, Ob, x_dev, T_dev)
        extra["qp_solves_admm_then_exact"] = qp_hybrid_rate(bx, torch, H, Ob, x_dev, T_dev)
        extra["qp_solves_warm_in_loop"] = qp_solve_rate_warm(bx, torch, H, Ob, x_dev, T_dev, P, adaptive_rho=0)
        extra["small_configs"] = small_configs(bx, torch)
        extra["e2e"] = e2e_rate(bx, torch, H, Ob, st, x0, T_dev, sp)
        extra["persistent_mixed"] = persistent_mixed(bx, torch, P)
        if args.serve_jobs > 0:
            extra["serving"] = serving_latency(bx, torch, P, args.serve_jobs)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        extra["cpu_baseline"] = cpu_baseline(args.cpu_seconds)
    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": value, "unit": "grasps/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": mean_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "grasps_per_gpu": B, "upper_steps": N_STEPS, "admm_iters": ADMM_ITERS,
                   "wrenches": S, "l2": "flushed (256 MB write) before each timed step",
                   "parallelism": f"replicas x{world} (independent grasp shards)"},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": TRAFFIC_BYTES if n_up == N_STEPS else None,
                     "traffic_source": TRAFFIC_SOURCE,
                     "kernel": "fused_kernel<5, step> (one launch per 200-step run)",
                     "peak_source": f"FP32 FMA: {sm_count()} SMs x 128 lanes x 2 FLOP x {sm_max:.0f} MHz",
                     "kernel_ms": float(np.mean(kern_ms)), "alg_flops_per_launch": fl},
        "gpu_launches": args.steps,
        "clocks": clocks,
        "energy_ratio_median": e_drop,
        "nonfinite_grasps": nonfinite,
    }
    if "e2e" in extra:
        line["e2e"] = extra.pop("e2e")
    line.update(extra)
    if "serving" in line:
        sv = line["serving"]["exact_qps"]
        cb, pl = sv["continuous_batching"], sv["plain_per_job"]
        line["p50_job_latency_s"], line["p99_job_latency_s"] = cb["p50_s"], cb["p99_s"]
        line["p50_p99_job_latency_plain_per_job_s"] = [pl["p50_s"], pl["p99_s"]]
    if "qp_solves" in line:
        line["qp_solves_per_s"] = line["qp_solves"]["value"]
    print(json.dumps(line), flush=True)


def _timed(torch, fn, reps=3):
    out = []
    for r in range(reps + 1):
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        torch.cuda.synchronize()
        if r:
            out.append(a.elapsed_time(b))
    return float(np.median(out))


def persistent_mixed(bx, torch, P):
    """Mixed-template batch (3-finger/3-contact, 4-finger/4-contact,
    5-finger/5-contact hands; 512 / 2048 / 6144 grasps over six grids of
    48-96 nodes), 200 upper steps: one persistent launch for all jobs; one
    launch per job and upper step; that per-step loop captured once in a
    CUDA graph and replayed -- each with 50 ADMM iterations per step and
    with every QP of every step solved exactly (qp.solver = EXACT: every
    QP at a Frank-Wolfe gap, an upper bound on Q - Q*, of 1e-5 Q + 1e-7,
    which is tighter than a 1e-5 ADMM residual); and the persistent launch
    with the autotuner's pick under each of its two rules (final energy;
    every QP at 1e-5 on 99% of the grasps)."""
    from paper_2412_16490_gb300.autotune import autotune, tuned_params
    jobs, T = I.mixed_workload(seed=4)
    Tt = torch.as_tensor(T).cuda()
    sp = bx.step_params(P, qp=bx.qp_params(max_iter=ADMM_ITERS))
    hands = {}
    J = []
    for hand, obj, x0 in jobs:
        if hand.name not in hands:
            hands[hand.name] = bx.Hand(hand)
        H = hands[hand.name]
        J.append(dict(hand=H, obj=bx.Object(obj), state=bx.State(H, x0.shape[0], 12), T=Tt,
                      x0=torch.as_tensor(x0).cuda(), tpl=hand))
    grasps = sum(int(j["x0"].shape[0]) for j in J)

    def reset():
        for j in J:
            j["state"].set_pose(j["x0"])

    def persistent(params):
        reset()
        bx.bodex_step_multi([dict(j, n_steps=N_STEPS) for j in J], params)

    def per_step(params):
        for _ in range(N_STEPS):
            for j in J:
                bx.bodex_step(j["hand"], j["obj"], j["state"], Tt, 1, params)

    def frac_le(lim):
        return float((torch.cat([j["state"].residual() for j in J]) <= lim).float().mean().item())

    def pulling(params):
        return bx.step_params(P, qp=params.qp, grasps_per_cta=params.grasps_per_cta, work_pulling=1)

    def three_forms(params):
        ms_p = _timed(torch, lambda: persistent(params))
        frac_p = frac_le(1e-5)
        ms_w = _timed(torch, lambda: persistent(pulling(params)))

        def plain():
            reset()
            per_step(params)

        ms_l = _timed(torch, plain, reps=2)
        frac_l = frac_le(1e-5)
        reset()
        per_step(params)  # warm-up outside the capture
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        reset()
        with torch.cuda.graph(g):
            per_step(params)

        def graph():
            reset()
            g.replay()

        ms_g = _timed(torch, graph)
        return {"persistent": {"ms": ms_p, "grasps_per_s": grasps / ms_p * 1e3, "launches": 1,
                               "frac_grasps_all_qps_le_1e-5": frac_p, "schedule": "one block per tile"},
                "persistent_work_pulling": {"ms": ms_w, "grasps_per_s": grasps / ms_w * 1e3, "launches": 1,
                                            "schedule": "grid = resident blocks, tiles from an atomic counter, "
                                                        "costliest jobs first"},
                "per_step_launches": {"ms": ms_l, "grasps_per_s": grasps / ms_l * 1e3, "launches": N_STEPS * len(J),
                                      "frac_grasps_all_qps_le_1e-5": frac_l},
                "per_step_cuda_graph": {"ms": ms_g, "grasps_per_s": grasps / ms_g * 1e3,
                                        "launches": N_STEPS * len(J)}}

    out = {"grasps": grasps, "jobs": len(J), "upper_steps": N_STEPS}
    fixed = three_forms(sp)
    out.update(fixed)  # 50 ADMM iterations per step
    out["exact_qps"] = three_forms(bx.step_params(P, qp=bx.qp_params(max_iter=64, solver=bx.QP_EXACT)))
    big = max(J, key=lambda j: j["x0"].shape[0])
    # tuned on the largest job at its full size: the best CTA tile depends on
    # how many CTAs the launch spreads over the SMs, so a small sample misleads
    for label, rule in (("autotuned_energy", None), ("autotuned_residual_1e-5", 1e-5)):
        t0 = time.perf_counter()
        tuned = autotune(big["hand"], big["obj"], big["x0"], Tt, P, steps=N_STEPS, residual=rule)
        tune_s = time.perf_counter() - t0
        ms_tuned = _timed(torch, lambda: persistent(tuned_params(tuned, P)))
        frac = frac_le(1e-5)
        ms_tw = _timed(torch, lambda: persistent(pulling(tuned_params(tuned, P))))
        out[label] = {"ms": ms_tuned, "grasps_per_s": grasps / ms_tuned * 1e3,
                      "work_pulling_grasps_per_s": grasps / ms_tw * 1e3,
                      "grasps_per_cta": tuned["grasps_per_cta"], "schedule": tuned["schedule"],
                      "rule": "median final energy within 1% of 50 ADMM iterations" if rule is None else
                              "every QP at <= 1e-5 on >= 99% of the grasps",
                      "tuning_job_median_E": tuned["median_E"], "tuning_job_reference_median_E": tuned["reference_median_E"],
                      "frac_grasps_all_qps_le_1e-5": frac, "tune_s": tune_s,
                      "candidates": [dict(tile=t["tile"], schedule=t["schedule"], ms=t["ms"], ok=t["ok"],
                                          frac_res_le_1e5=t["frac_res_le_1e5"]) for t in tuned["table"]]}
    return out


def serving_latency(bx, torch, P, n_jobs):
    """Poisson arrivals (20 jobs/s, seeded) of jobs with 32-128^3 grids, one of
    the three hand templates and 256-4096 grasps x 200 steps, served by the
    continuous-batching server and by one-job-at-a-time per-step launches,
    both with every QP of every step solved exactly (qp.solver = EXACT, each
    QP's Frank-Wolfe gap <= 1e-5 Q + 1e-7: the comparison at a QP accuracy
    of at least 1e-5) and with the fixed 50 ADMM iterations of the bench
    line; the fraction of grasps whose QPs all ended at <= 1e-5 is reported
    with each."""
    from paper_2412_16490_gb300.serving import PlainServer, PoissonWorkload, Server, latency_stats
    t0 = time.perf_counter()
    specs = PoissonWorkload(n_jobs=n_jobs, rate=20.0, seed=5).build()
    build_s = time.perf_counter() - t0
    out = {"arrival_rate_per_s": 20.0, "jobs": n_jobs, "workload_build_s": build_s}
    warm = PoissonWorkload(n_jobs=3, rate=1000.0, seed=6, grid_choices=(32,), grasp_choices=(256,), n_steps=20).build()
    exact = bx.qp_params(max_iter=64, solver=bx.QP_EXACT)
    for label, qp in (("exact_qps", exact), ("fixed_50_iters", bx.qp_params(max_iter=ADMM_ITERS))):
        Server(P, qp=qp).replay(warm, realtime=False)  # load the kernels
        srv = Server(P, qp=qp, steps_per_tick=10)
        cont = latency_stats(srv.replay(specs, realtime=True))
        cont.update(launches=srv.launches, peak_active_jobs=srv.peak_active, steps_per_tick=10)
        pl = PlainServer(P, qp=qp)
        plain = latency_stats(pl.replay(specs, realtime=True))
        plain.update(launches=pl.launches)
        out[label] = {"continuous_batching": cont, "plain_per_job": plain}
    # saturated load: the first 60 jobs all submitted at once (exact QPs)
    qp = exact
    burst = specs[:60]
    for sp in burst:
        sp.arrival = 0.0
    bs = Server(P, qp=qp, steps_per_tick=10)
    b_cont = latency_stats(bs.replay(burst, realtime=False))
    b_cont.update(launches=bs.launches, peak_active_jobs=bs.peak_active)
    bp = PlainServer(P, qp=qp)
    b_plain = latency_stats(bp.replay(burst, realtime=False))
    b_plain.update(launches=bp.launches)
    out["burst_60_jobs_exact_qps"] = {"continuous_batching": b_cont, "plain_per_job": b_plain}
    return out


def admm_sweep(bx, torch, H, Ob, x_dev, T_dev, P, B, steps=50, iters=(0, 25, 50, 100), reps=4):
    """Fused-step time (one launch of `steps` upper iterations) against the
    ADMM iteration count.  The slope is the cost of one ADMM iteration over
    all B*s QPs; the intercept the per-step setup (FK, SDF, G, K^-1, adjoint,
    Adam)."""
    st = bx.State(H, B, S)
    out = {}
    for k in iters:
        sp = bx.step_params(P, qp=bx.qp_params(max_iter=k, eps_abs=0.0))
        ts = []
        for r in range(reps):
            st.set_pose(x_dev)
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            bx.bodex_step(H, Ob, st, T_dev, steps, sp)
            b.record()
            torch.cuda.synchronize()
            if r:
                ts.append(a.elapsed_time(b))
        out[k] = float(np.median(ts))
    ks = np.array(iters, float)
    ms = np.array([out[k] for k in iters])
    slope, icpt = np.polyfit(ks, ms, 1)
    us_iter = slope / steps * 1e3
    return {"upper_steps": steps, "ms_by_admm_iters": {str(k): out[k] for k in iters},
            "us_per_admm_iter": us_iter, "setup_us_per_upper_step": icpt / steps * 1e3,
            "admm_tflops": B * S * admm_iter_flops(H.m) / (us_iter * 1e-6) / 1e12}


def cta_sweep(bx, torch, H, Ob, T_dev, P, steps=50, reps=4):
    """ADMM rate of the fused step against the CTAs resident per SM: batches
    of 1, 2, 3 and 4 CTAs (8 grasps each) per SM and the 4096-grasp batch,
    each timed at 0 and 50 ADMM iterations (50 upper steps).  An SM's time
    is set by its busiest warp scheduler, so the rate steps with the largest
    count of warps on one scheduler rather than with the grasps."""
    hand = I.hand_template("hand5")
    obj = I.grid_object(2)
    sms = sm_count()
    out = {}
    for B in (sms * 8, sms * 16, sms * 24, B_PER_GPU, sms * 32):
        x_dev = torch.as_tensor(I.initial_poses(hand, obj, B, seed=2)).cuda()
        st = bx.State(H, B, S)
        ms = {}
        for k in (0, 50):
            sp = bx.step_params(P, qp=bx.qp_params(max_iter=k, eps_abs=0.0))
            ts = []
            for r in range(reps + 1):
                st.set_pose(x_dev)
                torch.cuda.synchronize()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record()
                bx.bodex_step(H, Ob, st, T_dev, steps, sp)
                b.record()
                torch.cuda.synchronize()
                if r:
                    ts.append(a.elapsed_time(b))
            ms[k] = float(np.median(ts))
        out[str(B)] = {"ctas_per_sm": B / 8 / sms, "ms_0_iters": ms[0], "ms_50_iters": ms[50],
                       "qp_iterations_per_us": B * S * 50 * steps / ((ms[50] - ms[0]) * 1e3)}
        del st
    return {"upper_steps": steps, "grasps_per_cta": 8, "by_grasps": out}


def synthesis_rate(bx, torch, H, Ob, x_dev, T_dev, sp, reps=2):
    """The full three-stage schedule (Sec. IV-D: 300 coarse, 100 fine, 100
    final iterations) on the bench workload, with the Contact Distance
    Consistency (Sec. V-B) of the resulting grasps."""
    bx.synthesize(H, Ob, x_dev, T_dev, sp)  # warm-up
    ts, out = [], None
    for _ in range(reps):
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        out = bx.synthesize(H, Ob, x_dev, T_dev, sp)
        b.record()
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    ms = float(np.median(ts))
    cdc_mm = out["cdc"].double().cpu().numpy() * 1e3
    d_mm = out["d"].double().cpu().numpy() * 1e3
    return {"schedule": "300 coarse + 100 fine + 100 final", "grasps": int(x_dev.shape[0]), "ms": ms,
            "grasps_per_s": x_dev.shape[0] / (ms / 1e3),
            "cdc_mm_median": float(np.median(cdc_mm)), "cdc_mm_p90": float(np.percentile(cdc_mm, 90)),
            "fingertip_penetration_mm_median": float(np.median(np.maximum(0.0, -d_mm.min(1))))}


def exact_run_rate(bx, torch, H, Ob, x_dev, T_dev, P, reps=3):
    """The bench workload's 200-step run with every QP of every step solved
    exactly (qp.solver = EXACT, warm-started from the previous step's working
    set), beside ADMM to a 1e-5 residual in the loop (cap 1000, warm-started)."""
    B = int(x_dev.shape[0])
    st = bx.State(H, B, S)
    E = torch.empty(B, device="cuda")
    out = {}
    for name, qp, r in (("exact", bx.qp_params(max_iter=64, solver=bx.QP_EXACT), reps),
                        ("admm_to_1e-5_cap_1000", bx.qp_params(eps_abs=1e-5, max_iter=1000, check_every=10), 1)):
        sp = bx.step_params(P, qp=qp)
        ts = []
        for k in range(r + 1):
            st.set_pose(x_dev)
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            bx.bodex_step(H, Ob, st, T_dev, N_STEPS, sp, E_last=E)
            b.record()
            torch.cuda.synchronize()
            if k:
                ts.append(a.elapsed_time(b))
        ms = float(np.median(ts))
        out[name] = {"ms": ms, "grasps_per_s": B / (ms / 1e3), "E_last_median": float(E.median().item()),
                     "frac_grasps_all_qps_le_1e-5": float((st.residual() <= 1e-5).float().mean().item())}
    return out


def energy_variants(bx, torch, H, Ob, x_dev, T_dev, P, reps=3):
    """The comparison energies of Sec. V-C in the same fused 200-step run:
    DFC (no QP) and the QP baseline (beta = 0), next to the paper's energy;
    the paper's energy on the elliptic friction cone instead of the pyramid;
    and the paper's energy with the collision-sphere constraint energies of
    Sec. IV-B (penetration, self-penetration, joint limits) switched on."""
    B = int(x_dev.shape[0])
    st = bx.State(H, B, S)
    E = torch.empty(B, device="cuda")
    out = {}
    for name, prm, qp in (("qp_beta1", dict(P), bx.qp_params(max_iter=ADMM_ITERS)),
                          ("qp_baseline_beta0", dict(P, beta=0.0), bx.qp_params(beta=0.0, max_iter=ADMM_ITERS)),
                          ("dfc", dict(P, energy=bx.ENERGY_DFC), bx.qp_params(max_iter=ADMM_ITERS)),
                          ("qp_beta1_elliptic_cone", dict(P), bx.qp_params(max_iter=ADMM_ITERS, cone=bx.CONE_ELLIPTIC)),
                          ("qp_beta1_with_collision_energies",
                           dict(P, w_pen=100.0, w_self=100.0, w_lim=10.0, eta_pen=0.005, eta_lim=0.05),
                           bx.qp_params(max_iter=ADMM_ITERS))):
        sp = bx.step_params(prm, qp=qp)
        ts = []
        for r in range(reps + 1):
            st.set_pose(x_dev)
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            bx.bodex_step(H, Ob, st, T_dev, N_STEPS, sp, E_last=E)
            b.record()
            torch.cuda.synchronize()
            if r:
                ts.append(a.elapsed_time(b))
        ms = float(np.median(ts))
        out[name] = {"ms": ms, "grasps_per_s": B / (ms / 1e3), "E_last_median": float(E.median().item())}
    return out


def qp_solve_rate(bx, torch, H, Ob, x_dev, T_dev, cone=0, adaptive_rho=0):
    """Standalone batched QPs at the paper-scale geometry: B*s = 49152 QPs,
    cold start, iterate to 1e-5 (inf-norm primal and dual), cap 5000; the
    8-facet pyramid or the elliptic cone, fixed or adaptive rho."""
    G = bx.bodex_fk_contacts(H, Ob, x_dev)["G"]
    prm = bx.qp_params(eps_abs=1e-5, max_iter=5000, check_every=10, cone=cone, adaptive_rho=adaptive_rho)
    bx.bodex_qp_solve_batch(G, T_dev, prm)  # warm-up
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    out = bx.bodex_qp_solve_batch(G, T_dev, prm)
    b.record()
    torch.cuda.synchronize()
    dt = a.elapsed_time(b) / 1e3
    conv = ((out["status"] & bx.ST_NOT_CONVERGED) == 0)
    it = out["iters"].float()
    # algorithmic FLOPs of the iterations actually executed (F_it per QP-iteration)
    m = int(G.shape[2]) // 3
    f_it = qp_iteration_flops(m, cone)
    tflops = float(it.sum().item()) * f_it / dt / 1e12
    peak = fp32_peak_tflops((measured_peaks() or {}).get("sm_max_mhz") or 2070.0)
    return {"value": float(conv.sum().item()) / dt, "unit": "QP solves/s (converged to 1e-5)",
            "qps": int(conv.numel()), "converged_frac": float(conv.float().mean().item()),
            "iters_median": float(it.median().item()), "iters_mean": float(it.mean().item()),
            "iters_max": int(it.max().item()), "ms": dt * 1e3,
            "roofline": {"bound": "alu", "achieved": tflops, "peak": peak, "unit": "TFLOP/s", "frac": tflops / peak,
                         "flops_per_qp_iteration": f_it}}


def qp_exact_rate(bx, torch, H, Ob, x_dev, T_dev):
    """The same 49152 QPs solved exactly (qp.solver = EXACT: the float32
    minimum-norm-point method, one QP per thread); a solve counts when the
    oracle-call cap (64) did not stop it.  Its Frank-Wolfe gap, an upper bound
    on Q - Q*, is reported beside it."""
    G = bx.bodex_fk_contacts(H, Ob, x_dev)["G"]
    prm = bx.qp_params(max_iter=64, solver=bx.QP_EXACT)
    bx.bodex_qp_solve_batch(G, T_dev, prm)  # warm-up
    ts, out = [], None
    for _ in range(5):
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        out = bx.bodex_qp_solve_batch(G, T_dev, prm)
        b.record()
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    dt = float(np.median(ts)) / 1e3
    ok = (out["status"] & bx.ST_NOT_CONVERGED) == 0
    it = out["iters"].float()
    gap = out["res"][..., 1]
    Q = out["Q"]
    return {"value": float(ok.sum().item()) / dt, "unit": "exact QP solves/s", "qps": int(ok.numel()),
            "finished_frac": float(ok.float().mean().item()), "oracle_calls_median": float(it.median().item()),
            "oracle_calls_max": int(it.max().item()), "ms": dt * 1e3,
            "gap_within_1e-4Q_plus_1e-6_frac": float((gap <= 1e-4 * Q + 1e-6).float().mean().item())}


def qp_hybrid_rate(bx, torch, H, Ob, x_dev, T_dev, caps=(200, 400, 1000)):
    """The same 49152 QPs: ADMM to 1e-5 with a smaller cap, then the exact
    float32 solve of the QPs it left unconverged (qp.polish = 2).  Every QP
    ends at a 1e-5 residual or exactly solved; each cap is timed, the best
    reported first."""
    G = bx.bodex_fk_contacts(H, Ob, x_dev)["G"]
    runs = []
    for cap in caps:
        prm = bx.qp_params(eps_abs=1e-5, max_iter=cap, check_every=10, polish=2)
        bx.bodex_qp_solve_batch(G, T_dev, prm)  # warm-up
        ts, out = [], None
        for _ in range(5):
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            out = bx.bodex_qp_solve_batch(G, T_dev, prm)
            b.record()
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        dt = float(np.median(ts)) / 1e3
        st = out["status"]
        done = (st & bx.ST_NOT_CONVERGED) == 0
        runs.append({"value": float(done.sum().item()) / dt, "unit": "QP solves/s (1e-5 residual or exact)",
                     "admm_cap": cap, "ms": dt * 1e3, "done_frac": float(done.float().mean().item()),
                     "exact_finished_frac": float(((st & bx.ST_POLISHED) != 0).float().mean().item())})
    runs.sort(key=lambda r: -r["value"])
    return dict(runs[0], other_caps=runs[1:])


def qp_iteration_flops(m, cone=0):
    """F_it of one ADMM iteration: admm_iter_flops for the pyramid; the
    elliptic cone's A has nnz(A) = 5m and nc = 4m + 1 rows."""
    if not cone:
        return admm_iter_flops(m)
    nv, nc, nnz = 3 * m, 4 * m + 1, 5 * m
    return 4 * nnz + 2 * nv * nv + 6 * nv + 10 * nc


def qp_solve_rate_warm(bx, torch, H, Ob, x_dev, T_dev, P, adaptive_rho=1, at_step=100):
    """The in-loop rate: the same 49152 QPs halfway through a 200-step run,
    warm-started from the previous upper step's solution (as the step loop
    does), to 1e-5 (cap 5000).  Poses x_t and x_(t+1) come from the fused
    step loop (50 ADMM iterations per step); the QPs at x_t are solved cold
    first to give the warm start."""
    B, s = x_dev.shape[0], T_dev.shape[0]
    st = bx.State(H, B, s)
    st.set_pose(x_dev)
    sp = bx.step_params(P, qp=bx.qp_params(max_iter=50))
    bx.bodex_step(H, Ob, st, T_dev, at_step, sp)
    x_t = st.pose().clone()
    bx.bodex_step(H, Ob, st, T_dev, 1, sp)
    x_t1 = st.pose().clone()
    cold = bx.qp_params(eps_abs=1e-5, max_iter=5000, check_every=10, adaptive_rho=adaptive_rho)
    prev = bx.bodex_qp_solve_batch(bx.bodex_fk_contacts(H, Ob, x_t)["G"], T_dev, cold)
    G1 = bx.bodex_fk_contacts(H, Ob, x_t1)["G"]
    warm = bx.qp_params(eps_abs=1e-5, max_iter=5000, check_every=10, adaptive_rho=adaptive_rho, warm=1)
    start = lambda: [prev[k].clone() for k in ("y", "z", "lam")]
    bx.bodex_qp_solve_batch(G1, T_dev, warm, *start())  # warm-up
    y, z, lam = start()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    out = bx.bodex_qp_solve_batch(G1, T_dev, warm, y, z, lam)
    b.record()
    torch.cuda.synchronize()
    dt = a.elapsed_time(b) / 1e3
    conv = ((out["status"] & bx.ST_NOT_CONVERGED) == 0)
    it = out["iters"].float()
    cold_it = bx.bodex_qp_solve_batch(G1, T_dev, cold)["iters"].float()
    return {"value": float(conv.sum().item()) / dt, "unit": "QP solves/s (converged to 1e-5, warm start)",
            "qps": int(conv.numel()), "at_upper_step": at_step, "converged_frac": float(conv.float().mean().item()),
            "iters_median": float(it.median().item()), "iters_max": int(it.max().item()),
            "cold_iters_median_same_qps": float(cold_it.median().item()), "ms": dt * 1e3,
            "adaptive_rho": bool(adaptive_rho)}


def small_configs(bx, torch):
    """The two small workloads: the tiny case (64 grasps of the 4-finger
    hand on an analytic sphere, 6 wrenches, 50 upper steps x 30 ADMM
    iterations) as one fused launch, latency-bound by construction (64 grasps
    fill 4 CTAs of 152 SMs, so its roofline fraction means nothing); and the
    autograd path on 1024 grasps of the same hand and object (forward: the
    fused evaluation to a 1e-5 residual; backward: the adjoint kernel)."""
    from paper_2412_16490_gb300.autograd import grasp_energy
    out = {}
    hand, obj, x0, T, P, steps, iters = I.workload("tiny")
    H, Ob = bx.Hand(hand), bx.Object(obj)
    st = bx.State(H, x0.shape[0], T.shape[0])
    x, Td = torch.as_tensor(x0).cuda(), torch.as_tensor(T).cuda()
    sp = bx.step_params(P, qp=bx.qp_params(max_iter=iters))

    def run():
        st.set_pose(x)
        bx.bodex_step(H, Ob, st, Td, steps, sp)

    ms = _timed(torch, run, reps=10)
    out["tiny_64_grasps"] = {"ms": ms, "grasps_per_s": x0.shape[0] / ms * 1e3, "upper_steps": steps,
                             "admm_iters": iters, "note": "latency-bound (4 CTAs); no roofline"}
    hand, obj, x0, T, P, _, iters = I.workload("grad")
    H, Ob = bx.Hand(hand), bx.Object(obj)
    Td = torch.as_tensor(T).cuda()
    sp = bx.step_params(P, qp=bx.qp_params(eps_abs=1e-5, max_iter=5000, check_every=10))
    xg = torch.as_tensor(x0).cuda().requires_grad_(True)

    def fwd_bwd():
        xg.grad = None
        grasp_energy(xg, H, Ob, Td, sp).sum().backward()

    ms = _timed(torch, fwd_bwd, reps=5)
    out["autograd_1024_grasps"] = {"ms": ms, "grasps_per_s": x0.shape[0] / ms * 1e3,
                                   "what": "forward (QPs to 1e-5, cap 5000) + backward (adjoint kernel)"}
    return out


def e2e_rate(bx, torch, H, Ob, st, x0, T_dev, sp, reps=3):
    """Same metric through the public API with host buffers: pinned pose
    upload, the 200-step run, pose + energy download, every step."""
    B = x0.shape[0]
    xh = torch.as_tensor(x0).pin_memory()
    xo = torch.empty_like(xh).pin_memory()
    Eo = torch.empty(B, dtype=torch.float32).pin_memory()
    xd = torch.empty_like(xh, device="cuda")
    Ed = torch.empty(B, device="cuda")
    times = []
    for r in range(reps + 1):
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        xd.copy_(xh, non_blocking=True)
        st.set_pose(xd)
        bx.bodex_step(H, Ob, st, T_dev, N_STEPS, sp, E_last=Ed)
        xo.copy_(st.pose(), non_blocking=True)
        Eo.copy_(Ed, non_blocking=True)
        b.record()
        torch.cuda.synchronize()
        if r > 0:
            times.append(a.elapsed_time(b) / 1e3)
    t = float(np.mean(times))
    return {"value": B / t, "unit": "grasps/s", "h2d_bytes_per_step": int(xh.numel() * 4),
            "d2h_bytes_per_step": int(xo.numel() * 4 + Eo.numel() * 4)}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=30.0,
                    help="time budget of the paper-workload oracle run in the CPU baseline")
    ap.add_argument("--quick", action="store_true", help="skip the QP and e2e side measurements")
    ap.add_argument("--serve-jobs", type=int, default=300, help="jobs in the serving measurement (0 skips it)")
    ap.add_argument("--qp-only", action="store_true", help="only the standalone QP measurement (profiler captures)")
    ap.add_argument("--exact-step-only", action="store_true",
                    help="only two fused runs with exact QPs (profiler captures; --upper-steps sets their length)")
    ap.add_argument("--setup-only", action="store_true",
                    help="only two fused runs at 0 ADMM iterations, i.e. the per-step set-up alone "
                         "(profiler captures; --upper-steps sets their length)")
    ap.add_argument("--qp-exact-only", action="store_true",
                    help="only the exact-solver QP measurement (profiler captures)")
    ap.add_argument("--mixed-only", action="store_true",
                    help="only two persistent launches of the mixed-template batch (profiler captures)")
    ap.add_argument("--work-pulling", action="store_true",
                    help="with --mixed-only: the persistent work-pulling schedule of the several-job launch")
    ap.add_argument("--upper-steps", type=int, default=N_STEPS,
                    help="upper iterations per run (200 for the bench line; fewer for profiler captures)")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", str(args.gpus)))
    if "WORLD_SIZE" not in os.environ:
        world = 1
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
