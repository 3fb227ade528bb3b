"""Benchmark of the fused polar discrete-Boltzmann detonation step on GB300.

A "step" is one time step of the whole update (moments, equilibrium, BGK +
chemical term, upwind streaming, lambda update) over the 2048 x 2048 reactive
implosion in FP32 (33 velocities, 1.4e8 site-velocity updates per step; the
f + lambda state is 0.57 GB per buffer, larger than the 129 MB L2, so no L2
flush is needed between steps).  The metric is GLUPS = 1e9 site x velocity
updates per second, with the HBM roofline of the step kernel beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle (the only other implementation of
the method) on the host cores, on a bounded sample of the same workload.
Under torchrun every rank runs its own replica (the update is one simulation
per GPU; no data-path collective), and rank 0 prints one JSON line.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1308_0653_gb300 import workloads as W  # noqa: E402

METRIC = "GLUPS (site x velocity updates/s)"
UNIT = "GLUPS"
NV = 33
BYTES_PER_SITE = {"fp32": 33 * 4 * 2 + 4 * 2, "fp64": 33 * 8 * 2 + 8 * 2}  # f + lambda, read + write
FALLBACK_HBM_GBS = 6800.0

# DRAM traffic of the FP32 step kernel measured by ncu (dram__bytes_read.sum +
# dram__bytes_write.sum per launch, one-pass capture of the bench workload; the
# summary with its command is in profiles/).  A capture counts only while the
# kernel and launch sources still hash to the value it was taken with.
KERNEL_SOURCES = ("dbm_device.cuh", "dbm_launch.h", "dbm_launch_impl.cuh", "dbm_fp32.cu", "dbm_api.cu")
TRAFFIC_CAPTURES = [  # profiles/step_kernel_fp32_v4_implosion2048_dram.md
    {"variant": 4, "nr": 2048, "ntheta": 2048, "bytes": 1105265493,
     "sources_sha256": "bdd051381a23082f4190497647b4570e17454e09f3f6b5838a8776a3eab2dce6"},
]


def kernel_sources_sha256():
    import hashlib
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1308_0653_gb300", "csrc", name), "rb") as fh:
            h.update(name.encode() + b"\0" + fh.read())
    return h.hexdigest()


def measured_traffic(variant, nr, ntheta):
    sha = kernel_sources_sha256()
    for c in TRAFFIC_CAPTURES:
        if (c["variant"], c["nr"], c["ntheta"]) == (variant, nr, ntheta) and c["sources_sha256"] == sha:
            return c["bytes"]
    return None


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=64)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--nr", type=int, default=2048)
    ap.add_argument("--ntheta", type=int, default=2048)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--fp64-steps", type=int, default=40)
    ap.add_argument("--variant", type=int, default=0,
                    help="step-kernel variant; 0 = the library's choice for this size")
    ap.add_argument("--autotune", action="store_true",
                    help="time every variant on a separate handle first and run the fastest")
    ap.add_argument("--mode", choices=["step", "batch", "serve"], default="step",
                    help="step: the default line; batch: 64 uneven instances in one persistent "
                         "launch per step; serve: Poisson arrivals through dbm_submit/dbm_poll")
    ap.add_argument("--instances", type=int, default=64)
    ap.add_argument("--rows-per-item", type=int, default=0,
                    help="theta rows per work item of batches and the server (0 = library default)")
    ap.add_argument("--batch-steps", type=int, default=5000)
    ap.add_argument("--warmup-batch", type=int, default=64)
    ap.add_argument("--rate", type=float, default=20.0)
    ap.add_argument("--max-queue", type=int, default=200,
                    help="server queue bound (requests beyond it are refused and counted)")
    ap.add_argument("--serve-window", type=float, default=30.0,
                    help="seconds of arrivals in each serving run")
    ap.add_argument("--serve-drain", type=float, default=30.0,
                    help="seconds after the window to finish the 0.7 x capacity run's requests")
    ap.add_argument("--no-batch", action="store_true", help="default line without the batch leg")
    ap.add_argument("--no-serve", action="store_true", help="default line without the serving leg")
    ap.add_argument("--smax", type=int, default=20000)
    ap.add_argument("--batch-nmin", type=int, default=128, help="smallest side of a batch instance")
    ap.add_argument("--batch-nmax", type=int, default=1024, help="largest side of a batch instance")
    ap.add_argument("--nmax", type=int, default=2048)
    return ap.parse_args()


def workload(args):
    return W.implosion(args.nr, args.ntheta, nsteps=args.steps, seed=0, precision="fp32")


def config_of(w, args, extra=None):
    cfg = {"workload": f"reactive implosion {w.params['nr']}x{w.params['ntheta']} "
                       "(r in [0.05,1.05], omega1=omega2=2, dt=5e-6, tau=1e-3, seed 0)",
           "nr": w.params["nr"], "ntheta": w.params["ntheta"], "velocities": NV,
           "site_velocity_updates_per_step": w.sites * NV,
           "l2": "inputs larger than L2 (f + lambda state 0.57 GB per buffer vs 129 MB L2); no flush",
           "parallelism": f"replicas x{args.gpus} (one independent simulation per GPU)"}
    if extra:
        cfg.update(extra)
    return cfg


# ---------------------------------------------------------------------------
# distributed helpers (replicas only: the collectives below time the run)
# ---------------------------------------------------------------------------
def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def aggregate(elapsed_s: float, units: float, backend_device=None):
    """Max elapsed and summed units over ranks (identity when not distributed)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return elapsed_s, units
    t = torch.tensor([elapsed_s], dtype=torch.float64, device=backend_device)
    u = torch.tensor([units], dtype=torch.float64, device=backend_device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier()


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu = gpu_id
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        def num(x):
            try:
                return float(x)
            except ValueError:
                return float("nan")
        sm = [num(r[1]) for r in rows]
        smax = max(num(r[2]) for r in rows)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        load = [x for x in sm if x > 0.5 * smax] or sm
        return {"sm_mhz": statistics.median(load), "sm_max_mhz": smax, "reasons": reasons,
                "samples": len(rows), "power_w_max": max(num(r[3]) for r in rows)}


def measured_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs, copy burst)"
    except (OSError, KeyError, ValueError):
        return FALLBACK_HBM_GBS, "fallback 6.8 TB/s"


# ---------------------------------------------------------------------------
# CPU side: the oracle
# ---------------------------------------------------------------------------
def oracle_sample(w, budget_s=12.0, max_rows=None):
    """Time the FP64 oracle on the host cores on a bounded sample: whole time
    steps of the same workload definition (all nr radial sites) on a grid of
    at most max_rows theta rows, as many steps as fit in budget_s.  The cost
    per site-velocity update does not depend on the number of rows."""
    import oracle
    threads = oracle.set_threads(0)
    nth = w.params["ntheta"] if max_rows is None else min(max_rows, w.params["ntheta"])
    sub = W.implosion(w.params["nr"], nth, nsteps=1, seed=0, precision="fp64")
    p = oracle.make_params(**{k: v for k, v in sub.params.items() if k != "precision"})
    f, lam = oracle.init(p, sub.fields)
    t0 = time.perf_counter()
    f, lam, _ = oracle.step(p, f, lam)
    one = time.perf_counter() - t0
    n = max(1, int(budget_s / max(one, 1e-6)) - 1)
    t0 = time.perf_counter()
    for _ in range(n):
        f, lam, _ = oracle.step(p, f, lam)
    el = time.perf_counter() - t0
    upd = sub.sites * NV * n
    return {"value": upd / el / 1e9, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"{n} oracle time steps of the implosion workload definition on a "
                      f"{w.params['nr']}x{nth} grid (same radial sites, {nth} theta rows "
                      f"instead of {w.params['ntheta']}), {el:.1f} s on {threads} threads"}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    w = workload(args)
    # each step: one oracle time step over a row block sized for ~0.05 s
    import oracle
    threads = oracle.set_threads(0)
    probe = oracle_sample(w, budget_s=1.0, max_rows=64)
    rate = probe["value"] * 1e9  # updates/s
    rows = int(max(8, min(w.params["ntheta"], 0.05 * rate / (w.params["nr"] * NV))))
    sub = W.implosion(w.params["nr"], rows, nsteps=1, seed=0, precision="fp64")
    p = oracle.make_params(**{k: v for k, v in sub.params.items() if k != "precision"})
    f, lam = oracle.init(p, sub.fields)
    for _ in range(args.warmup):
        f, lam, _ = oracle.step(p, f, lam)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        f, lam, _ = oracle.step(p, f, lam)
    el = time.perf_counter() - t0
    upd = sub.sites * NV * args.steps
    value = upd / el / 1e9
    sample = (f"each step: one oracle time step of the implosion workload definition on a "
              f"{w.params['nr']}x{rows} grid (same radial sites, {rows} theta rows instead of "
              f"{w.params['ntheta']}), {threads} threads")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_of(w, args, {"reference_rows_per_step": rows}),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# GPU side
# ---------------------------------------------------------------------------
def run_ours(args):
    import torch
    import torch.distributed as dist
    from paper_1308_0653_gb300 import dbm

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1 and not dist.is_initialized():
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    w = workload(args)
    sites = w.sites
    stream = torch.cuda.Stream(device=dev)

    tune = None
    if args.variant == 0 and args.autotune:
        # autotuner: time every kernel variant on a separate handle of the same
        # size; the choice is remembered for this size class (used below)
        t = dbm.Simulation(dict(w.params, precision="fp32"), device=dev)
        t.init_state(w.fields, stream=stream)
        best, ms = t.autotune(steps=20, stream=stream)
        t.close()
        tune = {"variant": best, "ms_per_step": {str(v + 1): round(x, 5) for v, x in enumerate(ms)}}
    sim = dbm.Simulation(dict(w.params, precision="fp32", variant=args.variant), device=dev)
    sim.init_state(w.fields, stream=stream)
    sim.step(args.warmup, stream=stream)
    torch.cuda.synchronize(dev)

    vis = [x for x in os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",") if x.strip()]
    clocks = ClockSampler(vis[local] if local < len(vis) else str(local))
    clocks.start()
    time.sleep(0.3)
    barrier()
    torch.cuda.synchronize(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sim.step(args.steps, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    barrier()
    clk = clocks.stop()
    elapsed = e0.elapsed_time(e1) / 1e3
    mom = sim.moments(stream=stream, raise_nonfinite=False)
    finite = mom["status"] == dbm.DBM_OK
    launch = sim.launch_info()
    elapsed_max, units = aggregate(elapsed, float(sites) * NV * args.steps,
                                   backend_device=dev if ws > 1 else None)
    value = units / elapsed_max / 1e9

    # roofline of the step kernel (the only kernel in the timed region)
    per_launch = elapsed / args.steps
    alg_bytes = BYTES_PER_SITE["fp32"] * sites
    achieved = alg_bytes / per_launch / 1e9
    peak, peak_src = measured_peak()
    kname = {1: "dbm::step_kernel<float,128,6> (v1, row barrier)",
             2: "dbm::step_kernel_v2<float,128,6,false,2,false> (bulk copies)",
             3: "dbm::step_kernel_v2<float,128,4,true,3,false> (bulk copies)",
             4: "dbm::step_kernel_v2<float,128,6,false,2,true> (tensor-map TMA)",
             5: "dbm::step_kernel_v2<float,128,4,true,3,true> (tensor-map TMA)"}.get(
                 launch["variant"], f"variant {launch['variant']}")
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "traffic": measured_traffic(launch["variant"], w.params["nr"],
                                                                 w.params["ntheta"]),
            "kernel": kname,
            "algorithmic_bytes_per_launch": alg_bytes, "launch_ms": per_launch * 1e3,
            "peak_source": peak_src}
    sim.close()

    # FP64 path on the same workload (ALU-bound on GB300), for the FP32 vs FP64 ratio
    fp64 = None
    if args.fp64_steps > 0:
        s64 = dbm.Simulation(dict(w.params, precision="fp64", variant=args.variant), device=dev)
        s64.init_state(w.fields, stream=stream)
        s64.step(4, stream=stream)
        torch.cuda.synchronize(dev)
        e0.record(stream)
        s64.step(args.fp64_steps, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        el64 = e0.elapsed_time(e1) / 1e3
        fp64 = {"value": sites * NV * args.fp64_steps / el64 / 1e9, "unit": UNIT,
                "steps": args.fp64_steps, "variant": s64.launch_info()["variant"]}
        s64.close()

    # end to end through the C ABI with pinned host buffers: init from host,
    # K time steps, moments back to host (one solve; copies inside the timing)
    e2e = None
    if not args.no_e2e:
        pinned = {k: torch.from_numpy(w.fields[k]).pin_memory() for k in dbm.FIELDS}
        host_in = {k: v.numpy() for k, v in pinned.items()}
        outs = {k: torch.empty(w.fields[k].shape, dtype=torch.float64).pin_memory().numpy()
                for k in dbm.FIELDS}
        tot = np.zeros(4)
        sim = dbm.Simulation(dict(w.params, precision="fp32", variant=args.variant), device=dev)
        sim.init_state(host_in, stream=stream)  # warm the path once
        sim.step(GRAPH_WARM, stream=stream)
        torch.cuda.synchronize(dev)
        barrier()
        t0 = time.perf_counter()
        dbm.dbm_init_state(sim.h, *[host_in[k] for k in dbm.FIELDS], stream=stream)
        dbm.dbm_step(sim.h, args.steps, stream)
        dbm.dbm_moments(sim.h, *[outs[k] for k in dbm.FIELDS], totals=tot, stream=stream)
        t_e2e = time.perf_counter() - t0
        # A stream of independent solves through the same calls, two handles on
        # two streams: solve i's upload (dbm_init_state) and solve i - 1's
        # download (dbm_moments) run on the copy engines while the other
        # handle's steps run on the SMs.
        sim2 = dbm.Simulation(dict(w.params, precision="fp32", variant=args.variant), device=dev)
        stream2 = torch.cuda.Stream(device=dev)
        sim2.init_state(host_in, stream=stream2)
        sim2.step(GRAPH_WARM, stream=stream2)
        outs2 = {k: torch.empty(w.fields[k].shape, dtype=torch.float64).pin_memory().numpy()
                 for k in dbm.FIELDS}
        pair = ((sim, stream, outs), (sim2, stream2, outs2))
        n_pipe = 6
        torch.cuda.synchronize(dev)
        barrier()
        t0 = time.perf_counter()
        for i in range(n_pipe + 1):
            if i < n_pipe:
                h, st_i, _ = pair[i % 2]
                dbm.dbm_init_state(h.h, *[host_in[k] for k in dbm.FIELDS], stream=st_i)
                dbm.dbm_step(h.h, args.steps, st_i)
            if i > 0:
                h, st_i, o = pair[(i - 1) % 2]
                dbm.dbm_moments(h.h, *[o[k] for k in dbm.FIELDS], totals=tot, stream=st_i)
        t_pipe = time.perf_counter() - t0
        barrier()
        sim2.close()
        sim.close()
        t_e2e_max, units_e2e = aggregate(t_e2e, float(sites) * NV * args.steps,
                                         backend_device=dev if ws > 1 else None)
        t_pipe_max, units_pipe = aggregate(t_pipe, float(sites) * NV * args.steps * n_pipe,
                                           backend_device=dev if ws > 1 else None)
        h2d = 5 * sites * 8
        d2h = 5 * sites * 8 + 4 * 8 + 4
        e2e = {"value": units_e2e / t_e2e_max / 1e9, "unit": UNIT,
               "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": d2h / args.steps,
               "solve": {"time_steps": args.steps, "h2d_bytes": h2d, "d2h_bytes": d2h,
                         "seconds": t_e2e,
                         "calls": "dbm_init_state(host) + dbm_step(K) + dbm_moments(host)"},
               "pipelined": {"value": units_pipe / t_pipe_max / 1e9, "unit": UNIT, "solves": n_pipe,
                             "seconds": t_pipe,
                             "how": "the same calls for a stream of independent solves, two handles on "
                                    "two streams: each solve's host copies overlap the other handle's "
                                    "steps; every solve's inputs are uploaded and its fields read back"}}

    # batched and served legs (one GPU: their figures are per GPU)
    single = batch = serve = None
    if args.gpus == 1 and not (args.no_batch and args.no_serve):
        single = single_instance_glups(stream)
        if not args.no_batch:
            batch = batch_leg(args, single)
        if not args.no_serve:
            serve = serve_leg(args, single)

    cpu = None
    if rank == 0 and args.gpus == 1 and not args.no_cpu_baseline:
        cpu = oracle_sample(w, budget_s=12.0, max_rows=256)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
                "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": elapsed_max / args.steps * 1e3, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": config_of(w, args, {"launch": launch, "autotune": tune}),
                "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "clocks": clk,
                "gpu_launches": args.steps, "fp64": fp64,
                "fp32_over_fp64": (value / args.gpus / fp64["value"]) if fp64 else None,
                "state_finite": bool(finite), "batch": batch, "serve": serve}
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()
    return 0


GRAPH_WARM = 64


def single_instance_glups(stream, steps=500):
    """FP32 GLUPS of one 2048^2 implosion alone (the default step workload),
    measured in the same process, for the batched and served ratios."""
    import torch
    from paper_1308_0653_gb300 import dbm
    w1 = W.implosion(2048, 2048, nsteps=0)
    s1 = dbm.Simulation(dict(w1.params, precision="fp32"))
    s1.init_state(w1.fields, stream=stream)
    s1.step(64, stream=stream)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    s1.step(steps, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    s1.close()
    return w1.sites * NV * steps / (e0.elapsed_time(e1) / 1e3) / 1e9


def batch_leg(args, single):
    """64 uneven square instances (N in [128, 1024], seeded) advanced together,
    one persistent launch per step, against the same instances one by one and
    against `single` (GLUPS of one 2048^2 instance alone)."""
    import torch
    from paper_1308_0653_gb300 import dbm
    ws = W.batch(args.instances, seed=0, nsteps=args.batch_steps, nmin=args.batch_nmin,
                 nmax=args.batch_nmax, align=1)
    sites = sum(w.sites for w in ws)
    stream = torch.cuda.Stream()
    sims = []
    for w in ws:
        s = dbm.Simulation(dict(w.params, precision="fp32"))
        s.init_state(w.fields, stream=stream)
        sims.append(s)
    b = dbm.Batch(len(ws), 1 << 22, precision="fp32", rows_per_item=args.rows_per_item)
    tune_steps = 64
    for k, s in enumerate(sims):
        b.attach(k, s, args.batch_steps + 8 * (32 + 2 * tune_steps))
    tune = None
    if args.rows_per_item == 0:
        # batch autotuner on the live batch: kernel x rows per item
        v, r, ms = b.autotune(steps=tune_steps, stream=stream)
        names = [f"v{vv}/r{rr}" for vv in (4, 2) for rr in (16, 32, 64, "scaled")]
        tune = {"variant": v, "rows_per_item": r,
                "ms_per_step": {n: round(x, 4) for n, x in zip(names, ms) if x > 0}}
    b.step(args.warmup_batch, stream=stream)
    torch.cuda.synchronize()
    info = b.launch_info()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    steps = args.batch_steps - args.warmup_batch
    e0.record(stream)
    b.step(steps, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    el = e0.elapsed_time(e1) / 1e3
    batched = sites * NV * steps / el / 1e9
    b.close()
    # the same instances one at a time (a few steps each), for the ratio
    t_one = 0.0
    k1 = 64
    for s in sims:
        s.step(2, stream=stream)
        e0.record(stream)
        s.step(k1, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        t_one += e0.elapsed_time(e1) / 1e3 / k1
    alone = sites * NV / t_one / 1e9
    for s in sims:
        s.close()
    return {"metric": METRIC + ", batched sweep", "value": batched, "unit": UNIT,
            "steps": steps, "warmup": args.warmup_batch, "ms_per_step": el / steps * 1e3,
            "workload": f"{len(ws)} instances, N x N with N uniform in [{args.batch_nmin}, "
                        f"{args.batch_nmax}] (seed 0), explosion/implosion alternating, shock ratio "
                        "logU[1.2, 3], omega1 logU[0.5, 8]; one persistent launch per step, CUDA "
                        "graph of 32 steps",
            "sites": sites, "launch": info, "autotune": tune,
            "one_by_one": {"value": alone, "unit": UNIT,
                           "how": "each instance alone, 64 graph-replayed steps, summed time"},
            "batched_over_one_by_one": batched / alone,
            "single_instance": {"value": single, "unit": UNIT,
                                "workload": "reactive implosion 2048x2048, 500 steps, same process"},
            "batched_over_single_instance": batched / single}


def mean_request_updates(seed=0, nmax=2048, smax=20000, n=4000):
    """Expected site x velocity updates of one serving request (mean over the
    first n requests of the stream's shapes)."""
    tot = 0.0
    for k in range(n):
        N, steps, _, _ = W.serving_shape(k, seed=seed, nmax=nmax, smax=smax)
        tot += N * N * NV * steps
    return tot / n


def serve_run(rate, duration, args, drain_s):
    """Poisson arrivals at `rate` for `duration` s through dbm_submit /
    dbm_poll; results are collected until every accepted request is done or
    drain_s after the window.  Returns the run's figures."""
    import torch
    from paper_1308_0653_gb300 import dbm
    free, total = torch.cuda.mem_get_info()
    pool = int(min(free * 0.8, 150e9))
    # The server copies each request's initial fields until it is admitted, so
    # the queue is bounded (requests beyond it are refused with DBM_EBUSY and
    # counted): under sustained overload an unbounded queue grows by ~30 MB of
    # host memory per request.
    srv = dbm.Server(pool_bytes=pool, max_slots=64, max_queue=args.max_queue, quantum=64,
                     max_items=1 << 20, rows_per_item=args.rows_per_item)
    arr = W.arrivals(rate, duration, seed=0)
    t0 = time.perf_counter()
    pending = []   # (ticket, sites): the fields are not kept here
    n_accepted = 0
    offered = 0.0
    refused = 0
    lat, upd = [], 0.0

    def collect(timeout_us):
        # results are taken (and their host copies freed) as soon as they are ready
        nonlocal pending, upd
        keep = []
        for t, sites in pending:
            st, res = srv.poll(t, timeout_us=timeout_us())
            if st == dbm.DBM_OK:
                if res["status"] == dbm.DBM_OK:
                    lat.append(res["t_end"] - res["t_submit"])
                    upd += sites * NV * res["steps"]
            else:
                keep.append((t, sites))
        pending = keep

    last = 0.0
    for k, ta in enumerate(arr):
        w = W.serving_request(k, seed=0, nmax=args.nmax, smax=args.smax)
        offered += w.sites * NV * w.nsteps
        while time.perf_counter() - t0 < ta:
            if time.perf_counter() - last > 0.5:
                collect(lambda: 0)
                last = time.perf_counter()
            time.sleep(0.001)
        try:
            pending.append((srv.submit(dict(w.params, precision="fp32"), w.fields, w.nsteps), w.sites))
            n_accepted += 1
        except dbm.DbmError as e:
            if e.status != dbm.DBM_EBUSY:
                raise
            refused += 1
        del w
    while time.perf_counter() - t0 < duration:
        collect(lambda: 0)
        time.sleep(0.05)
    window = time.perf_counter() - t0
    stats_w = srv.stats()
    # then drain: what is still not done after drain_s is the backlog
    collect(lambda: int(max(duration + drain_s - (time.perf_counter() - t0), 0) * 1e6))
    wall = time.perf_counter() - t0
    stats = srv.stats()
    srv.close()
    lat = np.array(lat) if lat else np.array([np.nan])
    done = int(np.isfinite(lat).sum())
    return {"rate_per_s": rate, "window_s": duration, "requests": len(arr), "accepted": n_accepted,
            "refused_queue_full": refused, "completed": done, "backlog": n_accepted - done,
            "p50_s": float(np.nanpercentile(lat, 50)), "p99_s": float(np.nanpercentile(lat, 99)),
            "executed_glups_window": stats_w["executed"] / window / 1e9,
            "executed_glups": stats["executed"] / wall / 1e9,
            "completed_glups": upd / wall / 1e9, "offered_glups": offered / duration / 1e9,
            "wall_s": wall, "pool_bytes": pool, "server_status": stats["status"]}


def serve_leg(args, single):
    """Two serving runs of the config-5 request stream (side logU[128, 2048],
    steps logU[1e3, 2e4], explosion/implosion 50/50): at its 20 req/s, which
    overloads the GPU about five times (sustained throughput; latencies are
    queue-dominated), then at 0.7 x the capacity that run measured
    (time to solution)."""
    over = serve_run(args.rate, args.serve_window, args, drain_s=0.0)
    mean_upd = mean_request_updates(nmax=args.nmax, smax=args.smax)
    capacity = over["executed_glups_window"] * 1e9 / mean_upd
    light = serve_run(0.7 * capacity, args.serve_window, args, drain_s=args.serve_drain)
    return {"metric": METRIC + ", served", "unit": UNIT,
            "value": over["executed_glups_window"],
            "executed_over_single_instance": over["executed_glups_window"] / single,
            "single_instance": {"value": single, "unit": UNIT,
                                "workload": "reactive implosion 2048x2048, 500 steps, same process"},
            "workload": f"Poisson arrivals, side logU[128, {args.nmax}], steps logU[1000, {args.smax}], "
                        "explosion/implosion 50/50, omega1 in {1, 2, 4}; max 64 resident, "
                        f"queue bounded at {args.max_queue}, quantum 64 steps",
            "mean_request_updates": mean_upd, "capacity_req_per_s": capacity,
            "overload": over, "at_0.7_capacity": light}


def run_batch(args):
    import torch
    torch.cuda.set_device(0)
    single = single_instance_glups(torch.cuda.Stream())
    leg = batch_leg(args, single)
    leg.update({"n_gpus": 1, "higher_is_better": True, "dtype": "f32", "data": "synthetic"})
    print(json.dumps(leg), flush=True)
    return 0


def run_serve(args):
    import torch
    torch.cuda.set_device(0)
    single = single_instance_glups(torch.cuda.Stream())
    leg = serve_leg(args, single)
    leg.update({"n_gpus": 1, "higher_is_better": True, "dtype": "f32", "data": "synthetic"})
    print(json.dumps(leg), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.mode == "batch":
        return run_batch(args)
    if args.mode == "serve":
        return run_serve(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
