"""Benchmark: interface Monte Carlo mesh steps of the large ring workload on GB300.

Workload (one "step" = one mesh step of the method, Sec. 4): w = 1 + 50
exp(-(r - 0.25 - 0.1 sin 2 pi t)^2 / 0.02^2), r = |(x, y) - (1/2, 1/2)|, on a
2049 x 2049 FP32 grid sampled at t_{n-1}, 8 x 8 subdomains, the 28,609
interface nodes with 2e4 paths each, dt = 1e-5, Delta t = 1e-3 (100
sub-steps), the paper's boundary test; then the FP64 implicit subdomain
solves. The default run times the workload's 20 mesh steps, then the same
steps with the two control variates (the previous fields' gradient and the
learned network) against the plain estimator on the same state.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload ring2049|front257|batch64|heat65|cv65|ring41|exit65]

Prints one JSON line (rank 0). Metric: Euler--Maruyama path-steps per second
over whole mesh steps (interface nodes per second alongside). Each rank runs
its own instance (its own seed); the ranks share no data.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as W  # noqa: E402

METRIC = "path-steps/s (interface Monte Carlo, whole mesh steps)"
UNIT = "path-steps/s"
# The mesh-step workloads: (inputs, w at time t, description)
WORKLOADS = {
    "ring2049": (W.RING2049, W.w_ring,
                 "w=1+50exp(-(r-0.25-0.1sin(2pi t))^2/0.02^2) on 2049x2049 FP32, 8x8 subdomains"),
    "front257": (W.FRONT257, W.w_front, "w=1+10exp(-(x-0.3-0.4t)^2/0.05^2) on 257x257 FP32, 2x2 subdomains"),
}
DEFAULT_WORKLOAD = "ring2049"
# Algorithmic lane operations per path-step of the path kernel, counted per
# coordinate: half a Philox4x32-10 block (10 rounds x 2 wide multiplies + 2
# three-input xors, over two sub-steps: 20), one Box-Muller pair (12), cell
# location (12), bilinear drift (6), Euler-Maruyama update (4), exit test (4).
ALG_OPS_PER_PATH_STEP = 58
SM_LANES_PER_CLK = 128       # 4 schedulers x 32 lanes issue per SM per clock


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None, help="timed mesh steps (default: the workload's)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-cv", action="store_true", help="skip the control-variate measurements")
    ap.add_argument("--no-model", action="store_true", help="skip the learned control variate's measurement")
    ap.add_argument("--cv-order", type=int, default=0,
                    help="binomial smoothing order of the field-gradient control variate (0: the library's choice)")
    ap.add_argument("--paths", type=int, default=None)
    ap.add_argument("--workload", choices=["ring2049", "front257", "batch64", "heat65", "cv65", "ring41", "exit65"],
                    default=DEFAULT_WORKLOAD)
    ap.add_argument("--key-spacing", type=int, default=8,
                    help="ring41: key points plus every k-th node (k > 0), key points only (0), every node (-1)")
    ap.add_argument("--solver", choices=["auto", "jacobi", "mg", "direct"], default="auto",
                    help="subdomain solver of the mesh steps")
    ap.add_argument("--no-pipeline", action="store_true",
                    help="run each step's subdomain solve after its paths instead of beside the next step's")
    ap.add_argument("--estimate-only", action="store_true",
                    help="time the interface estimate alone (no mesh-step graph) on every --node-stride-th "
                         "interface node of the first mesh step: the path kernel outside any graph, for profiling")
    ap.add_argument("--node-stride", type=int, default=1)
    ap.add_argument("--shape", default=None,
                    help="--estimate-only: block_threads,paths_per_task,zero_map (1 on, 2 off); default: autotuned")
    ap.add_argument("--cv", choices=["off", "fields", "model"], default="off",
                    help="--estimate-only: control variate of the estimate")
    return ap.parse_args()


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def dist_init(backend=None):
    """One process per GPU under torchrun: NCCL where there is a GPU, else gloo (host tensors)."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        if backend is None:
            backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def allreduce(vals, op, world):
    if world == 1:
        return vals
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor(vals, dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return t.tolist()


def whole_job(units, seconds, world):
    """Whole-job throughput: the units every rank processed over the slowest rank's time.
    Returns (units / s, total units, max seconds)."""
    tot = allreduce([float(units)], "sum", world)[0]
    mx = allreduce([float(seconds)], "max", world)[0]
    return tot / mx, tot, mx


# ------------------------------------------------------------------ oracle leg

class OracleSampler:
    """The FP64 oracle's interface estimate on seeded samples of a workload's nodes,
    one mesh step's w per call (fields of the uniform mesh, xi0 = x, eta0 = y)."""

    def __init__(self, name):
        import oracle
        oracle.build()
        self.oracle = oracle
        self.wl, self.wfun, _ = WORKLOADS[name]
        n = self.wl.n
        self.xs, self.ys = W.interface_node_coords(n, n, self.wl.sub, self.wl.sub)
        self.ids = np.arange(self.xs.size, dtype=np.uint32)
        self.xi0, self.eta0 = W.identity_fields(n)
        self.problems = {}
        self.rng = np.random.default_rng(12345)

    def problem(self, k):
        k = k % self.wl.steps
        if k not in self.problems:
            if len(self.problems) > 2:
                self.problems.clear()
            self.problems[k] = self.oracle.Problem(self.wfun(self.wl.n, k * self.wl.Dt), self.xi0, self.eta0)
        return self.problems[k]

    def call(self, k, nodes, threads=None):
        """One oracle estimate at `nodes` seeded random interface nodes of mesh step k:
        (path-steps, seconds)."""
        pick = np.sort(self.rng.choice(self.xs.size, size=min(nodes, self.xs.size), replace=False))
        P = self.problem(k)
        t0 = time.perf_counter()
        r = self.oracle.interface_mc(P, self.xs[pick], self.ys[pick], self.wl.paths, dt=self.wl.dt, Dt=self.wl.Dt,
                                     seed=0, step_index=k, node_ids=self.ids[pick], threads=threads)
        return int(r["path_steps"].sum()), time.perf_counter() - t0

    def timed(self, target_s, nodes, threads=None):
        """Calls of `nodes` nodes, mesh step after mesh step, until target_s seconds of oracle time."""
        steps, el, calls = 0, 0.0, 0
        while el < target_s or calls == 0:
            a, b = self.call(calls, nodes, threads)
            steps += a
            el += b
            calls += 1
        return steps, el, calls


def cpu_baseline(name):
    """The oracle on the host cores, all of them and one, on seeded node samples
    (about 10 s of oracle work each); throughput per path-step."""
    S = OracleSampler(name)
    wl = S.wl
    cores = os.cpu_count() or 1
    S.call(0, 1)   # the first step's tables, outside the timing
    nodes_all = max(1, min(S.xs.size, 4 * cores))
    st_a, el_a, calls_a = S.timed(10.0, nodes_all)
    st_1, el_1, calls_1 = S.timed(10.0, 2, threads=1)
    return {"value": st_a / el_a, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{calls_a} call(s) of {nodes_all} seeded random interface nodes of the {name} mesh steps x "
                      f"{wl.paths} paths ({st_a} path-steps in {el_a:.1f} s, all {cores} cores, one thread per node "
                      f"chunk); the rate per path-step carries over to the whole workload",
            "single_thread": {"value": st_1 / el_1, "unit": UNIT, "cores": 1,
                              "sample": f"{calls_1} call(s) of 2 nodes ({st_1} path-steps in {el_1:.1f} s)"}}


def run_reference(args, world, rank):
    if rank != 0:
        return
    name = args.workload if args.workload in WORKLOADS else DEFAULT_WORKLOAD
    S = OracleSampler(name)
    wl = S.wl
    cores = os.cpu_count() or 1
    K = args.steps or wl.steps
    per_call_nodes = 2 * cores
    # untimed warm-up, then K timed steps (each: the oracle's estimate at a node sample of one mesh step)
    for k in range(max(1, args.warmup)):
        S.call(k, 1)
    steps_done, el = 0, 0.0
    for k in range(K):
        a, b = S.call(k, per_call_nodes)
        steps_done += a
        el += b
    value = steps_done / el
    desc = WORKLOADS[name][2]
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": K,
        "warmup": args.warmup, "ms_per_step": 1e3 * el / K, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "impl": "reference",
        "config": {"workload": f"{name}: {desc}, interface estimate at {per_call_nodes} seeded random interface "
                               f"nodes per mesh step, {wl.paths} paths/node, dt={wl.dt}, Dt={wl.Dt} (K={wl.K})",
                   "global_batch": per_call_nodes * wl.paths, "seq_len": wl.K, "parallelism": "cpu threads"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{per_call_nodes} seeded random interface nodes x {wl.paths} paths per mesh step"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ GPU leg

def profiled_counters(path):
    """From a committed ncu summary: DRAM bytes per launch, the path-steps of
    that launch and the issue-slot utilisation (smsp__issue_active, a
    fraction), or None when the kernel's sources changed since the counters
    were taken."""
    import hashlib
    import re
    try:
        lines = open(path).read().splitlines()
    except OSError:
        return None
    fields = dict(l.split(": ", 1) for l in lines if ": " in l and l.split(": ", 1)[0] in
                  ("dram_bytes_per_launch", "path_steps_per_launch", "source_sha256", "sources"))
    if not {"dram_bytes_per_launch", "source_sha256", "sources"} <= fields.keys():
        return None
    h = hashlib.sha256()
    for f in fields["sources"].split(", "):
        try:
            h.update(open(os.path.join(ROOT, f), "rb").read())
        except OSError:
            return None
    if h.hexdigest() != fields["source_sha256"]:
        return None
    issue = None
    for l in lines:
        m = re.search(r"`smsp__issue_active\.avg\.pct_of_peak_sustained_active`\) \| ([0-9.]+) %", l)
        if m:
            issue = float(m.group(1)) / 100.0
    return {"dram_bytes_per_launch": float(fields["dram_bytes_per_launch"]),
            "path_steps_per_launch": float(fields["path_steps_per_launch"]) if "path_steps_per_launch" in fields else None,
            "issue_slots": issue}


def run_ours(args, world, rank, local):
    import torch

    import paper_1402_0266_gb300 as sdd
    from paper_1402_0266_gb300 import build as b
    b.build()
    name = args.workload
    WL, wfun, desc = WORKLOADS[name]
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    n, Wm = WL.n, args.warmup
    K = args.steps or WL.steps
    paths = args.paths or WL.paths
    seed = WL.seed + rank
    stream = torch.cuda.current_stream()
    xi0, eta0 = W.identity_fields(n)
    xi0_d = torch.from_numpy(xi0).to(dev)
    eta0_d = torch.from_numpy(eta0).to(dev)
    # the mesh density of every step, resident on the device before timing
    nsteps = max(K, Wm, 1)
    w_host = torch.from_numpy(np.stack([wfun(n, k * WL.Dt) for k in range(nsteps)]))
    w_all = w_host.to(dev)
    ctx = sdd.sdd_init(n, n, WL.sub, WL.sub, w=w_all[0], xi0=xi0_d, eta0=eta0_d)
    sdd.sdd_set_solver(ctx, {"auto": 0, "jacobi": 1, "mg": 2, "direct": 3}[args.solver])
    sdd.sdd_set_pipeline(ctx, not args.no_pipeline)
    sp = dict(dt=WL.dt, Dt=WL.Dt, seed=seed, paths_per_node=paths, exit_mode=0, rtol=1e-12, max_iter=40000, tune=1)

    def reset():
        sdd.sdd_set_fields(ctx, xi0_d, eta0_d)
        sdd.sdd_set_step_index(ctx, 0)

    # the launch shape of the steps' path kernel: the autotuner's choice for the interface node set
    # (the steps find it in the context's cache)
    ix, iy = sdd.sdd_interface_nodes(ctx)
    shape = sdd.sdd_autotune(ctx, ix, iy, np.full(len(ix), paths), WL.dt, WL.Dt)
    for k in range(Wm):
        sdd.sdd_set_w(ctx, w_all[k % nsteps])
        sdd.sdd_step(ctx, **sp)
    sdd.sdd_sync(ctx)
    reset()

    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # > L2 (129 MB)
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    steps_dev = torch.zeros(K, dtype=torch.int64, device=dev)
    paths_ms, est_ms, solve_ms = [], [], []
    kernel_nodes = 0
    clocks = ClockSampler(local)
    barrier(world)
    torch.cuda.synchronize()
    clocks.start()
    torch.cuda.nvtx.range_push("timed_steps")
    for k in range(K):
        flush.zero_()
        ev0[k].record(stream)
        sdd.sdd_set_w(ctx, w_all[k])
        sdd.sdd_step(ctx, **sp)
        if k == K - 1:
            # the last step's deferred solve iterations run inside the timed region too
            sdd.sdd_flush(ctx)
        ev1[k].record(stream)
        st = sdd.sdd_last_interface_stats(ctx)
        steps_dev[k] = st["path_steps"].sum()
        info = sdd.sdd_last_step_info(ctx)   # waits: outside the event pair
        paths_ms.append(info["paths_ms"])
        est_ms.append(info["estimate_ms"])
        solve_ms.append(info["solve_ms"])
        kernel_nodes += info["kernel_nodes"]
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    barrier(world)
    clk = clocks.stop()
    pipelined = sdd.sdd_pipeline_in_use(ctx)
    solver_name = {1: "Jacobi-PCG", 2: "multigrid-PCG", 3: "direct (banded Cholesky)"}.get(sdd.sdd_solver_in_use(ctx), "PCG")
    sdd.sdd_sync(ctx)
    step_ms = [ev0[k].elapsed_time(ev1[k]) for k in range(K)]
    total_ms = sum(step_ms)
    path_steps = int(steps_dev.sum().item())
    value, tot_steps, max_s = whole_job(path_steps, total_ms / 1e3, world)
    max_ms = max_s * 1e3
    nodes = len(ix)
    nodes_per_s = world * nodes * K / (max_ms / 1e3)

    # dominant kernel: the path kernel, timed by events recorded inside the step graph
    mean_paths_ms = statistics.mean(paths_ms)
    steps_per_launch = path_steps / K
    achieved = ALG_OPS_PER_PATH_STEP * steps_per_launch / (mean_paths_ms / 1e3) / 1e12
    props = torch.cuda.get_device_properties(dev)
    sm_max = 2070.0
    try:
        mp = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        sm_max = float(mp.get("sm_max_mhz", sm_max))
    except Exception:
        pass
    peak = props.multi_processor_count * SM_LANES_PER_CLK * sm_max * 1e6 / 1e12
    # DRAM bytes of one launch, from the committed profile of this workload's path kernel when its sources
    # are unchanged (a capture of a node sample, scaled to the launch by path-steps)
    # and the schedulers' issue-slot utilisation in that capture (how busy the kernel keeps them: a
    # path-step issues more instructions than its algorithmic operations)
    # (the summary of the kernel variant the tuner took: with or without the zero map)
    traffic, issue_slots = None, None
    pname = f"k_paths_{name}.md"
    if shape.get("zero_map") == 2 and os.path.exists(os.path.join(ROOT, "profiles", f"k_paths_nozm_{name}.md")):
        pname = f"k_paths_nozm_{name}.md"
    prof = profiled_counters(os.path.join(ROOT, "profiles", pname))
    if prof is not None:
        per = prof["path_steps_per_launch"]
        traffic = prof["dram_bytes_per_launch"] * (steps_per_launch / per if per else 1.0)
        if prof["issue_slots"] is not None:
            issue_slots = {"value": prof["issue_slots"], "source": f"profiles/{pname} (ncu smsp__issue_active)"}

    # end to end through the C ABI with host buffers: w in from pinned host memory,
    # the interface statistics back to pinned host memory, every step
    e2e = None
    if not args.no_e2e:
        reset()
        w_pin = w_host[:K].pin_memory()
        # one set of pinned result buffers per step: the steps are enqueued back to back (the API is
        # stream-ordered) and every step's statistics land in host memory before the clock stops
        hosts = []
        for _ in range(K):
            h = {k: torch.empty(nodes, dtype=torch.float64).pin_memory() for k in ("mean_xi", "mean_eta", "se_xi", "se_eta")}
            h["n_exit"] = torch.empty(nodes, dtype=torch.int64).pin_memory()
            h["path_steps"] = torch.empty(nodes, dtype=torch.int64).pin_memory()
            hosts.append(h)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in range(K):
            sdd.sdd_set_w_host(ctx, w_pin[k])
            sdd.sdd_step(ctx, **sp)
            sdd.sdd_last_interface_stats(ctx, out=hosts[k])
        sdd.sdd_flush(ctx)
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        e2e_steps = sum(int(h["path_steps"].sum()) for h in hosts)
        e2e_value = whole_job(e2e_steps, el, world)[0]
        e2e = {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": n * n * 4,
               "d2h_bytes_per_step": nodes * 48}

    # the path kernel alone (unpipelined steps): in the timed pipelined steps it shares SMs with
    # the previous step's solve for part of its launch
    alone = None
    if pipelined:
        reset()
        sdd.sdd_set_pipeline(ctx, False)
        a_ms, a_step = [], []
        for k in range(min(K, 8)):
            flush.zero_()
            sdd.sdd_set_w(ctx, w_all[k])
            sdd.sdd_step(ctx, **sp)
            info = sdd.sdd_last_step_info(ctx)
            a_ms.append(info["paths_ms"])
            a_step.append(info["step_ms"])
        sdd.sdd_set_pipeline(ctx, True)
        a_mean = statistics.mean(a_ms[1:] if len(a_ms) > 1 else a_ms)
        a_ach = ALG_OPS_PER_PATH_STEP * steps_per_launch / (a_mean / 1e3) / 1e12
        alone = {"paths_kernel_ms": a_mean, "achieved": a_ach, "frac": a_ach / peak,
                 "unpipelined_step_ms": statistics.mean(a_step[1:] if len(a_step) > 1 else a_step),
                 "note": "unpipelined steps after the timed region (the same launches without the solve beside)"}

    # control variates at equal error: the previous fields' gradient (no training) and the learned
    # network, each timed over mesh steps from the same start, and its variance against the plain
    # estimator on the same state (one estimate each at every 16th interface node, same seed)
    equal_error = None
    if not args.no_cv:
        pick = np.arange(0, nodes, 16 if nodes > 2000 else 1)
        xs_, ys_ = np.asarray(ix)[pick], np.asarray(iy)[pick]
        equal_error = {"sample_nodes": int(pick.size)}
        modes = [("fields", sdd.SDD_CV_FIELDS, "gradient of the fields at t_{n-1} (no training)")]
        if not args.no_model:
            modes.append(("model", sdd.SDD_CV_MODEL, "learned 5-64-64-1 network, trained on the GPU at the first "
                                                    "mesh step, re-tabulated from each step's w"))
        kc = min(K, 5)
        for key, mode, what in modes:
            reset()
            train = None
            if key == "model":
                train = sdd.sdd_cv_train(ctx, per_horizon=10000, dt=WL.dt, Dt=WL.Dt, seed=100 + rank, epochs=10,
                                         batch=4096, lr=3e-3, slices=4, init_seed=7)
                train = {k2: train[k2] for k2 in ("samples_ms", "train_ms", "tabulate_ms", "rows", "steps")}
            sdd.sdd_cv_enable(ctx, mode)
            if key == "fields":
                sdd.sdd_cv_set_fields_order(ctx, args.cv_order)
            cv_ms, cv_steps, cv_pk = 0.0, 0, []
            for k in range(kc):
                flush.zero_()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                sdd.sdd_set_w(ctx, w_all[k])
                sdd.sdd_step(ctx, **sp)
                sdd.sdd_flush(ctx)
                e1.record(stream)
                torch.cuda.synchronize()
                cv_ms += e0.elapsed_time(e1)
                cv_steps += int(sdd.sdd_last_interface_stats(ctx)["path_steps"].sum())
                cv_pk.append(sdd.sdd_last_step_info(ctx)["paths_ms"])
            est = {}
            for which, m in (("plain", sdd.SDD_CV_OFF), ("cv", mode)):
                sdd.sdd_cv_enable(ctx, m)
                o = sdd.sdd_interface_mc(ctx, xs_, ys_, np.full(xs_.size, paths), dt=WL.dt, Dt=WL.Dt, seed=seed + 99)
                est[which] = {k2: v.cpu().numpy() for k2, v in o.items()}
            sdd.sdd_cv_enable(ctx, sdd.SDD_CV_OFF)
            # equal error over the sampled nodes: the plain estimator's summed variance over the
            # control variate's (the paths per node that match its RMS error); the median of the
            # per-node ratios for information
            ratio, median = {}, {}
            for f in ("xi", "eta"):
                a_, c_ = est["plain"]["se_" + f], est["cv"]["se_" + f]
                ok = c_ > 0
                ratio[f] = float(np.sum(a_ ** 2) / np.sum(c_ ** 2))
                median[f] = float(np.median((a_[ok] / c_[ok]) ** 2))
            cv_value = cv_steps / (cv_ms / 1e3)
            equal_error[key] = {"control_variate": what, "steps": kc, "path_steps_per_s": cv_value,
                                "paths_kernel_ms": statistics.mean(cv_pk),
                                "paths_kernel_ms_per_step": [round(v, 2) for v in cv_pk],
                                "paths_kernel_ms_vs_plain": statistics.mean(cv_pk) / mean_paths_ms,
                                "variance_ratio_vs_plain": ratio, "variance_ratio_median_node": median,
                                "path_steps_per_s_at_equal_error": cv_value * min(ratio.values()),
                                "interface_nodes_per_s_at_equal_error": nodes * kc / (cv_ms / 1e3) * min(ratio.values()),
                                "training": train}
            if key == "fields":
                equal_error[key]["smoothing_order"] = sdd.sdd_cv_fields_order(ctx)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(name)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": Wm,
            "ms_per_step": max_ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"{name}: {desc}, {nodes} interface nodes x {paths} paths, dt={WL.dt}, "
                                   f"Dt={WL.Dt} (K={WL.K}), plain exit test, "
                                   f"{solver_name} subdomain solves (FP64 residuals, rtol 1e-12)"
                                   + (", each step's solve iterations beside the next step's paths (pipelined)"
                                      if pipelined else ""),
                       "global_batch": world * nodes * paths, "seq_len": WL.K,
                       "parallelism": f"{world} independent instance(s), one per GPU",
                       "l2": "flushed before every step (256 MB write, outside the step's events)",
                       "launch_shape": {"block_threads": shape["block_threads"],
                                        "paths_per_task": shape["paths_per_task"],
                                        "zero_map": shape["zero_map"] == 1}},
            "interface_nodes_per_s": nodes_per_s,
            "path_steps_per_step": tot_steps / K / world,
            "paths_kernel_ms": mean_paths_ms,
            "estimate_ms": statistics.mean(est_ms),
            "solve_ms": statistics.mean(solve_ms),
            "pipelined": pipelined,
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tops/s",
                         "frac": achieved / peak, "traffic": traffic, "issue_slots": issue_slots,
                         "kernel": "k_paths", "ops_per_path_step": ALG_OPS_PER_PATH_STEP,
                         "peak_basis": f"{props.multi_processor_count} SMs x 128 lanes x {sm_max:.0f} MHz (of measured "
                                       f"maximum SM clock)",
                         "alone": alone},
            "equal_error": equal_error,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": kernel_nodes + (1 if pipelined else 0),   # + the last step's flushed iterations
            "clocks": clk,
        }
        print(json.dumps(line), flush=True)


def run_estimate(args, world, rank, local):
    """The interface estimate of the mesh-step workload's first step, alone: sdd_interface_mc on every
    node_stride-th interface node (outside any graph), K timed calls inside the NVTX range "estimate"."""
    import torch

    import paper_1402_0266_gb300 as sdd
    from paper_1402_0266_gb300 import build as b
    b.build()
    name = args.workload
    WL, wfun, desc = WORKLOADS[name]
    torch.cuda.set_device(local)
    n = WL.n
    K = args.steps or 3
    paths = args.paths or WL.paths
    xi0, eta0 = W.identity_fields(n)
    ctx = sdd.sdd_init(n, n, WL.sub, WL.sub, w=torch.from_numpy(wfun(n, 0.0)).cuda(),
                       xi0=torch.from_numpy(xi0).cuda(), eta0=torch.from_numpy(eta0).cuda())
    ix, iy = sdd.sdd_interface_nodes(ctx)
    xs, ys = np.asarray(ix)[::args.node_stride], np.asarray(iy)[::args.node_stride]
    npaths = np.full(xs.size, paths)
    if args.cv != "off":
        if args.cv == "model":
            sdd.sdd_cv_train(ctx, per_horizon=10000, dt=WL.dt, Dt=WL.Dt, seed=100, epochs=10, batch=4096, lr=3e-3,
                             slices=4, init_seed=7)
        sdd.sdd_cv_enable(ctx, {"fields": sdd.SDD_CV_FIELDS, "model": sdd.SDD_CV_MODEL}[args.cv])
    if args.shape:
        blk, ppt, zm = (int(v) for v in args.shape.split(","))
    else:
        sh = sdd.sdd_autotune(ctx, xs, ys, npaths, WL.dt, WL.Dt)
        blk, ppt, zm = sh["block_threads"], sh["paths_per_task"], sh["zero_map"]
    kw = dict(dt=WL.dt, Dt=WL.Dt, seed=WL.seed + rank, block_threads=blk, paths_per_task=ppt, zero_map=zm)
    for k in range(args.warmup):
        sdd.sdd_interface_mc(ctx, xs, ys, npaths, step_index=k, **kw)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    ms, steps = 0.0, 0
    torch.cuda.nvtx.range_push("estimate")
    for k in range(K):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        o = sdd.sdd_interface_mc(ctx, xs, ys, npaths, step_index=args.warmup + k, **kw)
        e1.record(stream)
        torch.cuda.synchronize()
        ms += e0.elapsed_time(e1)
        steps += int(o["path_steps"].sum())
    torch.cuda.nvtx.range_pop()
    if rank == 0:
        print(json.dumps({"metric": "path-steps/s (interface estimate alone, first mesh step)",
                          "value": steps / (ms / 1e3), "unit": UNIT, "n_gpus": world, "steps": K,
                          "warmup": args.warmup, "ms_per_step": ms / K, "higher_is_better": True, "scaling": "weak",
                          "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                          "config": {"workload": f"{name}: {desc}, every {args.node_stride}th of the interface nodes "
                                                 f"({xs.size}) x {paths} paths, dt={WL.dt}, Dt={WL.Dt}, control "
                                                 f"variate {args.cv}",
                                     "launch_shape": {"block_threads": blk, "paths_per_task": ppt,
                                                      "zero_map": zm == 1}},
                          "path_steps_per_launch": steps / K}), flush=True)


def run_batch64(args, world, rank, local):
    """The 64-instance workload: one batched interface estimate (one persistent launch) per step."""
    import torch

    import paper_1402_0266_gb300 as sdd
    from paper_1402_0266_gb300 import build as b
    b.build()
    torch.cuda.set_device(local)
    insts = W.batch64_instances(seed=0)
    ctxs, lists = [], []
    for I in insts:
        w = torch.from_numpy(W.w_bump(I.n, I.cx, I.cy, I.width, I.alpha)).cuda()
        ctxs.append(sdd.sdd_init(I.n, I.n, 2, 2, w=w))
        lists.append((I.nodes_i / (I.n - 1), I.nodes_j / (I.n - 1), I.paths))
    batch = sdd.sdd_batch_create(ctxs)
    dt, Dt = 1e-4, 1e-2
    shape = sdd.sdd_batch_autotune(batch, lists, dt, Dt)
    for k in range(args.warmup):
        sdd.sdd_batch_interface_mc(batch, lists, dt, Dt, seed=rank, step_index=k)
    torch.cuda.synchronize()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    times, steps = [], 0
    for k in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        outs = sdd.sdd_batch_interface_mc(batch, lists, dt, Dt, seed=rank, step_index=k)
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
        steps += sum(int(o["path_steps"].sum()) for o in outs)
    ms = sum(times)
    nodes = sum(l[0].size for l in lists)
    if rank == 0:
        print(json.dumps({"metric": METRIC.replace("whole mesh steps", "batched estimate"), "value": steps / (ms / 1e3),
                          "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                          "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
                          "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                          "config": {"workload": f"batch64: 64 instances, grids 65..513, {nodes} nodes, paths 1e3..1e5 "
                                                 f"log-uniform, dt={dt}, Dt={Dt}, one persistent launch per step",
                                     "tuned_shape": shape},
                          "interface_nodes_per_s": nodes * args.steps / (ms / 1e3),
                          "path_steps_per_step": steps / args.steps}), flush=True)


def run_cv65(args, world, rank, local):
    """The learned control variate on the w = 1 heat problem (65 x 65, 33 nodes on
    x = 1/2, dt = 1e-3, Dt = 0.05): train on 1e6 single-path samples of the method,
    then compare the plain estimator at 1e4 paths per node with the control variate
    at 2e3 paths per node against a 1e6-path estimate. Value: path-steps per second
    of plain-estimator work matched at the control variate's error."""
    import torch

    import paper_1402_0266_gb300 as sdd
    from paper_1402_0266_gb300 import build as b
    b.build()
    torch.cuda.set_device(local)
    n, dt, Dt = 65, 1e-3, 0.05
    xi0, eta0 = W.heat65_fields()
    ctx = sdd.sdd_init(n, n, 2, 1, w=torch.from_numpy(W.w_const(n)).cuda(), xi0=torch.from_numpy(xi0).cuda(),
                       eta0=torch.from_numpy(eta0).cuda())
    sdd.sdd_set_boundary(ctx, torch.zeros(4 * n + 4 * n, dtype=torch.float64, device="cuda"))
    info = sdd.sdd_cv_train(ctx, per_horizon=20000, dt=dt, Dt=Dt, seed=1, epochs=20, batch=4096, lr=3e-3, init_seed=7)
    xs, ys = W.heat65_nodes()
    xs, ys = xs[1:32], ys[1:32]

    def run(paths, seed, mode, timed=False):
        sdd.sdd_cv_enable(ctx, mode)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        o = sdd.sdd_interface_mc(ctx, xs, ys, np.full(xs.size, paths), dt=dt, Dt=Dt, seed=seed)
        e1.record()
        torch.cuda.synchronize()
        return {k: v.cpu().numpy() for k, v in o.items()}, e0.elapsed_time(e1)

    ref, _ = run(10 ** 6, 1000, sdd.SDD_CV_OFF)
    for k in range(args.warmup):
        run(10000, 10 + k, sdd.SDD_CV_OFF)
        run(2000, 20 + k, sdd.SDD_CV_TABLE)
    ep, ec, tp, tc, sp_, sc = [], [], 0.0, 0.0, 0, 0
    for r in range(args.steps):
        a, ta = run(10000, 2000 + r, sdd.SDD_CV_OFF)
        c, tcv = run(2000, 3000 + r, sdd.SDD_CV_TABLE)
        ep.append(np.concatenate([a["mean_xi"] - ref["mean_xi"], a["mean_eta"] - ref["mean_eta"]]))
        ec.append(np.concatenate([c["mean_xi"] - ref["mean_xi"], c["mean_eta"] - ref["mean_eta"]]))
        tp += ta
        tc += tcv
        sp_ += int(a["path_steps"].sum())
        sc += int(c["path_steps"].sum())
    rms_p = math.sqrt(np.mean(np.square(ep)))
    rms_c = math.sqrt(np.mean(np.square(ec)))
    # plain path-steps needed for the control variate's error, per second of control-variate run
    equiv = sp_ * (rms_p / rms_c) ** 2
    if rank == 0:
        print(json.dumps({
            "metric": "path-steps/s at equal MC error (plain-estimator work matched by the learned control variate)",
            "value": equiv / (tc / 1e3), "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": tc / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": "cv65: w=1 heat problem on 65x65, 31 interior nodes on x=1/2, dt=1e-3, Dt=0.05; "
                                   "network 5-64-64-1 trained on 1e6 samples (20 epochs, batch 4096); "
                                   "plain at 1e4 paths vs control variate at 2e3 paths, both against a 1e6-path "
                                   "estimate; one step = one estimate of each"},
            "rms_plain_1e4": rms_p, "rms_cv_2e3": rms_c,
            "path_steps_plain": sp_ / args.steps, "path_steps_cv": sc / args.steps,
            "path_step_ratio": sp_ / sc, "error_ratio": rms_c / rms_p,
            "ms_plain_1e4": tp / args.steps, "ms_cv_2e3": tc / args.steps,
            "speedup_at_equal_error": (tp * (rms_p / rms_c) ** 2) / tc,
            "training": {k: info[k] for k in ("samples_ms", "train_ms", "tabulate_ms", "rows", "steps", "slices",
                                              "loss_xi", "loss_eta")},
        }), flush=True)


def run_ring41(args, world, rank, local):
    """The paper's Sec. 5 experiment: w = 1 / rho (moving ring), 41 x 41, four subdomains, Dt = 1e-3 up to
    t = 0.75 (750 mesh steps) with 20 sub-steps and 1e4 paths per interface node, from the uniform mesh.
    One step = one mesh step (w of the step uploaded from the host, then the graph of the step)."""
    import torch

    import paper_1402_0266_gb300 as sdd
    from paper_1402_0266_gb300 import build as b
    b.build()
    torch.cuda.set_device(local)
    wl = W.RING41
    n, Dt = wl.n, wl.Dt
    steps = args.steps or wl.steps
    xi0, eta0 = W.identity_fields(n)
    w_all = torch.from_numpy(np.stack([W.w_paper_ring(n, k * Dt) for k in range(steps)])).cuda()
    ctx = sdd.sdd_init(n, n, wl.sub, wl.sub, w=w_all[0], xi0=torch.from_numpy(xi0).cuda(),
                       eta0=torch.from_numpy(eta0).cuda())
    # the paper's setup: estimates at the key points (and every 8th node of a line), PCHIP elsewhere
    sdd.sdd_set_keypoints(ctx, args.key_spacing >= 0, max(args.key_spacing, 0))
    sdd.sdd_set_solver(ctx, {"auto": 0, "jacobi": 1, "mg": 2, "direct": 3}[args.solver])
    sp = dict(dt=wl.dt, Dt=Dt, seed=rank, paths_per_node=wl.paths, rtol=1e-12, max_iter=20000)
    nodes = len(sdd.sdd_interface_nodes(ctx)[0])
    # the statistics of every step land in buffers made once (no allocation inside the timed loop)
    stats = {k: torch.empty(nodes, dtype=torch.float64, device="cuda") for k in ("mean_xi", "mean_eta", "se_xi", "se_eta")}
    stats["n_exit"] = torch.empty(nodes, dtype=torch.int64, device="cuda")
    stats["path_steps"] = torch.empty(nodes, dtype=torch.int64, device="cuda")
    counts = torch.zeros(steps, dtype=torch.int64, device="cuda")

    def one_step(k):
        sdd.sdd_set_w(ctx, w_all[k % steps])
        sdd.sdd_step(ctx, **sp)
        sdd.sdd_last_interface_stats(ctx, out=stats)
        torch.sum(stats["path_steps"], dim=0, out=counts[k % steps])

    # a step here is about 0.3 ms of small kernels: warm up for at least a second (and W steps),
    # so that the clocks have settled before the timed region
    t0 = time.perf_counter()
    k = 0
    while k < args.warmup or time.perf_counter() - t0 < 1.0:
        one_step(k)
        k += 1
        if k % 100 == 0:
            torch.cuda.synchronize()
    sdd.sdd_set_fields(ctx, torch.from_numpy(xi0).cuda(), torch.from_numpy(eta0).cuda())
    sdd.sdd_set_step_index(ctx, 0)
    counts.zero_()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(local)
    clocks.start()
    e0.record()
    for k in range(steps):
        one_step(k)
    e1.record()
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    xi, eta = (a.cpu().numpy() for a in sdd.sdd_get_fields(ctx))
    p = np.stack([xi, eta], axis=-1)
    quad = [p[:-1, :-1], p[:-1, 1:], p[1:, 1:], p[1:, :-1]]
    folded = np.zeros(xi[:-1, :-1].shape, dtype=bool)
    for k in range(4):
        e1_, e2_ = quad[k] - quad[k - 1], quad[(k + 1) % 4] - quad[k]
        folded |= (e1_[..., 0] * e2_[..., 1] - e1_[..., 1] * e2_[..., 0]) <= 0
    tot = int(counts.sum().item())
    key_nodes = int(sdd.sdd_keypoint_mask(ctx).sum().item()) if args.key_spacing >= 0 else nodes
    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": tot / (ms / 1e3), "unit": UNIT, "n_gpus": world, "steps": steps,
            "warmup": args.warmup, "ms_per_step": ms / steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"ring41 (Sec. 5): w = 1/rho, {n}x{n}, 2x2 subdomains, {nodes} interface nodes "
                                   f"(estimates at the key points, spacing {args.key_spacing}; PCHIP elsewhere) x "
                                   f"{wl.paths} paths, dt={wl.dt}, Dt={Dt}, {steps} mesh steps from the uniform mesh"},
            "key_nodes_at_end": key_nodes,
            "interface_nodes_per_s": nodes * steps / (ms / 1e3), "path_steps_per_step": tot / steps,
            "folded_cells_at_end": int(folded.sum()),
            "max_mesh_displacement": float(max(np.abs(xi - W.grid(n)[0]).max(), np.abs(eta - W.grid(n)[1]).max())),
            "clocks": clk,
        }), flush=True)


def run_exit65(args, world, rank, local):
    """Exit tests at equal accuracy on the w = 1 heat problem (65 x 65, 31 interior nodes on x = 1/2,
    Dt = 0.05, closed form exp(-2 pi^2 t) sin(pi x) sin(pi y)): the RMS error and the time of the
    estimate with 2e6 paths per node for the paper's fixed-step test, the Brownian-bridge test and
    exponential time-stepping over a range of dt. Value: path-steps per second of the fixed-step
    test matched at the bridge test's error (the fixed-step test's error falls like sqrt(dt))."""
    import torch

    import paper_1402_0266_gb300 as sdd
    from paper_1402_0266_gb300 import build as b
    b.build()
    torch.cuda.set_device(local)
    n, Dt, N = 65, 0.05, 2_000_000
    xi0, eta0 = W.heat65_fields()
    ctx = sdd.sdd_init(n, n, 2, 1, w=torch.from_numpy(W.w_const(n)).cuda(), xi0=torch.from_numpy(xi0).cuda(),
                       eta0=torch.from_numpy(eta0).cuda())
    sdd.sdd_set_boundary(ctx, torch.zeros(8 * n, dtype=torch.float64, device="cuda"))
    xs, ys = W.heat65_nodes()
    xs, ys = xs[1:32], ys[1:32]
    ex, ee = W.heat_exact(xs, ys, Dt)
    rows = []
    for mode in (0, 1, 2):
        for dt in (1e-2, 2.5e-3, 1e-3, 2.5e-4):
            for k in range(args.warmup if not rows else 0):
                sdd.sdd_interface_mc(ctx, xs, ys, np.full(xs.size, N), dt=dt, Dt=Dt, seed=99, exit_mode=mode)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            o = sdd.sdd_interface_mc(ctx, xs, ys, np.full(xs.size, N), dt=dt, Dt=Dt, seed=3, exit_mode=mode)
            e1.record()
            torch.cuda.synchronize()
            o = {k: v.cpu().numpy() for k, v in o.items()}
            err = np.concatenate([o["mean_xi"] - ex, o["mean_eta"] - ee])
            rows.append({"exit_mode": mode, "dt": dt, "rms_error": float(math.sqrt(np.mean(err ** 2))),
                         "mean_se": float(np.mean(np.concatenate([o["se_xi"], o["se_eta"]]))),
                         "ms": e0.elapsed_time(e1), "path_steps": int(o["path_steps"].sum())})
    plain = [r for r in rows if r["exit_mode"] == 0]
    bridge = [r for r in rows if r["exit_mode"] == 1 and r["dt"] == 1e-2][0]
    # fixed-step error c sqrt(dt), c from the smallest dt measured; dt needed for the bridge test's error
    c = plain[-1]["rms_error"] / math.sqrt(plain[-1]["dt"])
    dt_eq = (bridge["rms_error"] / c) ** 2
    steps_eq = plain[-1]["path_steps"] * plain[-1]["dt"] / dt_eq
    rate_plain = plain[-1]["path_steps"] / (plain[-1]["ms"] / 1e3)
    if rank == 0:
        print(json.dumps({
            "metric": "path-steps/s at equal exit accuracy (fixed-step test matched at the bridge test's error)",
            "value": steps_eq / (bridge["ms"] / 1e3), "unit": UNIT, "n_gpus": world, "steps": 1,
            "warmup": args.warmup, "ms_per_step": bridge["ms"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "exit65: w=1 heat problem on 65x65, 31 interior nodes on x=1/2, Dt=0.05, 2e6 paths "
                                   "per node; exit modes 0 (fixed steps, plain test), 1 (bridge test), 2 (exponential "
                                   "time-stepping) at dt = 1e-2 .. 2.5e-4"},
            "dt_fixed_step_for_bridge_error": dt_eq, "fixed_step_path_steps_per_s": rate_plain,
            "speedup_at_equal_error": (plain[-1]["ms"] * plain[-1]["dt"] / dt_eq) / bridge["ms"],
            "runs": rows,
        }), flush=True)


def run_heat65(args, world, rank, local):
    """The small heat-equation case (w = 1 on 65 x 65, 33 nodes on x = 1/2 x 1000 paths, dt = 1e-3, Dt = 0.05,
    zero boundary data): one step = one interface estimate of all 33 nodes, inputs resident on the device.
    Latency-bound by design (1.6e6 path-steps); the closed form is its correctness check."""
    import torch

    import paper_1402_0266_gb300 as sdd
    from paper_1402_0266_gb300 import build as b
    b.build()
    torch.cuda.set_device(local)
    n, dt, Dt, paths = 65, 1e-3, 0.05, 1000
    xi0, eta0 = W.heat65_fields()
    ctx = sdd.sdd_init(n, n, 2, 2, w=torch.from_numpy(W.w_const(n)).cuda(), xi0=torch.from_numpy(xi0).cuda(),
                       eta0=torch.from_numpy(eta0).cuda())
    sdd.sdd_set_boundary(ctx, torch.zeros(4 * n + 4 * n, dtype=torch.float64, device="cuda"))
    xs, ys = W.heat65_nodes()
    npaths = np.full(xs.size, paths, dtype=np.int64)
    stream = torch.cuda.current_stream()
    for k in range(args.warmup):
        sdd.sdd_interface_mc(ctx, xs, ys, npaths, dt=dt, Dt=Dt, seed=k)
    K = args.steps
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    outs = []
    torch.cuda.synchronize()
    barrier(world)
    e0.record(stream)
    for k in range(K):
        outs.append(sdd.sdd_interface_mc(ctx, xs, ys, npaths, dt=dt, Dt=Dt, seed=100 + k))
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    ms = e0.elapsed_time(e1)
    steps = sum(int(o["path_steps"].sum()) for o in outs)
    value, tot, mx = whole_job(steps, ms / 1e3, world)
    # the closed form at t = Dt: xi = exp(-2 pi^2 Dt) sin(pi x) sin(pi y) (plain test: biased like sqrt(dt))
    o = {k2: v.cpu().numpy() for k2, v in outs[-1].items()}
    exact = np.exp(-2 * np.pi ** 2 * Dt) * np.sin(np.pi * xs) * np.sin(np.pi * ys)
    if rank == 0:
        print(json.dumps({"metric": "path-steps/s (interface Monte Carlo, one estimate per step)", "value": value,
                          "unit": UNIT, "n_gpus": world, "steps": K, "warmup": args.warmup, "ms_per_step": ms / K,
                          "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                          "data": "synthetic",
                          "config": {"workload": f"heat65: w=1 on {n}x{n}, {xs.size} nodes on x=1/2 x {paths} paths, "
                                                 f"dt={dt}, Dt={Dt} (K=50), zero boundary data, plain exit test"},
                          "interface_nodes_per_s": world * xs.size * K / (mx),
                          "max_abs_error_vs_closed_form": float(np.abs(o["mean_xi"] - exact).max()),
                          "max_se": float(o["se_xi"].max())}), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        # the CPU oracle on a sample of the mesh-step workload: rank 0 alone runs; other ranks exit without work
        run_reference(args, int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")))
        return
    world, rank, local = dist_init()
    if args.workload == "heat65":
        args.steps = args.steps or 200
        run_heat65(args, world, rank, local)
    elif args.workload == "batch64":
        args.steps = args.steps or 20
        run_batch64(args, world, rank, local)
    elif args.workload == "exit65":
        run_exit65(args, world, rank, local)
    elif args.workload == "ring41":
        run_ring41(args, world, rank, local)
    elif args.workload == "cv65":
        args.steps = args.steps or 12
        run_cv65(args, world, rank, local)
    elif args.estimate_only:
        run_estimate(args, world, rank, local)
    else:
        run_ours(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
