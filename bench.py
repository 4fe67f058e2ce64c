#!/usr/bin/env python
"""Throughput benchmark of the GB300 HPS solver.

Workload (one "step" = one pass of the whole hot path): build the ItI
solution operator of the 2D variable-coefficient Helmholtz problem
Lap u + k^2 (1 - n(x)) u = f on [-1, 1]^2 (k = 20, eta = 20, n = four seeded
Gaussian bumps, complex128, uniform quadtree of depth 6 = 4096 leaves,
p = 16, q = 14: leaf stage + all merges), then solve for incoming impedance
data g with a second seeded source f2 (upward particular pass with the stored
factors, downward pass, leaf output), then release the handle.

Device-timed numbers use CUDA events on the launching stream with every input
already in HBM; the e2e number goes through the same public calls with host
(NumPy) buffers, so host-to-device and device-to-host copies are inside the
timed region.  The working set (about 11 GB of factors per step) is far larger
than the 129 MB L2, so no flush is needed between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun (N > 1) every rank runs an independent replica (the problems
are independent: no collective on the data path) and rank 0 prints the
aggregate.
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

METRIC = "served solves/s & p50/p99 vs plain GPU HPS; FP64 roofline frac; rel err≤1e-10"
UNIT = "solves/s"
WORKLOAD = {"workload": "helmholtz2d_iti_c128_depth6_p16", "equation": "Lap u + k^2 (1 - n(x)) u = f",
            "n_leaves": 4096, "depth": 6, "p": 16, "q": 14, "k": 20.0, "eta": 20.0,
            "seed_problem": 1, "seed_solve_source": 11, "root_map": False,
            "step": "hps_build + hps_solve(new f) + hps_free",
            "l2": "no flush: about 11 GB of factors per step, far above the 129 MB L2"}
CPU_SAMPLE_DEPTH = 3
# FP64 FMA throughput per SM per clock (flops), measured on this GPU type by a
# dependency-free DFMA stream with the SM clock sampled alongside
FP64_FLOP_PER_CLK_SM = None


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--depth", type=int, default=6,
                    help="quadtree depth (6 = the benchmark workload; smaller for profiler captures)")
    args = ap.parse_args()
    if args.depth != WORKLOAD["depth"]:
        WORKLOAD["depth"] = args.depth
        WORKLOAD["n_leaves"] = 4 ** args.depth
        WORKLOAD["workload"] = f"helmholtz2d_iti_c128_depth{args.depth}_p16"
    return args


def problem(seed_offset=0):
    import workloads as W
    return W.helmholtz_bumps_2d(seed=WORKLOAD["seed_problem"] + seed_offset, k=WORKLOAD["k"],
                                eta=WORKLOAD["eta"])


def host_inputs(P, depth, seed_offset=0):
    pr = problem(seed_offset)
    p, q = WORKLOAD["p"], WORKLOAD["q"]
    t = P.uniform_tree(2, depth, pr.lo, pr.hi)
    x, xb = P.hps_nodes(t, p, q)
    nl, ppl, nr = P.hps_sizes(t, p, q)
    c = pr.coeffs(x)["c"].reshape(nl, ppl).copy()
    f = pr.source(x).reshape(nl, ppl).astype(np.complex128)
    g = pr.boundary(xb).astype(np.complex128)
    rng = np.random.default_rng(WORKLOAD["seed_solve_source"] + seed_offset)
    f2 = (rng.standard_normal((nl, ppl)) + 1j * rng.standard_normal((nl, ppl))) * np.abs(f).max()
    return pr, t, c, f, g, np.ascontiguousarray(f2)


# ------------------------------------------------------------------ clocks --

class ClockSampler:
    """nvidia-smi samples every 200 ms during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except (FileNotFoundError, OSError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, pw, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [s.strip() for s in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                pw.append(float(parts[3]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "samples": len(sm),
                "power_w_max": max(pw), "reasons": sorted(reasons)}


# ----------------------------------------------------------------- our arm --

def run_ours(args, rank, world):
    import torch
    import paper_2503_17535_gb300 as P

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pr, t, c, f, g, f2 = host_inputs(P, WORKLOAD["depth"], seed_offset=rank)
    p, q = WORKLOAD["p"], WORKLOAD["q"]
    nl, ppl, nr = P.hps_sizes(t, p, q)
    cd, fd, gd, f2d = (torch.from_numpy(v).to(dev) for v in (c, f, g, f2))
    ud = torch.zeros((nl, ppl), dtype=torch.complex128, device=dev)
    stream = torch.cuda.current_stream(dev)

    launches = [0]

    def step():
        h = P.hps_build(t, p, q, P.HPS_ITI, c=cd, f=fd, eta=WORKLOAD["eta"])
        launches[0] += P.hps_last_launch_count(h)
        P.hps_solve(h, gd, ud, f=f2d)
        launches[0] += P.hps_last_launch_count(h)
        P.hps_free(h)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    launches[0] = 0
    cvd = os.environ.get("CUDA_VISIBLE_DEVICES")
    gpu_id = cvd.split(",")[local].strip() if cvd else str(local)
    sampler = ClockSampler(gpu_id)
    sampler.start()
    time.sleep(0.3)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for i in range(args.steps):
        evs[i][0].record(stream)
        step()
        evs[i][1].record(stream)
    t1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = sampler.stop()
    total_ms = t0.elapsed_time(t1)
    per = sorted(a.elapsed_time(b) for a, b in evs)
    if world > 1:
        tt = torch.tensor([total_ms], device=dev)
        torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
        total_ms = float(tt.item())
    value = world * args.steps / (total_ms / 1e3)

    # ---- one profiled step (untimed): per-class kernel times with CUDA events
    h = P.hps_build(t, p, q, P.HPS_ITI, c=cd, f=fd, eta=WORKLOAD["eta"], profile=True)
    sb = P.hps_kernel_stats(h)
    P.hps_solve(h, gd, ud, f=f2d)
    ss = P.hps_kernel_stats(h)
    P.hps_free(h)
    classes = {k: {"launches": sb[k]["launches"] + ss[k]["launches"],
                   "flops": sb[k]["flops"] + ss[k]["flops"],
                   "ms": sb[k]["ms"] + ss[k]["ms"]} for k in sb}
    flops_step = sum(v["flops"] for v in classes.values())
    # algorithmic flops of the CPU-baseline sample (same problem, smaller depth)
    _, ts_, cs_, fs_, gs_, f2s_ = host_inputs(P, CPU_SAMPLE_DEPTH, seed_offset=rank)
    nls, ppls, _ = P.hps_sizes(ts_, p, q)
    hs_ = P.hps_build(ts_, p, q, P.HPS_ITI, c=cs_, f=fs_, eta=WORKLOAD["eta"])
    fl_s = sum(v["flops"] for v in P.hps_kernel_stats(hs_).values())
    P.hps_solve(hs_, gs_, np.zeros((nls, ppls), np.complex128), f=f2s_)
    fl_s += sum(v["flops"] for v in P.hps_kernel_stats(hs_).values())
    P.hps_free(hs_)
    sample_ratio = flops_step / fl_s
    dom = max(classes, key=lambda k: classes[k]["ms"])
    sm_mhz = clocks.get("sm_mhz") or 1485.0
    peak_tf = (FP64_FLOP_PER_CLK_SM or 4.0) * 152 * sm_mhz * 1e6 / 1e12
    ach = classes[dom]["flops"] / (classes[dom]["ms"] / 1e3) / 1e12 if classes[dom]["ms"] > 0 else 0.0
    roofline = {"bound": "alu", "kernel_class": dom, "achieved": round(ach, 4), "peak": round(peak_tf, 4),
                "unit": "TFLOP/s", "frac": round(ach / peak_tf, 4), "traffic": None,
                "peak_source": "FP64 FMA pipe: flop/clk/SM x 152 SMs x median SM clock of this run",
                "launches_per_step": classes[dom]["launches"], "ms_per_step": round(classes[dom]["ms"], 3)}

    # ---- end to end through the C ABI with host buffers
    e2e = None
    if not args.no_e2e:
        uh = np.zeros((nl, ppl), np.complex128)

        def step_host():
            h = P.hps_build(t, p, q, P.HPS_ITI, c=c, f=f, eta=WORKLOAD["eta"])
            P.hps_solve(h, g, uh, f=f2)
            P.hps_free(h)

        step_host()
        torch.cuda.synchronize()
        ts = time.perf_counter()
        for _ in range(args.steps):
            step_host()
        torch.cuda.synchronize()
        te = time.perf_counter() - ts
        if world > 1:
            tt = torch.tensor([te], device=dev)
            torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
            te = float(tt.item())
        e2e = {"value": round(world * args.steps / te, 4), "unit": UNIT,
               "h2d_bytes_per_step": int(c.nbytes + f.nbytes + g.nbytes + f2.nbytes),
               "d2h_bytes_per_step": int(uh.nbytes)}
    return {"value": value, "total_ms": total_ms, "per": per, "clocks": clocks, "roofline": roofline,
            "classes": classes, "flops_step": flops_step, "launches": launches[0] // max(args.steps, 1),
            "e2e": e2e, "sample_ratio": sample_ratio}


# ------------------------------------------------------------- CPU oracle --

def oracle_sample_step(depth=CPU_SAMPLE_DEPTH):
    """One oracle build + new-source solve on the same problem at a smaller
    depth; returns its wall time in seconds."""
    import workloads as W  # noqa: F401
    from oracle import geometry as geo
    from oracle import hps as O
    pr = problem()
    p, q = WORKLOAD["p"], WORKLOAD["q"]
    x, a, b, c, f, g = O.sample_problem(pr, p, q, depth)
    rng = np.random.default_rng(WORKLOAD["seed_solve_source"])
    f2 = (rng.standard_normal(f.shape) + 1j * rng.standard_normal(f.shape)) * np.abs(f).max()
    t0 = time.perf_counter()
    O.build(2, "iti", p, q, depth, pr.lo, pr.hi, a, b, c, f, eta=pr.eta)
    s2 = O.build(2, "iti", p, q, depth, pr.lo, pr.hi, a, b, c, f2, eta=pr.eta)
    O.solve(s2, g)
    del geo
    return time.perf_counter() - t0


def flop_ratio():
    """Algorithmic flops of the full workload over those of the CPU sample,
    from a closed-form count of the leaf stage (LU of B, solves, T = QH Y)
    and of the ItI merges (W, its LU, the W^{-1} and D21 solves, B X); it
    agrees with the library's own launch counts to a few percent and is used
    by the reference arm, which runs no GPU code."""
    def flops(depth):
        p, q = WORKLOAD["p"], WORKLOAD["q"]
        npts, nb = p * p, 4 * q
        nl = 4 ** depth
        # leaf: LU of B (npts), solve with nb + 1 columns, T = QH Y
        leaf = nl * 8 * (npts ** 3 / 3 + npts ** 2 * (nb + 1) + nb * npts * (nb + 1))
        merge = 0.0
        n = q
        for m in range(depth):
            nm = 4 ** (depth - m - 1)
            hn, ne = 4 * n, 8 * n
            per = (hn ** 3 + hn * hn * (ne + 1) + hn ** 3 / 3 + hn * hn * (ne + 1)
                   + hn * hn * (ne + 1) + (0 if m == depth - 1 else 4 * (2 * n) * (2 * n) * (ne + 1)))
            merge += nm * 8 * per
            n *= 2
        return leaf + merge
    return flops(WORKLOAD["depth"]) / flops(CPU_SAMPLE_DEPTH)


def cpu_baseline(ratio, reps=1):
    ts = [oracle_sample_step() for _ in range(reps)]
    t = min(ts)
    return {"value": round(1.0 / (t * ratio), 6), "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
            "sample": (f"oracle (NumPy/SciPy LAPACK) build + new-source solve of the same problem at "
                       f"depth {CPU_SAMPLE_DEPTH} (64 leaves, p=16), {t:.2f} s, scaled to depth "
                       f"{WORKLOAD['depth']} by the algorithmic flop ratio {ratio:.1f} (library counts)"),
            "blas_threads_env": os.environ.get("OPENBLAS_NUM_THREADS") or os.environ.get("OMP_NUM_THREADS")
            or "default (all cores)"}


def run_reference(args, rank):
    if rank != 0:
        return None
    for _ in range(args.warmup):
        oracle_sample_step()
    ratio = flop_ratio()
    ts = [oracle_sample_step() for _ in range(args.steps)]
    scaled = [t * ratio for t in ts]
    value = args.steps / sum(scaled)
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 6), "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(1e3 * sum(scaled) / args.steps, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "c128", "data": "synthetic",
            "config": WORKLOAD,
            "cpu_baseline": {"value": round(value, 6), "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                             "sample": (f"each step: oracle build + new-source solve at depth {CPU_SAMPLE_DEPTH} "
                                        f"(mean {statistics.mean(ts):.2f} s), scaled to depth 6 by the flop "
                                        f"ratio {ratio:.1f}")},
            "e2e": {"value": round(value, 6), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    return line


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        line = run_reference(args, rank)
        if line is not None:
            print(json.dumps(line), flush=True)
        return 0
    import torch
    if world > 1:
        torch.distributed.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    r = run_ours(args, rank, world)
    if rank == 0:
        per = r["per"]
        p50 = per[len(per) // 2]
        p99 = per[min(len(per) - 1, int(round(0.99 * (len(per) - 1))))]
        step_tf = r["flops_step"] / (statistics.median(per) / 1e3) / 1e12
        line = {"metric": METRIC, "value": round(r["value"], 4), "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": round(r["total_ms"] / args.steps, 3), "p50_ms": round(p50, 3),
                "p99_ms": round(p99, 3), "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "c128", "data": "synthetic",
                "config": dict(WORKLOAD, parallelism=f"replicas x{world}"),
                "clocks": r["clocks"], "e2e": r["e2e"], "gpu_launches": r["launches"] * args.steps,
                "roofline": r["roofline"],
                "step_fp64": {"algorithmic_flops": r["flops_step"], "achieved_tflops": round(step_tf, 4),
                              "frac_of_peak": round(step_tf / r["roofline"]["peak"], 4)},
                "kernel_classes": {k: {"launches": v["launches"], "ms": round(v["ms"], 3),
                                       "gflops": round(v["flops"] / 1e9, 3)} for k, v in r["classes"].items()}}
        if world == 1 and not args.no_cpu:
            line["cpu_baseline"] = cpu_baseline(r["sample_ratio"])
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
