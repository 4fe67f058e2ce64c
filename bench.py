#!/usr/bin/env python
"""Throughput benchmark of the GB300 HPS solver.

Default workload (one "step" = one pass of the whole hot path): build the ItI
solution operator of the 2D variable-coefficient Helmholtz problem
Lap u + k^2 (1 - n(x)) u = f on [-1, 1]^2 (k = 20, eta = 20, n = four seeded
Gaussian bumps, complex128, uniform quadtree of depth 6 = 4096 leaves,
p = 16, q = 14: leaf stage + all merges), then solve for incoming impedance
data g with a second seeded source f2 (upward particular pass with the stored
factors, downward pass, leaf output), then release the handle.

Other workloads (--workload): poisson2d (16 leaves, p = 8, Dirichlet),
elliptic3d (512 leaves, p = 8, divergence-form 3D DtN) and adaptive3d (the
3D operator with a sharp seeded source on an octree refined by hps_refine,
eps = 1e-4, leaf depths 2..5).

Device-timed numbers use CUDA events on the launching stream with every input
already in HBM; the e2e number goes through the same public calls with host
(NumPy) buffers, so host-to-device and device-to-host copies are inside the
timed region.  The factor working set of a step (gigabytes for the large
workloads) is far above the 129 MB L2, so no flush is needed between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                    [--workload helmholtz2d|poisson2d|elliptic3d|adaptive3d]

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
FP64_FLOP_PER_CLK_SM = 4.0   # 2 DFMA per clock per SM: 152 x 4 x 2.07 GHz = 1.26 TFLOP/s

def tensor_peak():
    """Sustained bf16 tensor rate (TFLOP/s) from the measured peaks file, else the fallback."""
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            v = float(json.load(fh)["bf16_tflops_sustained"])
        return v, "measured: MEASURED_PEAKS.json bf16_tflops_sustained (cuBLAS bf16, seconds-long loop)"
    except (OSError, KeyError, ValueError):
        return 1700.0, "fallback: 1.7 PFLOP/s sustained bf16"


WORKLOADS = {
    "helmholtz2d": {"workload": "helmholtz2d_iti_c128_depth6_p16", "equation": "Lap u + k^2 (1 - n(x)) u = f",
                    "dim": 2, "kind": "iti", "n_leaves": 4096, "depth": 6, "p": 16, "q": 14, "k": 20.0,
                    "eta": 20.0, "seed_problem": 1},
    "poisson2d": {"workload": "poisson2d_dtn_f64_depth2_p8", "equation": "Lap u = f, Dirichlet",
                  "dim": 2, "kind": "dtn", "n_leaves": 16, "depth": 2, "p": 8, "q": 6, "seed_problem": 0},
    "elliptic3d": {"workload": "elliptic3d_dtn_f64_depth3_p8", "equation": "div(a grad u) + c u = f",
                   "dim": 3, "kind": "dtn", "n_leaves": 512, "depth": 3, "p": 8, "q": 6, "seed_problem": 2},
    "adaptive3d": {"workload": "adaptive3d_dtn_f64_p8_eps1e-4_depths2-5",
                   "equation": "div(a grad u) + c u = f, sharp source", "dim": 3, "kind": "dtn",
                   "depth": -1, "p": 8, "q": 6, "seed_problem": 3, "eps": 1e-4, "min_depth": 2,
                   "max_depth": 5},
}
# Serving workload: seeded operators (kind, depth, p drawn as listed) resident
# in a request server; a Poisson stream of requests, 80 % apply-only solves
# (new seeded boundary data, the operator's build-time source) on a resident
# operator, 20 % rebuilds of an operator with a new seeded coefficient field.
SERVE = {"workload": "serve2d_poisson_arrivals", "seed": 4, "n_ops": 6, "depths": [3, 7], "ps": [8, 12, 16],
         "kinds": ["dtn", "iti"], "rebuild_frac": 0.2, "requests": 60, "rates": [0.5, 0.9, 1.5],
         "pool": 3, "max_batch": 8, "n_streams": 4, "op_budget_gb": 150}

# bf16 digit products per FP64 multiply-add in the tensor-core products
# (ten 6-bit digits per operand, the pairs of digit indices summing to <= 11)
TC_DIGIT_PRODUCTS = 55
# DRAM bytes (read + write) per launch of a kernel class, averaged over every
# launch of one build, from an ncu capture of the same workload (summaries
# under profiles/); None where no capture of the current kernels exists
NCU_TRAFFIC = {
    ("helmholtz2d_iti_c128_depth6_p16", "gemm_tc"): {
        "bytes_per_launch": 182930000,
        "source": "ncu dram__bytes_read.sum + dram__bytes_write.sum over the 581 k_gemm_tc launches of one "
                  "build (106.3 GB), profiles/k_gemm_tc_traffic_helmholtz2d_depth6.md"},
}

COMMON = {"seed_solve_source": 11, "root_map": False, "step": "hps_build + hps_solve(new f) + hps_free",
          "l2": "no flush: the step's factor working set is far above the 129 MB L2"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="helmholtz2d", choices=sorted(WORKLOADS) + ["serve", "diff", "gemm"])
    ap.add_argument("--requests", type=int, default=None, help="serve: requests per arrival rate")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--root", default="lazy", choices=["lazy", "explicit"],
                    help="lazy: the top merge keeps D's factors and [C | h_int] and each solve applies "
                         "D^-1 (hps_options.lazy_root); explicit: the top merge forms S and w as well")
    ap.add_argument("--trace", default=None,
                    help="write the per-launch trace of the profiled step (JSON) to this path")
    ap.add_argument("--depth", type=int, default=None,
                    help="uniform tree depth override (smaller cases for profiler captures)")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving leg of the default line")
    ap.add_argument("--oracle-threads", type=int, default=8,
                    help="BLAS threads of the oracle timings (OpenBLAS on many small matrices is slower "
                         "with one thread per core)")
    ap.add_argument("--oracle-sample", type=int, default=None, help=argparse.SUPPRESS)
    ap.add_argument("--oracle-reps", type=int, default=1, help=argparse.SUPPRESS)
    ap.add_argument("--gemm", default="tc", choices=["tc", "fp64"],
                    help="tc: large build products on the tensor cores as exact digit-slice products "
                         "(default); fp64: every product on the FP64 pipe (hps_options.fp64_gemm)")
    args = ap.parse_args()
    if args.workload == "serve":
        args.spec = dict(SERVE)
        if args.requests:
            args.spec["requests"] = args.requests
        return args
    if args.workload == "diff":
        args.spec = {"workload": "diff_helmholtz2d_theta64_depth5_p16", "depth": 5, "p": 16, "k": 20.0,
                     "grid": 64, "seed": 5}
        return args
    if args.workload == "gemm":
        args.spec = {"workload": "gemm_lu_update_and_schur_shapes"}
        return args
    spec = dict(WORKLOADS[args.workload])
    if args.depth is not None and spec["depth"] >= 0 and args.depth != spec["depth"]:
        spec["depth"] = args.depth
        spec["n_leaves"] = (4 if spec["dim"] == 2 else 8) ** args.depth
        spec["workload"] = spec["workload"].replace(f"depth{WORKLOADS[args.workload]['depth']}",
                                                    f"depth{args.depth}")
    spec["root"] = args.root
    spec["gemm"] = args.gemm
    if args.gemm == "fp64":
        spec["workload"] += "_fp64gemm"
    args.spec = spec
    return args


def problem(spec, seed_offset=0):
    import workloads as W
    s = spec["seed_problem"] + seed_offset
    if spec["workload"].startswith("helmholtz"):
        return W.helmholtz_bumps_2d(seed=s, k=spec["k"], eta=spec["eta"])
    if spec["workload"].startswith("poisson"):
        return W.poisson_poly_2d(seed=s)
    if spec["workload"].startswith("elliptic"):
        return W.elliptic_3d(seed=s)
    return W.adaptive_3d(seed_coeffs=2 + seed_offset, seed_source=s)


def make_tree(P, spec, pr, depth=None):
    depth = spec["depth"] if depth is None else depth
    if depth >= 0:
        return P.uniform_tree(spec["dim"], depth, pr.lo, pr.hi), None
    fa = lambda x: pr.coeffs(x)["a"]  # noqa: E731
    fc = lambda x: pr.coeffs(x)["c"]  # noqa: E731
    leaves = P.hps_refine(pr.lo, pr.hi, spec["p"], spec["eps"], spec["min_depth"], spec["max_depth"],
                          [pr.source, fa, fc])
    return P.adaptive_tree(leaves, pr.lo, pr.hi), leaves


def host_inputs(P, spec, seed_offset=0, depth=None):
    """Coefficients (only the non-default ones), sources and boundary data
    sampled at the library's nodes."""
    pr = problem(spec, seed_offset)
    p, q = spec["p"], spec["q"]
    t, leaves = make_tree(P, spec, pr, depth)
    x, xb = P.hps_nodes(t, p, q)
    nl, ppl, nr = P.hps_sizes(t, p, q)
    cf = pr.coeffs(x)
    cdt = np.complex128 if spec["kind"] == "iti" else np.float64
    arrs = {}
    if not np.all(cf["a"] == 1.0):
        arrs["a"] = np.ascontiguousarray(cf["a"].reshape(nl, ppl))
    if any(np.any(bk != 0.0) for bk in cf["b"]):
        arrs["b"] = [np.ascontiguousarray(bk.reshape(nl, ppl)) for bk in cf["b"]]
    if np.any(cf["c"] != 0.0):
        arrs["c"] = np.ascontiguousarray(cf["c"].reshape(nl, ppl))
    f = np.ascontiguousarray(pr.source(x).reshape(nl, ppl).astype(cdt))
    g = np.ascontiguousarray(pr.boundary(xb).astype(cdt))
    rng = np.random.default_rng(COMMON["seed_solve_source"] + seed_offset)
    f2 = rng.standard_normal((nl, ppl)) * max(np.abs(f).max(), 1.0)
    if spec["kind"] == "iti":
        f2 = f2 + 1j * rng.standard_normal((nl, ppl)) * max(np.abs(f).max(), 1.0)
    return {"pr": pr, "t": t, "leaves": leaves, "coef": arrs, "f": f, "g": g,
            "f2": np.ascontiguousarray(f2.astype(cdt)), "nl": nl, "ppl": ppl}


# ------------------------------------------------------------------ clocks --

class ClockSampler:
    """nvidia-smi samples every 200 ms during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu = gpu_id
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


# ----------------------------------------------------------- replicas ----

def max_over_ranks(x: float, world: int, device=None) -> float:
    """Largest value of x over all ranks (the step time of the slowest
    replica); identity for a single process."""
    if world <= 1:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(steps: int, total_ms: float, world: int, device=None) -> float:
    """Whole-job solves/s of `world` independent replicas that each ran
    `steps` steps: all steps over the slowest replica's time."""
    return world * steps / (max_over_ranks(total_ms, world, device) / 1e3)


def pct(sorted_ms, q):
    """Nearest-rank percentile of an ascending list."""
    return sorted_ms[min(len(sorted_ms) - 1, int(round(q / 100.0 * (len(sorted_ms) - 1))))]


# ----------------------------------------------------------------- our arm --

def _build(P, spec, inp, arrs, f, profile=False):
    kind = P.HPS_ITI if spec["kind"] == "iti" else P.HPS_DTN
    return P.hps_build(inp["t"], spec["p"], spec["q"], kind, a=arrs.get("a"), b=arrs.get("b"), c=arrs.get("c"),
                       f=f, eta=spec.get("eta", 0.0), profile=profile, lazy_root=spec["root"] == "lazy",
                       fp64_gemm=spec.get("gemm") == "fp64")


def run_ours(args, rank, world):
    import torch
    import paper_2503_17535_gb300 as P

    spec = args.spec
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    inp = host_inputs(P, spec, seed_offset=rank)
    nl, ppl = inp["nl"], inp["ppl"]
    to_dev = lambda v: torch.from_numpy(v).to(dev)  # noqa: E731
    darr = {k: ([to_dev(x) for x in v] if isinstance(v, list) else to_dev(v)) for k, v in inp["coef"].items()}
    fd, gd, f2d = to_dev(inp["f"]), to_dev(inp["g"]), to_dev(inp["f2"])
    udt = torch.complex128 if spec["kind"] == "iti" else torch.float64
    ud = torch.zeros((nl, ppl), dtype=udt, device=dev)
    stream = torch.cuda.current_stream(dev)
    launches = [0]

    def step():
        h = _build(P, spec, inp, darr, fd)
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
    value = replica_throughput(args.steps, total_ms, world, dev)
    total_ms = max_over_ranks(total_ms, world, dev)

    # ---- build and solve timed separately (p50 / p99 over `steps` runs each):
    # hps_build alone, a solve with a new source (upward + downward pass) and
    # an apply-only solve (downward pass with the build-time source)
    def timed(fn, n):
        ts = []
        for _ in range(n):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            b.synchronize()
            ts.append(a.elapsed_time(b))
        ts.sort()
        return {"p50_ms": round(pct(ts, 50), 3), "p99_ms": round(pct(ts, 99), 3), "runs": n}

    hold = []

    def build_only():
        if hold:
            P.hps_free(hold.pop())
        hold.append(_build(P, spec, inp, darr, fd))

    phases = {"build": timed(build_only, args.steps)}
    hk = hold.pop()
    phases["solve_new_f"] = timed(lambda: P.hps_solve(hk, gd, ud, f=f2d), max(args.steps, 10))
    phases["solve_apply"] = timed(lambda: P.hps_solve(hk, gd, ud), max(args.steps, 10))
    P.hps_free(hk)

    # ---- one profiled step (untimed): per-class kernel times with CUDA events
    h = _build(P, spec, inp, darr, fd, profile=True)
    sb = P.hps_kernel_stats(h)
    tr = P.hps_trace(h) if args.trace else None
    P.hps_solve(h, gd, ud, f=f2d)
    ss = P.hps_kernel_stats(h)
    if args.trace and rank == 0:
        with open(args.trace, "w") as fh:
            json.dump({"workload": spec["workload"], "build": tr, "solve": P.hps_trace(h)}, fh)
    P.hps_free(h)
    classes = {k: {"launches": sb[k]["launches"] + ss[k]["launches"],
                   "flops": sb[k]["flops"] + ss[k]["flops"],
                   "exec_flops": sb[k]["exec_flops"] + ss[k]["exec_flops"],
                   "ms": sb[k]["ms"] + ss[k]["ms"]} for k in sb}
    flops_step = sum(v["flops"] for v in classes.values())
    dom = max(classes, key=lambda k: classes[k]["ms"])
    sm_mhz = clocks.get("sm_mhz") or 2070.0
    peak_tf = FP64_FLOP_PER_CLK_SM * 152 * sm_mhz * 1e6 / 1e12
    sec = classes[dom]["ms"] / 1e3
    ach = classes[dom]["flops"] / sec / 1e12 if sec > 0 else 0.0
    ach_exec = classes[dom]["exec_flops"] / sec / 1e12 if sec > 0 else 0.0
    if dom == "gemm_tc":
        # digit-slice products on the bf16 tensor cores: algorithmic FP64
        # flops against the scheme's ceiling, the measured sustained cuBLAS
        # bf16 rate (the kernel runs inside a long build) over the 55 bf16
        # digit products each FP64 multiply-add takes; the executed bf16
        # rate (padded tiles) beside it
        bf16, src = tensor_peak()
        ceil = bf16 / TC_DIGIT_PRODUCTS
        nl_launch = classes[dom]["launches"] or 1
        traffic = NCU_TRAFFIC.get((spec["workload"], dom))
        roofline = {"bound": "tensor", "kernel_class": dom, "achieved": round(ach, 4), "peak": round(ceil, 3),
                    "unit": "TFLOP/s", "frac": round(ach / ceil, 4),
                    "traffic": traffic["bytes_per_launch"] if traffic else None,
                    "flops_counted": "algorithmic FP64 flops of the products (real multiply-add 2, complex 8)",
                    "peak_source": f"{src}, divided by {TC_DIGIT_PRODUCTS} bf16 digit products per FP64 "
                                   "multiply-add (the digit-slice scheme's ceiling)",
                    "traffic_source": traffic["source"] if traffic else None,
                    "executed_bf16_tflops": round(ach_exec, 4), "executed_bf16_frac": round(ach_exec / bf16, 4),
                    "fp64_equivalent_vs_fp64_pipe": round(ach / peak_tf, 4),
                    "launches_per_step": nl_launch, "ms_per_step": round(classes[dom]["ms"], 3)}
    else:
        roofline = {"bound": "alu", "kernel_class": dom, "achieved": round(ach, 4), "peak": round(peak_tf, 4),
                    "unit": "TFLOP/s", "frac": round(ach / peak_tf, 4), "traffic": None,
                    "flops_counted": "algorithmic: real multiply-add = 2, complex multiply-add = 8",
                    "pipe_executed_tflops": round(ach_exec, 4), "pipe_frac": round(ach_exec / peak_tf, 4),
                    "peak_source": "FP64 FMA pipe: 4 flop/clk/SM x 152 SMs x median SM clock of this run",
                    "launches_per_step": classes[dom]["launches"], "ms_per_step": round(classes[dom]["ms"], 3)}

    # ---- end to end through the C ABI with host buffers
    e2e = None
    if not args.no_e2e:
        uh = np.zeros((nl, ppl), inp["f"].dtype)

        def step_host():
            h = _build(P, spec, inp, inp["coef"], inp["f"])
            P.hps_solve(h, inp["g"], uh, f=inp["f2"])
            P.hps_free(h)

        step_host()
        torch.cuda.synchronize()
        ts = time.perf_counter()
        for _ in range(args.steps):
            step_host()
        torch.cuda.synchronize()
        te = max_over_ranks(time.perf_counter() - ts, world, dev)
        coef_bytes = sum((sum(x.nbytes for x in v) if isinstance(v, list) else v.nbytes)
                         for v in inp["coef"].values())
        e2e = {"value": round(world * args.steps / te, 4), "unit": UNIT,
               "h2d_bytes_per_step": int(coef_bytes + inp["f"].nbytes + inp["g"].nbytes + inp["f2"].nbytes),
               "d2h_bytes_per_step": int(uh.nbytes)}
    return {"value": value, "total_ms": total_ms, "per": per, "clocks": clocks, "roofline": roofline,
            "fp64_peak": peak_tf,
            "classes": classes, "flops_step": flops_step, "launches": launches[0] // max(args.steps, 1),
            "e2e": e2e, "n_leaves": nl, "phases": phases}


# ------------------------------------------------------------- CPU oracle --

def oracle_sample_step(spec, depth=None):
    """One oracle build + new-source solve of the same problem (at a smaller
    depth when the spec names one); returns its wall time in seconds."""
    from oracle import adaptive as ad
    from oracle import hps as O
    pr = problem(spec)
    p, q = spec["p"], spec["q"]
    rng = np.random.default_rng(COMMON["seed_solve_source"])
    if spec["depth"] < 0:
        fa = lambda x: pr.coeffs(x)["a"]  # noqa: E731
        fc = lambda x: pr.coeffs(x)["c"]  # noqa: E731
        leaves = ad.refine([pr.source, fa, fc], pr.lo, pr.hi, p, spec["eps"], spec["min_depth"],
                           spec["max_depth"])
        x, a, b, c, f, g = ad.sample_adaptive(pr, leaves, p)
        f2 = rng.standard_normal(f.shape) * max(np.abs(f).max(), 1.0)
        t0 = time.perf_counter()
        ad.solve_adaptive(ad.build_adaptive(leaves, p, pr.lo, pr.hi, a, b, c, f2), g)
        return time.perf_counter() - t0
    depth = spec["depth"] if depth is None else depth
    x, a, b, c, f, g = O.sample_problem(pr, p, q, depth)
    f2 = rng.standard_normal(f.shape) * max(np.abs(f).max(), 1.0)
    if spec["kind"] == "iti":
        f2 = f2 + 1j * rng.standard_normal(f.shape) * max(np.abs(f).max(), 1.0)
    # the oracle has no separate particular pass: a build with the solve's
    # source followed by the solve gives the same u as build(f) + solve(new f)
    t0 = time.perf_counter()
    s2 = O.build(spec["dim"], spec["kind"], p, q, depth, pr.lo, pr.hi, a, b, c, f2, eta=pr.eta)
    O.solve(s2, g)
    return time.perf_counter() - t0


def oracle_times(args, depth, threads, reps=1):
    """Wall times (s) of `reps` oracle build + new-source solves at `depth`,
    run in a child process whose BLAS uses `threads` threads (the thread
    count must be set before NumPy loads)."""
    env = dict(os.environ)
    for var in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
        env[var] = str(threads)
    cmd = [sys.executable, os.path.abspath(__file__), "--workload", args.workload, "--oracle-sample",
           str(-1 if depth is None else depth), "--oracle-reps", str(reps)]
    out = subprocess.run(cmd, env=env, capture_output=True, text=True, check=True)
    return json.loads(out.stdout.strip().splitlines()[-1])["seconds"]


def run_oracle_sample(args):
    spec = args.spec
    depth = None if args.oracle_sample < 0 else args.oracle_sample
    ts = [oracle_sample_step(spec, depth) for _ in range(args.oracle_reps)]
    print(json.dumps({"seconds": ts}), flush=True)
    return 0


def sample_depth(spec):
    """Depth of the per-step oracle sample of the reference arm: one below
    the workload's (a step of a few seconds), the full problem when that is
    already small or adaptive."""
    if spec["depth"] < 0 or spec["depth"] <= 3:
        return None
    return spec["depth"] - 1


def cpu_baseline(args, spec):
    """The oracle on the host: the full problem once with --oracle-threads
    BLAS threads (the line's value, no scaling), and one single-threaded run
    of the one-level-smaller problem."""
    th = max(1, min(args.oracle_threads, os.cpu_count() or 1))
    t_full = min(oracle_times(args, None, th))
    out = {"value": round(1.0 / t_full, 6), "unit": UNIT, "cores": th, "kind": "oracle",
           "sample": (f"oracle (NumPy/SciPy LAPACK) build + new-source solve of the full problem "
                      f"({'depth ' + str(spec['depth']) if spec['depth'] >= 0 else 'the same refined tree'}): "
                      f"{t_full:.2f} s with {th} BLAS threads (OPENBLAS_NUM_THREADS={th}; host has "
                      f"{os.cpu_count()} cores)")}
    sd = sample_depth(spec)
    if sd is not None:
        t1 = min(oracle_times(args, sd, 1))
        out["single_thread"] = {"depth": sd, "seconds": round(t1, 3), "solves_per_s": round(1.0 / t1, 6),
                                "blas_threads": 1}
    return out


def run_reference(args, rank):
    """The oracle as the reference arm: each step one oracle build +
    new-source solve of the one-level-smaller problem (a few seconds), scaled
    to the full problem by the ratio of one full-size run to the mean of
    those samples, all with --oracle-threads BLAS threads."""
    if rank != 0:
        return None
    spec = args.spec
    th = max(1, min(args.oracle_threads, os.cpu_count() or 1))
    sd = sample_depth(spec)
    ts = oracle_times(args, sd, th, reps=args.warmup + args.steps)[args.warmup:]
    ratio, t_full = 1.0, None
    if sd is not None:
        t_full = min(oracle_times(args, None, th))
        ratio = t_full / statistics.mean(ts)
    scaled = [t * ratio for t in ts]
    value = args.steps / sum(scaled)
    cfg = dict(spec)
    cfg.update(COMMON)
    what = (f"each step: oracle build + new-source solve at depth {sd} (mean {statistics.mean(ts):.2f} s), "
            f"scaled by {ratio:.2f} = one full-depth run ({t_full:.2f} s) over that mean" if sd is not None
            else f"each step: oracle build + new-source solve of the full problem (mean {statistics.mean(ts):.2f} s)")
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 6), "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(1e3 * sum(scaled) / args.steps, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "c128" if spec["kind"] == "iti" else "f64",
            "data": "synthetic", "config": cfg,
            "cpu_baseline": {"value": round(value, 6), "unit": UNIT, "cores": th, "kind": "oracle",
                             "sample": what + f"; {th} BLAS threads of {os.cpu_count()} host cores"},
            "e2e": {"value": round(value, 6), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    return line


# ----------------------------------------------------------------- serving --

def serve_operators(P, spec):
    """The seeded operator set: (kind, depth, p) per slot, redrawn with the
    next seed while the planned footprint exceeds op_budget_gb."""
    seed = spec["seed"]
    while True:
        rng = np.random.default_rng(seed)
        ops = []
        for i in range(spec["n_ops"]):
            kind = spec["kinds"][int(rng.integers(0, len(spec["kinds"])))]
            depth = int(rng.integers(spec["depths"][0], spec["depths"][1] + 1))
            p = int(spec["ps"][int(rng.integers(0, len(spec["ps"])))])
            ops.append({"kind": kind, "depth": depth, "p": p, "q": p - 2})
        tot = sum(P.hps_plan_bytes(P.uniform_tree(2, o["depth"]), o["p"], o["q"],
                                   P.HPS_ITI if o["kind"] == "iti" else P.HPS_DTN) for o in ops)
        if tot <= spec["op_budget_gb"] * 1e9:
            return ops, seed, tot
        seed += 1000


def serve_inputs(P, op, field_seed, rng):
    """Coefficient arrays of one operator (coefficient field seed), plus
    solve inputs drawn from rng."""
    import workloads as W
    pr = (W.helmholtz_bumps_2d(seed=field_seed) if op["kind"] == "iti" else W.elliptic_2d(seed=field_seed))
    t = P.uniform_tree(2, op["depth"], pr.lo, pr.hi)
    x, xb = P.hps_nodes(t, op["p"], op["q"])
    nl, ppl, nr = P.hps_sizes(t, op["p"], op["q"])
    cf = pr.coeffs(x)
    cdt = np.complex128 if op["kind"] == "iti" else np.float64
    d = {"t": t, "kind": P.HPS_ITI if op["kind"] == "iti" else P.HPS_DTN, "eta": pr.eta or 0.0,
         "a": np.ascontiguousarray(cf["a"].reshape(nl, ppl)),
         "b": [np.ascontiguousarray(bk.reshape(nl, ppl)) for bk in cf["b"]],
         "c": np.ascontiguousarray(cf["c"].reshape(nl, ppl)),
         "f": np.ascontiguousarray(pr.source(x).reshape(nl, ppl).astype(cdt)), "shape": (nl, ppl), "cdt": cdt}
    return d


def serve_measure(spec):
    """Served requests/s and p50 / p99 latency of the request server against
    the plain path (one request at a time, hps_build / hps_solve directly) on
    the same seeded request stream and arrival times, at each load of
    spec["rates"] (a multiple of the plain path's measured capacity)."""
    import torch
    import paper_2503_17535_gb300 as P

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    ops, op_seed, op_bytes = serve_operators(P, spec)
    rng = np.random.default_rng(op_seed + 1)
    pools = []
    for i, op in enumerate(ops):
        fields = [serve_inputs(P, op, 100 + 10 * i + k, rng) for k in range(spec["pool"])]
        sol = []
        for k in range(spec["pool"]):
            d = fields[0]
            nl, ppl = d["shape"]
            nr = P.hps_sizes(d["t"], op["p"], op["q"])[2]
            g = rng.standard_normal(nr)
            f = rng.standard_normal((nl, ppl))
            if d["cdt"] == np.complex128:
                g = g + 1j * rng.standard_normal(nr)
                f = f + 1j * rng.standard_normal((nl, ppl))
            sol.append((np.ascontiguousarray(g.astype(d["cdt"])), np.ascontiguousarray(f.astype(d["cdt"]))))
        pools.append({"fields": fields, "solves": sol})
    R = spec["requests"]
    req = []
    for r in range(R):
        slot = int(rng.integers(0, len(ops)))
        if rng.random() < spec["rebuild_frac"]:
            req.append(("build", slot, int(rng.integers(1, spec["pool"]))))
        else:
            req.append(("solve", slot, int(rng.integers(0, spec["pool"]))))

    def plain_initial():
        hs = []
        for i, op in enumerate(ops):
            d = pools[i]["fields"][0]
            hs.append(P.hps_build(d["t"], op["p"], op["q"], d["kind"], a=d["a"], b=d["b"], c=d["c"], f=d["f"],
                                  eta=d["eta"], lazy_root=True))
        torch.cuda.synchronize()
        return hs

    def plain_run(arrivals):
        hs = plain_initial()
        outs = [np.zeros(pools[i]["fields"][0]["shape"], pools[i]["fields"][0]["cdt"]) for i in range(len(ops))]
        t0 = time.perf_counter()
        lat, service = [], []
        for r, (kind, slot, k) in enumerate(req):
            if arrivals is not None:
                wait = arrivals[r] - (time.perf_counter() - t0)
                if wait > 0:
                    time.sleep(wait)
            ts = time.perf_counter()
            op = ops[slot]
            if kind == "build":
                d = pools[slot]["fields"][k]
                P.hps_free(hs[slot])
                hs[slot] = P.hps_build(d["t"], op["p"], op["q"], d["kind"], a=d["a"], b=d["b"], c=d["c"],
                                       f=d["f"], eta=d["eta"], lazy_root=True)
                torch.cuda.synchronize()
            else:
                g, _ = pools[slot]["solves"][k]
                P.hps_solve(hs[slot], g, outs[slot])   # apply-only: new g, the build-time source
            te = time.perf_counter()
            service.append(te - ts)
            lat.append(te - t0 - (arrivals[r] if arrivals is not None else (ts - t0)))
        span = time.perf_counter() - t0
        for h in hs:
            P.hps_free(h)
        return {"lat_ms": [1e3 * v for v in lat], "service_s": service, "span_s": span}

    def served_run(arrivals):
        S = P.Server(n_slots=len(ops), n_streams=spec["n_streams"], max_batch=spec["max_batch"], lazy_root=True)
        # one output buffer per slot: the benchmark does not read the results
        # (the GPU tests check them), so requests of a slot may share it
        outs = [np.zeros(pools[i]["fields"][0]["shape"], pools[i]["fields"][0]["cdt"]) for i in range(len(ops))]
        for i, op in enumerate(ops):
            d = pools[i]["fields"][0]
            S.wait(S.submit_build(i, d["t"], op["p"], op["q"], d["kind"], a=d["a"], b=d["b"], c=d["c"],
                                  f=d["f"], eta=d["eta"]))
        t0 = time.perf_counter()
        tickets = []
        for r, (kind, slot, k) in enumerate(req):
            wait = arrivals[r] - (time.perf_counter() - t0)
            if wait > 0:
                time.sleep(wait)
            op = ops[slot]
            if kind == "build":
                d = pools[slot]["fields"][k]
                tickets.append(S.submit_build(slot, d["t"], op["p"], op["q"], d["kind"], a=d["a"], b=d["b"],
                                              c=d["c"], f=d["f"], eta=d["eta"]))
            else:
                g, _ = pools[slot]["solves"][k]
                tickets.append(S.submit_solve(slot, g, outs[slot]))   # apply-only
        infos = [S.wait(t) for t in tickets]
        st = S.stats()
        S.close()
        lat = [i["t_done_ms"] - i["t_submit_ms"] for i in infos]
        span = (max(i["t_done_ms"] for i in infos) - min(i["t_submit_ms"] for i in infos)) / 1e3
        return {"lat_ms": lat, "span_s": span, "max_batch": st["max_batch_seen"], "batches": st["batches"],
                "multi_batches": st["multi_batches"], "max_group": st["max_group_seen"]}

    def pct_of(v, q):
        return round(float(np.percentile(np.asarray(v), q)), 3)

    base = plain_run(None)  # back to back: the one-at-a-time capacity
    cap = R / sum(base["service_s"])
    rates = []
    for rho in spec["rates"]:
        lam = rho * cap
        arr = np.cumsum(np.random.default_rng(spec["seed"] + int(100 * rho)).exponential(1.0 / lam, size=R))
        arr -= arr[0]
        sv = served_run(arr)
        pl = plain_run(arr)
        rates.append({"load": rho, "offered_per_s": round(lam, 3),
                      "served": {"solves_per_s": round(R / sv["span_s"], 3), "p50_ms": pct_of(sv["lat_ms"], 50),
                                 "p99_ms": pct_of(sv["lat_ms"], 99), "max_batch": sv["max_batch"],
                                 "batches": sv["batches"], "multi_operator_batches": sv["multi_batches"],
                                 "max_operators_in_a_batch": sv["max_group"]},
                      "plain": {"solves_per_s": round(R / pl["span_s"], 3), "p50_ms": pct_of(pl["lat_ms"], 50),
                                "p99_ms": pct_of(pl["lat_ms"], 99)}})
    n_build = sum(1 for r in req if r[0] == "build")
    return {"rates": rates, "ops": ops, "op_seed": op_seed, "op_bytes": op_bytes, "cap": cap,
            "n_build": n_build, "R": R}


def run_serve(args, rank, world):
    spec = args.spec
    m = serve_measure(spec)
    rates, ops, op_seed, op_bytes, cap, n_build, R = (m["rates"], m["ops"], m["op_seed"], m["op_bytes"],
                                                      m["cap"], m["n_build"], m["R"])
    top = rates[-1]
    cfg = {k: v for k, v in spec.items() if k not in ("op_budget_gb",)}
    cfg.update({"operators": ops, "operator_seed": op_seed, "operator_bytes": int(op_bytes),
                "requests_build": n_build, "requests_solve": R - n_build, "root": "lazy",
                "plain_capacity_per_s": round(cap, 3),
                "value_at": f"load {top['load']} x plain capacity (saturated): whole-run served requests/s"})
    line = {"metric": METRIC, "value": top["served"]["solves_per_s"], "unit": "requests/s", "n_gpus": world,
            "steps": R, "warmup": 0, "p50_ms": top["served"]["p50_ms"], "p99_ms": top["served"]["p99_ms"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64+c128",
            "data": "synthetic", "config": cfg, "rates": rates,
            "vs_plain": round(top["served"]["solves_per_s"] / max(top["plain"]["solves_per_s"], 1e-9), 3)}
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def serving_leg(args):
    """A short run of the serving workload for the default line: its seeded
    operators and request mix (apply-only solves and rebuilds) at 0.9 x and
    1.5 x the plain path's capacity."""
    spec = dict(SERVE)
    spec["requests"] = 40
    spec["rates"] = [0.9, 1.5]
    m = serve_measure(spec)
    r = m["rates"][0]
    return {"workload": spec["workload"], "operators": m["ops"], "requests": m["R"],
            "requests_build": m["n_build"], "mix": "apply-only solves (new g, build-time source) and rebuilds",
            "load": r["load"], "offered_per_s": r["offered_per_s"],
            "plain_capacity_per_s": round(m["cap"], 3), "served": r["served"], "plain": r["plain"],
            "more_loads": [{"load": q["load"], "offered_per_s": q["offered_per_s"], "served": q["served"],
                            "plain": q["plain"]} for q in m["rates"][1:]],
            "unit": "requests/s", "latency": "host clock, submit to result on the host"}


# ------------------------------------------------------------ differentiation --

def run_diff(args, rank, world):
    """Gradient of J(theta) = ||u(theta) - u(theta_true)||^2 over a 64 x 64
    grid theta (Helmholtz operator, 1024 leaves, p = 16): one step = forward
    (build + solve) and backward (adjoint solve + coefficient gradient +
    interpolation transpose) through the autograd Function."""
    import torch
    import paper_2503_17535_gb300 as P
    import workloads as W
    from paper_2503_17535_gb300.autograd import hps_solve_fn

    spec = args.spec
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    d = W.helmholtz_theta_2d(seed=spec["seed"], k=spec["k"], n=spec["grid"])
    pr, k = d["problem"], d["k"]
    p, L = spec["p"], spec["depth"]
    t = P.uniform_tree(2, L, pr.lo, pr.hi)
    x, xb = P.hps_nodes(t, p, p - 2)
    nl, ppl, nr = P.hps_sizes(t, p, p - 2)
    I = W.grid_interp_matrix(x, d["n"]).tocoo()
    Imat = torch.sparse_coo_tensor(np.vstack([I.row, I.col]), I.data, I.shape, dtype=torch.float64,
                                   device="cuda").coalesce()
    f = torch.from_numpy(np.ascontiguousarray(pr.source(x).reshape(nl, ppl).astype(np.complex128))).cuda()
    g = torch.from_numpy(np.ascontiguousarray(pr.boundary(xb).astype(np.complex128))).cuda()

    def forward(theta):
        c = (k ** 2 * (1.0 - torch.sparse.mm(Imat, theta[:, None])[:, 0])).reshape(nl, ppl)
        return hps_solve_fn(c, g, f, t, p, P.HPS_ITI, eta=pr.eta, lazy_root=True)

    with torch.no_grad():
        u_obs = forward(torch.from_numpy(d["theta_true"]).cuda())
    theta0 = torch.from_numpy(d["theta_0"]).cuda()

    def step():
        th = theta0.clone().requires_grad_(True)
        J = ((forward(th) - u_obs).abs() ** 2).sum()
        J.backward()
        return th.grad

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for i in range(args.steps):
        evs[i][0].record(stream)
        step()
        evs[i][1].record(stream)
    t1.record(stream)
    torch.cuda.synchronize()
    total = t0.elapsed_time(t1)
    per = sorted(a.elapsed_time(b) for a, b in evs)
    line = {"metric": "gradients/s of J(theta) through the adjoint kernels", "value": round(args.steps / (total / 1e3), 4),
            "unit": "gradients/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(total / args.steps, 3), "p50_ms": round(pct(per, 50), 3),
            "p99_ms": round(pct(per, 99), 3), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "c128", "data": "synthetic",
            "config": {"workload": spec["workload"], "n_leaves": nl, "p": p, "grid": spec["grid"],
                       "step": "forward (build + solve) + backward (adjoint solve + coefficient gradient)",
                       "root": "lazy"}}
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def run_gemm(args, rank, world):
    """The build's two product shapes alone through hps_gemm: an LU / triangular
    update (inner dimension 32) and a Schur complement (inner dimension 448),
    C -= A B in FP64, on the tensor cores (mode 0) and on the FP64 pipe
    (mode 1); checks mode 0 against mode 1 and times both with CUDA events
    (each call synchronises and allocates its workspace, so the times include
    that host overhead; ncu gives the kernel alone)."""
    import torch
    import paper_2503_17535_gb300 as P
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    out = {}
    for name, (m, n, k, b) in {"lu_update": (1696, 3457, 32, 2), "schur": (448, 1793, 448, 4)}.items():
        g = torch.Generator(device="cuda").manual_seed(m + n + k)
        A = torch.randn(b, k, m, dtype=torch.float64, device="cuda", generator=g)
        B = torch.randn(b, n, k, dtype=torch.float64, device="cuda", generator=g)
        C0 = torch.randn(b, n, m, dtype=torch.float64, device="cuda", generator=g)
        res = {}
        for mode in (0, 1):
            C = C0.clone()
            P.hps_gemm(A, B, C, alpha=-1.0, beta=1.0, mode=mode)   # warm-up (and result)
            ts = []
            for _ in range(max(args.steps, 1)):
                Ct = C0.clone()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                P.hps_gemm(A, B, Ct, alpha=-1.0, beta=1.0, mode=mode)
                e1.record()
                e1.synchronize()
                ts.append(e0.elapsed_time(e1))
            res[mode] = (C, statistics.median(ts))
        mag = torch.bmm(A.abs().transpose(1, 2), B.abs().transpose(1, 2))
        err = ((res[0][0] - res[1][0]).abs().transpose(1, 2) / (mag + 1.0)).max().item()
        if err >= 1e-13:
            raise SystemExit(f"gemm {name}: tensor-core result differs from the FP64 pipe by {err:.3e}")
        fl = 2.0 * m * n * k * b
        out[name] = {"m": m, "n": n, "k": k, "batch": b, "max_err_rel_AB": err,
                     "tc_ms": round(res[0][1], 4), "fp64_ms": round(res[1][1], 4),
                     "tc_fp64_equiv_tflops": round(fl / res[0][1] / 1e9, 3),
                     "fp64_tflops": round(fl / res[1][1] / 1e9, 3)}
    if rank == 0:
        print(json.dumps({"metric": "hps_gemm FP64 products: tensor-core digit slices vs FP64 pipe",
                          "unit": "ms", "higher_is_better": False, "data": "synthetic",
                          "config": {"workload": args.spec["workload"]}, "shapes": out}), flush=True)
    return 0


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.workload == "serve":
        return run_serve(args, rank, world)
    if args.workload == "diff":
        return run_diff(args, rank, world)
    if args.workload == "gemm":
        return run_gemm(args, rank, world)
    spec = args.spec
    if args.oracle_sample is not None:
        return run_oracle_sample(args)
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
        p50, p99 = pct(per, 50), pct(per, 99)
        step_tf = r["flops_step"] / (statistics.median(per) / 1e3) / 1e12
        cfg = dict(spec)
        cfg.update(COMMON)
        cfg["n_leaves"] = r["n_leaves"]
        cfg["parallelism"] = f"replicas x{world}"
        line = {"metric": METRIC, "value": round(r["value"], 4), "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": round(r["total_ms"] / args.steps, 3), "p50_ms": round(p50, 3),
                "p99_ms": round(p99, 3), "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "c128" if spec["kind"] == "iti" else "f64", "data": "synthetic",
                "config": cfg, "clocks": r["clocks"], "e2e": r["e2e"], "gpu_launches": r["launches"] * args.steps,
                "roofline": r["roofline"], "phases": r["phases"],
                "step_fp64": {"algorithmic_flops": r["flops_step"], "achieved_tflops": round(step_tf, 4),
                              "fp64_pipe_peak_tflops": round(r["fp64_peak"], 4),
                              "frac_of_fp64_pipe_peak": round(step_tf / r["fp64_peak"], 4)},
                "kernel_classes": {k: {"launches": v["launches"], "ms": round(v["ms"], 3),
                                       "gflops": round(v["flops"] / 1e9, 3),
                                       "exec_gflops": round(v["exec_flops"] / 1e9, 3)}
                                   for k, v in r["classes"].items()}}
        if world == 1 and not args.no_serve and spec["workload"].startswith("helmholtz"):
            line["serving"] = serving_leg(args)
        if world == 1 and not args.no_cpu:
            line["cpu_baseline"] = cpu_baseline(args, spec)
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
