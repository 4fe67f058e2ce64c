"""Autotuner for the batched LU shapes and the tensor-core routing thresholds.

The library reads its shape choices from a process-wide table (hps_tune_set /
hps_tune_get in include/hps.h) whose defaults are compiled in from
csrc/tuned.h.  This tool times hps_build on the benchmark workloads -- the
Helmholtz ItI operator (k = 20, p = 16, 4096 leaves), the 3D elliptic
operator (p = 8, 512 leaves) and the adaptive 3D octree (p = 8, leaf depths
2-5) -- for candidate values of each parameter, by coordinate descent (two
passes over the parameters, the others held at their current best), and
writes the setting with the smallest summed median build time to tuned.h.
Every setting gives the same factorisation up to rounding (same pivots), so
only time is compared.

    python -m paper_2503_17535_gb300.autotune [--out PATH] [--reps 3] [--params a,b]

Needs a GPU; rebuild the library afterwards to make the values the defaults.
"""

from __future__ import annotations

import argparse
import json
import os
import statistics
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)

CANDIDATES = {
    "lu_cluster_panel": [0, 1],
    "lu_base_panels_few": [0, 4, 8, 16, 32],
    "lu_few_min_n": [1024, 2048, 4096, 8192],
    "lu_base_panels_many": [2, 4, 8],
    "tc_min_work_real": [25, 50, 100, 200, 400],
    "tc_min_work_cplx": [6, 12, 25, 50, 100],
    "tc_min_k": [16, 33, 48, 64, 96],
    "tc_chunk_mb": [16, 32, 64, 128, 1024],
    "tc_persist_min_k": [0, 48, 64, 128, 1 << 20],
    "lu_panel_nb_few": [16, 32],
}
MACROS = {
    "lu_base_panels_few": "HPS_TUNED_LU_BASE_PANELS_FEW",
    "lu_base_panels_many": "HPS_TUNED_LU_BASE_PANELS_MANY",
    "lu_few_min_n": "HPS_TUNED_LU_FEW_MIN_N",
    "lu_cluster_panel": "HPS_TUNED_LU_CLUSTER_PANEL",
    "tc_min_work_real": "HPS_TUNED_TC_MIN_WORK_REAL",
    "tc_min_work_cplx": "HPS_TUNED_TC_MIN_WORK_CPLX",
    "tc_min_k": "HPS_TUNED_TC_MIN_K",
    "tc_chunk_mb": "HPS_TUNED_TC_CHUNK_MB",
    "tc_persist_min_k": "HPS_TUNED_TC_PERSIST_MIN_K",
    "lu_panel_nb_few": "HPS_TUNED_LU_PANEL_NB_FEW",
}


def workloads(P, torch):
    """(name, build callable) for the three benchmark operators; inputs are
    sampled once and kept on the device."""
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import numpy as np
    import workloads as W

    def dev(x):
        return torch.from_numpy(np.ascontiguousarray(x)).cuda()

    out = []
    for name, pr, p, depth in (("helmholtz2d_iti_p16_depth6", W.helmholtz_bumps_2d(seed=1), 16, 6),
                               ("elliptic3d_dtn_p8_depth3", W.elliptic_3d(seed=2), 8, 3),
                               ("adaptive3d_dtn_p8", W.adaptive_3d(), 8, -1)):
        q = p - 2
        if depth >= 0:
            t = P.uniform_tree(pr.dim, depth, pr.lo, pr.hi)
        else:
            leaves = P.hps_refine(pr.lo, pr.hi, p, 1e-4, 2, 5, [pr.source, lambda x: pr.coeffs(x)["a"],
                                                                lambda x: pr.coeffs(x)["c"]])
            t = P.adaptive_tree(leaves, pr.lo, pr.hi)
        x, _ = P.hps_nodes(t, p, q)
        nl, ppl, _ = P.hps_sizes(t, p, q)
        cf = pr.coeffs(x)
        a = dev(cf["a"].reshape(nl, ppl))
        b = [dev(bk.reshape(nl, ppl)) for bk in cf["b"]]
        c = dev(cf["c"].reshape(nl, ppl))
        cdt = np.complex128 if pr.kind == "iti" else np.float64
        f = dev(pr.source(x).reshape(nl, ppl).astype(cdt))
        kind = P.HPS_ITI if pr.kind == "iti" else P.HPS_DTN

        def build(t=t, p=p, q=q, kind=kind, a=a, b=b, c=c, f=f, eta=pr.eta or 0.0):
            h = P.hps_build(t, p, q, kind, a=a, b=b, c=c, f=f, eta=eta, lazy_root=True)
            P.hps_free(h)

        out.append((name, build))
    return out


def time_setting(P, torch, setting, ops, reps):
    for k, v in setting.items():
        P.hps_tune_set(k, v)
    res = {}
    for name, build in ops:
        build()  # warm-up
        ts = []
        for _ in range(reps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            build()
            torch.cuda.synchronize()
            ts.append(1e3 * (time.perf_counter() - t0))
        res[name] = statistics.median(ts)
    return res


def write_header(path, best, table):
    lines = ["// Shape choices of the batched LU and the tensor-core routing thresholds on",
             "// GB300 (hps_tune_set in include/hps.h).  Written by",
             "// paper_2503_17535_gb300/autotune.py from timed builds of the benchmark",
             "// workloads (summed median build time, ms, at the chosen values:",
             f"// {json.dumps(table)}); rerun it to regenerate.",
             "#pragma once", ""]
    for k in CANDIDATES:
        lines.append(f"#define {MACROS[k]} {best[k]}")
    with open(path, "w") as fh:
        fh.write("\n".join(lines) + "\n")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=os.path.join(HERE, "csrc", "tuned.h"))
    ap.add_argument("--log", default=None, help="write every measurement (JSON) to this path")
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--passes", type=int, default=2)
    ap.add_argument("--params", default=None,
                    help="comma-separated parameters to tune (default: all); the others keep their values")
    args = ap.parse_args()
    tuned = list(CANDIDATES) if not args.params else args.params.split(",")
    for k in tuned:
        if k not in CANDIDATES:
            raise SystemExit(f"unknown parameter {k}; known: {', '.join(CANDIDATES)}")
    import torch
    import paper_2503_17535_gb300 as P
    if not torch.cuda.is_available():
        raise SystemExit("the autotuner needs a CUDA device")
    torch.cuda.set_device(0)
    ops = workloads(P, torch)
    best = {k: P.hps_tune_get(k) for k in CANDIDATES}
    log = []
    cur = time_setting(P, torch, best, ops, args.reps)
    log.append({"setting": dict(best), "ms": cur})
    best_total = sum(cur.values())
    print("start", best, round(best_total, 1), flush=True)
    for _ in range(args.passes):
        for k in tuned:
            for v in CANDIDATES[k]:
                if v == best[k]:
                    continue
                trial = dict(best)
                trial[k] = v
                ms = time_setting(P, torch, trial, ops, args.reps)
                log.append({"setting": trial, "ms": ms})
                tot = sum(ms.values())
                print(k, v, {n: round(x, 1) for n, x in ms.items()}, round(tot, 1), flush=True)
                if tot < best_total * 0.995:
                    best, best_total, cur = trial, tot, ms
    for k, v in best.items():
        P.hps_tune_set(k, v)
    print("best", best, {n: round(x, 1) for n, x in cur.items()}, round(best_total, 1), flush=True)
    write_header(args.out, best, {n: round(x, 2) for n, x in cur.items()})
    if args.log:
        with open(args.log, "w") as fh:
            json.dump({"best": best, "best_ms": cur, "trials": log}, fh, indent=1)


if __name__ == "__main__":
    main()
