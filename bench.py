#!/usr/bin/env python
"""Benchmark of the LC covariance hot path on the mid workload.

Workload (per GPU, weak scaling): 100 mocks in a periodic box L = 1000 Mpc/h,
N_d = 100 000 Neyman-Scott points (parents 1e-5 (Mpc/h)^-3, sigma = 3 Mpc/h)
and two uniform random subsets R1, R2 of N_d points each (the M_a = 1 pair of
the linear construction), 40 linear s bins on [0, 200) Mpc/h x 10 mu bins
with the x line of sight.

One step = the whole hot path: quantisation + chaining-mesh build + pair
counts DD, DR1, DR2, RR1, RR2 of every mock (one persistent launch) + split
Landy-Szalay for R1, R2 and R1 u R2 + the LC covariance (Eqs. R1R2, LCdef)
with M = 50.  `value` is mocks/s with inputs resident in HBM; `e2e` is the
same metric through the public API with the positions copied from pinned
host memory and C^LC copied back inside every step.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
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
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "G pairs/s binned + LC-cov mocks/s, batched vs per-mock launch; cov err vs FP64"
LANE_OPS_PER_CAND = 7      # 3 sub + 3 mul/fma + 1 compare per candidate pair
LANE_OPS_PER_BINNED = 8    # s-bin, mu-bin, address, shared atomic per binned pair
SM_MAX_MHZ = 2070.0        # GB300 maximum SM clock
LANES_PER_SM = 128         # FP32/INT32 lanes per SM
M_FINAL = 50.0             # random-catalogue size of the target covariance (the paper's M = 50)


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    p.add_argument("--mocks", type=int, default=synth.MID.n_mock, help="mocks per GPU")
    p.add_argument("--nd", type=int, default=synth.MID.n_d, help="data points per mock")
    p.add_argument("--precision", default="tf32x3", choices=["fp64", "tf32x3", "bf16x3"])
    p.add_argument("--no-precision-config", action="store_true",
                   help="skip the covariance-only measurement on 3500 mocks x 200 bins")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--subdiv", type=int, default=0, help="pin the mesh subdivision (0: library choice)")
    p.add_argument("--cpu-seconds", type=float, default=12.0)
    p.add_argument("--batching-mocks", type=int, default=8,
                   help="mocks of the cut-sky batching shape timed as context (0: skip)")
    p.add_argument("--scale-mocks", type=int, default=2,
                   help="mocks of the scale shape (1e6 points) timed as context (0: skip)")
    p.add_argument("--smp-mocks", type=int, default=4,
                   help="mocks of the brute-force (Smp, M=50) comparison run; 0 skips it")
    p.add_argument("--cov-only", action="store_true",
                   help="two split-precision LC covariances of 3500 mocks x 200 bins, then exit (profiler captures)")
    p.add_argument("--count-only", action="store_true",
                   help="one warm-up and one batched tpcf_count of the workload, then exit (profiler captures)")
    p.add_argument("--count-only-batching", type=int, default=0, metavar="N",
                   help="like --count-only on N mocks of the cut-sky batching shape (midpoint line of sight)")
    return p.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={self.FIELDS}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self) -> dict:
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.f.name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# workload
# ---------------------------------------------------------------------------

def make_host_inputs(n_mock, n_d, first_mock):
    """Positions of all mocks in one float64 array; per mock (data, R1, R2) offsets."""
    w = synth.MID
    blocks, layout = [], []
    off = 0
    for m in range(first_mock, first_mock + n_mock):
        mk = w.make_mock(m, n_d=n_d, M=2)
        parts = [mk.data] + mk.randoms
        sizes = [len(x) for x in parts]
        layout.append((off, sizes))
        blocks.extend(parts)
        off += sum(sizes)
    return np.concatenate(blocks), layout


def mock_views(pos_dev, layout):
    mocks = []
    for off, (nd, n1, n2) in layout:
        mocks.append({"data": pos_dev[off:off + nd], "randoms": pos_dev[off + nd:off + nd + n1 + n2],
                      "offsets": [0, n1, n1 + n2]})
    return mocks


# ---------------------------------------------------------------------------
# CPU oracle timing (bounded sample of the same workload)
# ---------------------------------------------------------------------------

def oracle_sample_rate(n_d, target_s, seed_mock=0):
    """Time the oracle's brute-force counts on a row sample of one mid mock.

    The five terms of one mock cost 3.5 N_d^2 pair tests (DD and RR_i: N_d^2/2
    each, DR_i: N_d^2 each).  A sample of k a-rows against all b-points runs
    k N_d tests per term; the rate in mocks/s is the executed fraction of the
    mock's pair tests divided by the time taken.
    """
    import oracle
    w = synth.MID
    mk = w.make_mock(seed_mock, n_d=n_d, M=2)
    ob = oracle.Binning(w.s_edges, w.n_mu, oracle.PERIODIC, w.L)
    qd = oracle.quantize(mk.data, oracle.PERIODIC, w.L)
    qr = [oracle.quantize(r, oracle.PERIODIC, w.L) for r in mk.randoms]

    def run(k):
        t0 = time.perf_counter()
        tests = 0
        a = np.ascontiguousarray(qd[:, :k])
        oracle.count_pairs(a, qd, ob)      # DD rows against all points
        tests += k * n_d
        for r in qr:
            oracle.count_pairs(a, r, ob)   # DR_i rows
            tests += k * n_d
            ar = np.ascontiguousarray(r[:, :k])
            oracle.count_pairs(ar, r, ob)  # RR_i rows against all points
            tests += k * n_d
        return time.perf_counter() - t0, tests

    k = max(16, n_d // 2000)
    dt, tests = run(k)
    # grow the sample until it takes at least ~70% of the target time (or the whole mock)
    while dt < 0.7 * target_s and k < n_d:
        k = int(min(n_d, max(2 * k, k * 0.9 * target_s / max(dt, 1e-3))))
        dt, tests = run(k)
    full = 3.5 * n_d * n_d
    frac = tests / full
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    return {"mocks_per_s": frac / dt, "seconds": dt, "rows": k, "fraction_of_mock": frac, "cores": cores,
            "pair_tests_per_s": tests / dt}


def smp_measure(tp, ctx, dev, b, prec, n_mock, n_d, M=50, reps=2):
    """Brute-force (Smp) path on the mid shape: every mock against all M random
    subsets in one batched launch, LS over all subsets, sample covariance
    (Eq. bruteforce).  Returns ms per step and the pair totals."""
    import torch
    w = synth.MID
    mks = [w.make_mock(m, n_d=n_d, M=M) for m in range(n_mock)]
    dm = [{"data": torch.from_numpy(mk.data).to(dev),
           "randoms": torch.from_numpy(np.concatenate(mk.randoms)).to(dev),
           "offsets": [i * n_d for i in range(M + 1)]} for mk in mks]
    nbin = w.n_s * w.n_mu
    out = {"dd": torch.empty((n_mock, nbin), dtype=torch.int64, device=dev),
           "dr": torch.empty((n_mock, M, nbin), dtype=torch.int64, device=dev),
           "rr": torch.empty((n_mock, M, nbin), dtype=torch.int64, device=dev)}
    xi = torch.empty((n_mock, nbin), dtype=torch.float64, device=dev)
    sel = list(range(M))
    n_r = [[n_d] * M for _ in range(n_mock)]

    def step():
        ctx.tpcf_count(dm, b, mode=tp.TPCF_BATCHED, out=out)
        ctx.tpcf_ls(out["dd"], out["dr"], out["rr"], [n_d] * n_mock, n_r, sel, out=xi)
        return ctx.tpcf_sample_cov(xi, prec)

    step()
    torch.cuda.synchronize()
    ctx.tpcf_set_timing(True)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    info = ctx.tpcf_last_count_info()
    ctx.tpcf_set_timing(False)
    rc = ctx.tpcf_sync()
    return {"ms": e0.elapsed_time(e1) / reps, "n_binned": info["n_binned"], "n_candidates": info["n_candidates"],
            "status": rc}


def batching_measure(tp, ctx, dev, n_mock, reps=2):
    """The cut-sky batching workload's shape on a sample of its mocks: uneven N_d (Poisson-scattered in
    50k-400k), octant shell 1200-2400 Mpc/h, midpoint line of sight, R1 + R2 of N_d each, 40 s x 5 mu
    bins; all mocks and terms in one batched call.  Returns ms per call and the pair totals."""
    import torch
    w = synth.BATCHING
    mks = [w.make_mock(m) for m in range(n_mock)]
    dm = [{"data": torch.from_numpy(mk.data).to(dev),
           "randoms": torch.from_numpy(np.concatenate(mk.randoms)).to(dev),
           "offsets": [0, len(mk.randoms[0]), len(mk.randoms[0]) + len(mk.randoms[1])]} for mk in mks]
    b = tp.make_binning(w.s_edges, w.n_mu, tp.TPCF_OPEN, w.L, los=tp.TPCF_LOS_MIDPOINT, observer=w.observer)
    nbin = w.n_s * w.n_mu
    out = {"dd": torch.empty((n_mock, nbin), dtype=torch.int64, device=dev),
           "dr": torch.empty((n_mock, 2, nbin), dtype=torch.int64, device=dev),
           "rr": torch.empty((n_mock, 2, nbin), dtype=torch.int64, device=dev)}
    for _ in range(2):
        ctx.tpcf_count(dm, b, mode=tp.TPCF_BATCHED, out=out)
    torch.cuda.synchronize()
    ctx.tpcf_set_timing(True)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        ctx.tpcf_count(dm, b, mode=tp.TPCF_BATCHED, out=out)
    e1.record(stream)
    torch.cuda.synchronize()
    info = ctx.tpcf_last_count_info()
    ctx.tpcf_set_timing(False)
    rc = ctx.tpcf_sync()
    ms = e0.elapsed_time(e1) / reps
    return {"workload": (f"batching shape, {n_mock} mocks (N_d {min(len(mk.data) for mk in mks)}-"
                         f"{max(len(mk.data) for mk in mks)}), cut-sky octant shell, midpoint line of sight, "
                         "40 s x 5 mu bins: counts only, one batched call"),
            "value": n_mock / (ms * 1e-3), "unit": "mocks/s", "ms_per_call": ms,
            "gpairs_binned_per_s": info["n_binned"] / (ms * 1e-3) / 1e9,
            "pairs_binned_per_call": info["n_binned"], "candidate_pairs_per_call": info["n_candidates"],
            "pair_kernel_ms": info["paircount_ms"] / max(1, info["timed_calls"]), "status": rc}


def scale_measure(tp, ctx, dev, n_mock, reps=2):
    """The scale workload's shape on a sample of its mocks: periodic L=2000 Mpc/h, N_d=1e6 Neyman-Scott,
    R1 + R2 of N_d each, 40 s x 10 mu bins, x line of sight; all mocks and terms in one batched call."""
    import torch
    w = synth.SCALE
    mks = [w.make_mock(m) for m in range(n_mock)]
    dm = [{"data": torch.from_numpy(mk.data).to(dev),
           "randoms": torch.from_numpy(np.concatenate(mk.randoms)).to(dev),
           "offsets": [0, w.n_d, 2 * w.n_d]} for mk in mks]
    b = tp.make_binning(w.s_edges, w.n_mu, tp.TPCF_PERIODIC, w.L)
    nbin = w.n_s * w.n_mu
    out = {"dd": torch.empty((n_mock, nbin), dtype=torch.int64, device=dev),
           "dr": torch.empty((n_mock, 2, nbin), dtype=torch.int64, device=dev),
           "rr": torch.empty((n_mock, 2, nbin), dtype=torch.int64, device=dev)}
    for _ in range(2):
        ctx.tpcf_count(dm, b, mode=tp.TPCF_BATCHED, out=out)
    torch.cuda.synchronize()
    ctx.tpcf_set_timing(True)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        ctx.tpcf_count(dm, b, mode=tp.TPCF_BATCHED, out=out)
    e1.record(stream)
    torch.cuda.synchronize()
    info = ctx.tpcf_last_count_info()
    ctx.tpcf_set_timing(False)
    rc = ctx.tpcf_sync()
    ms = e0.elapsed_time(e1) / reps
    return {"workload": (f"scale shape, {n_mock} mocks: periodic L=2000 Mpc/h, N_d=1e6 Neyman-Scott (n_p=2e-6, "
                         "sigma=3), R1 + R2 of 1e6 each, 40 s x 10 mu bins, x line of sight: counts only, one "
                         "batched call"),
            "value": n_mock / (ms * 1e-3), "unit": "mocks/s", "ms_per_call": ms,
            "gpairs_binned_per_s": info["n_binned"] / (ms * 1e-3) / 1e9,
            "pairs_binned_per_call": info["n_binned"], "candidate_pairs_per_call": info["n_candidates"],
            "status": rc}


def next_rows_measure(tp, ctx, dev, reps=20):
    """Timings of the steps after the LC covariance, on the covariance workload shape: the brute-force
    sample covariance, the multipole projection, the covariance-of-covariance variances, the predicted
    chi^2 and the eigenvalue check."""
    import torch
    stream = torch.cuda.current_stream()

    def timed(fn):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    n_s, n_mu, n_mock = 40, 5, 3500
    xs = [torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in synth.synthetic_xi_variants(3, n_mock, n_s * n_mu)]
    P = torch.from_numpy(tp.tpcf_multipole_matrix(n_s, n_mu, (0, 2, 4))).to(dev)
    out = {"workload": f"{n_mock} mocks x {n_s} s x {n_mu} mu bins; multipoles l=0,2,4 (120 rows)"}
    out["sample_cov_ms"] = {name: timed(lambda pr=pr: ctx.tpcf_sample_cov(xs[2], pr))
                            for name, pr in (("fp64", tp.TPCF_FP64), ("tf32x3", tp.TPCF_TF32X3))}
    out["project_multipoles_ms"] = timed(lambda: ctx.tpcf_project(P, xs[0]))
    ys = [ctx.tpcf_project(P, x) for x in xs]
    lc = ctx.tpcf_lc_cov(*ys, 1, M_FINAL, tp.TPCF_FP64)
    out["lc_cov_multipoles_fp64_ms"] = timed(lambda: ctx.tpcf_lc_cov(*ys, 1, M_FINAL, tp.TPCF_FP64))
    big = ctx.tpcf_lc_cov(*xs, 1, M_FINAL, tp.TPCF_FP64)
    for tag, parts in (("120", lc), ("200", big)):
        out[f"covcov_var_{tag}_ms"] = timed(lambda parts=parts: ctx.tpcf_covcov_var(parts["A"], parts["B"], n_mock,
                                                                                     1, M_FINAL))
        out[f"chi2_predict_{tag}_ms"] = timed(lambda parts=parts: ctx.tpcf_chi2_predict(parts["A"], parts["B"],
                                                                                         parts["C_lc"], 1, M_FINAL))
        out[f"eigvalsh_{tag}_ms"] = timed(lambda parts=parts: ctx.tpcf_eigvalsh(parts["C_lc"]))
    w = ctx.tpcf_eigvalsh(lc["C_lc"])
    out["lc_multipole_cov_min_eigenvalue_over_max"] = float(w[0] / w[-1])
    out["chi2_2_predicted_multipoles"] = {
        "lc": float(ctx.tpcf_chi2_predict(lc["A"], lc["B"], lc["C_lc"], 1, M_FINAL)),
        "smp": float(ctx.tpcf_chi2_predict(lc["C_lc"], None, lc["C_lc"]))}
    out["status"] = ctx.tpcf_sync()
    return out


def kernel_code_hash(path):
    """sha256 prefix of a CUDA source with comments and blank space removed: it changes
    only when the code does (a profile taken before a comment edit still describes it)."""
    import hashlib, re
    src = open(path, encoding="utf-8").read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    src = re.sub(r"//[^\n]*", "", src)
    src = "\n".join(line.strip() for line in src.splitlines() if line.strip())
    return hashlib.sha256(src.encode()).hexdigest()[:16]


def measured_traffic(n_mock):
    """DRAM bytes of one pair-count launch from the committed ncu summary, if it was
    taken on the current kernel code (else None)."""
    try:
        rec = json.load(open(os.path.join(ROOT, "profiles", "paircount_traffic.json")))
        code = kernel_code_hash(os.path.join(ROOT, "paper_2205_11852_gb300", "csrc", "paircount.cu"))
    except OSError:
        return None
    if code != rec.get("kernel_code_sha256_prefix"):
        return None
    return rec["dram_bytes_per_mock"] * n_mock


def run_reference(args, rank, world):
    """--impl reference: the CPU oracle as it stands, on the host cores (rank 0 only)."""
    if rank != 0:
        return
    rates = []
    for i in range(args.warmup + args.steps):
        r = oracle_sample_rate(args.nd, target_s=max(2.0, 60.0 / max(1, args.warmup + args.steps)))
        if i >= args.warmup:
            rates.append(r)
    v = statistics.median([r["mocks_per_s"] for r in rates])
    sample = (f"brute-force counts of {rates[0]['rows']} a-rows of mock 0 against all points "
              f"(DD, DR1, DR2, RR1, RR2), {rates[0]['fraction_of_mock']:.3%} of one mock's pair tests per step")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "mocks/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * statistics.median(
                [r["seconds"] for r in rates]), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": {"workload": f"mid: {args.mocks} mocks/GPU, periodic L=1000, N_d={args.nd} Neyman-Scott, "
                                   "R1+R2 of N_d each, 40 s x 10 mu bins to 200", "global_batch": args.mocks * world},
            "cpu_baseline": {"value": v, "unit": "mocks/s", "cores": rates[0]["cores"], "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": v, "unit": "mocks/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def main():
    args = parse()
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if args.impl == "gb300" else "gloo")
    if args.impl == "reference":
        run_reference(args, rank, world)
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return

    import torch
    torch.cuda.set_device(local)
    import __graft_entry__
    __graft_entry__.build()
    import paper_2205_11852_gb300 as tp

    dev = torch.device("cuda", local)
    w = synth.MID
    n_mock, n_d = args.mocks, args.nd
    prec = {"fp64": tp.TPCF_FP64, "tf32x3": tp.TPCF_TF32X3, "bf16x3": tp.TPCF_BF16X3}[args.precision]

    if args.cov_only:
        xs = synth.synthetic_xi_variants(3, 3500, 200)
        gx = [torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in xs]
        ctx0 = tp.Context(local)
        for _ in range(2):
            ctx0.tpcf_lc_cov(*gx, 1, M_FINAL, prec, want_parts=False)
        print(json.dumps({"cov_only": True, "precision": args.precision, "status": ctx0.tpcf_sync()}))
        ctx0.close()
        return

    from paper_2205_11852_gb300 import multi
    host, layout = make_host_inputs(n_mock, n_d, multi.mock_range(rank, n_mock).start)
    pinned = torch.from_numpy(host).pin_memory()
    pos = pinned.to(dev)
    mocks = mock_views(pos, layout)
    nd_list = [sz[0] for _, sz in layout]
    nr_list = [[sz[1], sz[2]] for _, sz in layout]
    ctx = tp.Context(local)
    if args.subdiv:
        ctx.tpcf_set_cell_subdiv(args.subdiv)
    b = tp.make_binning(w.s_edges, w.n_mu, tp.TPCF_PERIODIC, w.L)
    nbin = w.n_s * w.n_mu
    outc = {"dd": torch.empty((n_mock, nbin), dtype=torch.int64, device=dev),
            "dr": torch.empty((n_mock, 2, nbin), dtype=torch.int64, device=dev),
            "rr": torch.empty((n_mock, 2, nbin), dtype=torch.int64, device=dev)}
    xi = {k: torch.empty((n_mock, nbin), dtype=torch.float64, device=dev) for k in ("a1", "a2", "b")}
    sels = {"a1": [0], "a2": [1], "b": [0, 1]}
    gather = None
    if world > 1:
        import torch.distributed as dist
        gather = {k: torch.empty((world * n_mock, nbin), dtype=torch.float64, device=dev) for k in xi}

    def step(mode=tp.TPCF_BATCHED, mocks_in=None):
        ctx.tpcf_count(mocks_in or mocks, b, mode=mode, out=outc)
        for k, sel in sels.items():
            ctx.tpcf_ls(outc["dd"], outc["dr"], outc["rr"], nd_list, nr_list, sel, out=xi[k])
        src = xi
        if gather is not None:
            src = {k: multi.gather_rows(v, world) for k, v in xi.items()}
            for k in src:
                gather[k] = src[k]
        return ctx.tpcf_lc_cov(src["a1"], src["a2"], src["b"], 1, M_FINAL, prec, want_parts=False)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    if args.count_only_batching:
        w = synth.BATCHING
        mks = [w.make_mock(m) for m in range(args.count_only_batching)]
        dm = [{"data": torch.from_numpy(mk.data).to(dev),
               "randoms": torch.from_numpy(np.concatenate(mk.randoms)).to(dev),
               "offsets": [0, len(mk.randoms[0]), len(mk.randoms[0]) + len(mk.randoms[1])]} for mk in mks]
        bb = tp.make_binning(w.s_edges, w.n_mu, tp.TPCF_OPEN, w.L, los=tp.TPCF_LOS_MIDPOINT, observer=w.observer)
        for _ in range(2):
            ctx.tpcf_count(dm, bb, mode=tp.TPCF_BATCHED)
        ctx.tpcf_sync()
        info = ctx.tpcf_last_count_info()
        print(json.dumps({"count_only": True, "workload": "batching", "mocks": len(mks),
                          "n_candidates": info["n_candidates"], "n_binned": info["n_binned"],
                          "n_exact": info["n_exact"]}))
        ctx.close()
        return
    if args.count_only:
        for _ in range(2):
            ctx.tpcf_count(mocks, b, mode=tp.TPCF_BATCHED, out=outc)
        ctx.tpcf_sync()
        info = ctx.tpcf_last_count_info()
        print(json.dumps({"count_only": True, "mocks": n_mock, "n_candidates": info["n_candidates"],
                          "n_binned": info["n_binned"], "n_exact": info["n_exact"]}))
        ctx.close()
        return

    # correctness of the timed configuration: batched == per-launch on 2 mocks
    chk_b = ctx.tpcf_count(mocks[:2], b, mode=tp.TPCF_BATCHED)
    chk_p = ctx.tpcf_count(mocks[:2], b, mode=tp.TPCF_PER_LAUNCH)
    ctx.tpcf_sync()
    same = all(torch.equal(chk_b[k], chk_p[k]) for k in ("dd", "dr", "rr"))

    for _ in range(args.warmup):
        step()
    barrier()
    ctx.tpcf_set_timing(True)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sampler = ClockSampler(local)
    barrier()
    e0.record(stream)
    for _ in range(args.steps):
        cov = step()
    e1.record(stream)
    barrier()
    clocks = sampler.stop()
    rc = ctx.tpcf_sync()
    info = ctx.tpcf_last_count_info()
    ctx.tpcf_set_timing(False)
    ms = e0.elapsed_time(e1) / args.steps
    t = torch.tensor([ms], dtype=torch.float64, device=dev)
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms = float(t.item())
    mocks_total = n_mock * world
    value = mocks_total / (ms * 1e-3)

    # pair-count kernel roofline (ALU-bound): algorithmic lane-ops / kernel time
    n_cand, n_binned = info["n_candidates"], info["n_binned"]
    k_ms = info["paircount_ms"] / max(1, info["timed_calls"])
    lane_ops = LANE_OPS_PER_CAND * n_cand + LANE_OPS_PER_BINNED * n_binned
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    peak = n_sm * LANES_PER_SM * SM_MAX_MHZ * 1e6
    achieved = lane_ops / (k_ms * 1e-3)
    f_run = clocks.get("sm_mhz") or SM_MAX_MHZ
    gpairs = n_binned / (k_ms * 1e-3) / 1e9

    # plain per-launch path on the same GPU (one launch per mock, term and subset)
    for _ in range(1):
        step(mode=tp.TPCF_PER_LAUNCH)
    barrier()
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    n_pl = max(1, min(args.steps, 3))
    p0.record(stream)
    for _ in range(n_pl):
        step(mode=tp.TPCF_PER_LAUNCH)
    p1.record(stream)
    barrier()
    ms_pl = p0.elapsed_time(p1) / n_pl
    per_launch = mocks_total / (ms_pl * 1e-3)

    # end to end through the public API: the positions are passed as pinned
    # HOST arrays (the library copies them in on the stream, TPCF_HOST_INPUT)
    # and C^LC is read back, every step
    h2d = pinned.numel() * pinned.element_size()
    d2h = nbin * nbin * 8
    res_host = torch.empty((nbin, nbin), dtype=torch.float64).pin_memory()
    mocks_host = mock_views(pinned, layout)
    # untimed warm-up steps of this path too: its staged inputs sit at new
    # device addresses, so its first call builds a launch plan and graph
    for _ in range(args.warmup):
        c = step(mocks_in=mocks_host)
        res_host.copy_(c["C_lc"], non_blocking=True)
    barrier()
    q0, q1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    q0.record(stream)
    for _ in range(args.steps):
        c = step(mocks_in=mocks_host)
        res_host.copy_(c["C_lc"], non_blocking=True)
    q1.record(stream)
    barrier()
    ms_e2e = q0.elapsed_time(q1) / args.steps
    te = torch.tensor([ms_e2e], dtype=torch.float64, device=dev)
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(te, op=dist.ReduceOp.MAX)
    e2e = mocks_total / (float(te.item()) * 1e-3)

    # covariance error of the timed path against the float64 oracle construction on the same xi
    cov_err = None
    if rank == 0:
        import oracle
        src = gather if gather is not None else xi
        ref = oracle.lc_cov(src["a1"].cpu().numpy(), src["a2"].cpu().numpy(), src["b"].cpu().numpy(), 1, M_FINAL)
        d = np.sqrt(np.abs(np.diag(ref["Ca"])))
        scale = np.outer(d, d)
        scale[scale == 0] = 1.0
        cov_err = float(np.max(np.abs(cov["C_lc"].cpu().numpy() - ref["C_lc"]) / scale))

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        r = oracle_sample_rate(n_d, args.cpu_seconds)
        cpu = {"value": r["mocks_per_s"], "unit": "mocks/s", "cores": r["cores"], "kind": "oracle",
               "sample": (f"brute-force counts of {r['rows']} a-rows of mock 0 against all points (DD, DR1, "
                          f"DR2, RR1, RR2), {r['fraction_of_mock']:.3%} of one mock's pair tests, "
                          f"{r['seconds']:.1f} s")}

    # covariance-only workload: 3500 mocks x 3 variants x 200 (s, mu) bins,
    # float64 vs split precision on the tensor cores, error against the oracle
    prec_cfg = None
    if rank == 0 and not args.no_precision_config:
        import oracle
        xs = synth.synthetic_xi_variants(3, 3500, 200)
        gx = [torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in xs]
        ref = oracle.lc_cov(*xs, 1, M_FINAL)
        d = np.sqrt(np.diag(ref["Ca"]))
        scale = np.outer(d, d)
        prec_cfg = {"workload": "3500 mocks x 3 variants x 200 (s, mu) bins, LC covariance with M=50"}
        for name, pr in (("fp64", tp.TPCF_FP64), ("tf32x3", tp.TPCF_TF32X3), ("bf16x3", tp.TPCF_BF16X3)):
            for _ in range(3):
                out = ctx.tpcf_lc_cov(*gx, 1, M_FINAL, pr, want_parts=False)
            torch.cuda.synchronize()
            c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            reps = 10
            c0.record(stream)
            for _ in range(reps):
                out = ctx.tpcf_lc_cov(*gx, 1, M_FINAL, pr, want_parts=False)
            c1.record(stream)
            torch.cuda.synchronize()
            err = float(np.max(np.abs(out["C_lc"].cpu().numpy() - ref["C_lc"]) / scale))
            prec_cfg[name] = {"ms": c0.elapsed_time(c1) / reps, "max_err_vs_fp64_oracle": err}

    # brute-force (Smp) comparison: the same mocks' shape with all M = 50 subsets
    smp = None
    if rank == 0 and world == 1 and args.smp_mocks >= 2:
        r = smp_measure(tp, ctx, dev, b, prec, args.smp_mocks, n_d)
        smp_rate = args.smp_mocks / (r["ms"] * 1e-3)
        smp = {"workload": (f"{args.smp_mocks} mocks of the mid shape with M=50 random subsets of N_d each: "
                            "DD, DR_1..50, RR_1..50 in one batched launch, LS over all 50, sample covariance"),
               "value": smp_rate, "unit": "mocks/s", "ms_per_step": r["ms"],
               "pairs_binned_per_mock": r["n_binned"] / args.smp_mocks,
               "lc_over_smp_speed": value / smp_rate,
               "lc_over_smp_binned_pairs": (r["n_binned"] / args.smp_mocks) / (n_binned / n_mock),
               "paper_cost_ratio_1p3M_over_7": (1 + 3 * 50) / 7, "status": r["status"]}

    nxt = None
    if rank == 0 and not args.no_precision_config:
        nxt = next_rows_measure(tp, ctx, dev)

    bat = None
    if rank == 0 and world == 1 and args.batching_mocks > 0:
        bat = batching_measure(tp, ctx, dev, args.batching_mocks)
    scl = None
    if rank == 0 and world == 1 and args.scale_mocks > 0:
        scl = scale_measure(tp, ctx, dev, args.scale_mocks)

    kernels_per_step = info["n_kernels"] + 3 + 4   # count + 3 LS + 4 covariance kernels
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "mocks/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": {"workload": (f"mid: {n_mock} mocks/GPU, periodic L=1000 Mpc/h, N_d={n_d} Neyman-Scott "
                                    "(n_p=1e-5, sigma=3), R1+R2 uniform of N_d each, 40 s x 10 mu bins to "
                                    "200 Mpc/h, LOS x; LS + LC covariance (M=50)"),
                       "global_batch": mocks_total, "cov_precision": args.precision,
                       "l2": "inputs larger than L2 (positions and mesh > 129 MB)"},
            "gpairs_binned_per_s": gpairs,
            "pairs_binned_per_step": n_binned * world,
            "candidate_pairs_per_step": n_cand * world,
            "per_launch": {"value": per_launch, "unit": "mocks/s", "ms_per_step": ms_pl,
                           "batched_over_per_launch": value / per_launch},
            "batched_equals_per_launch": bool(same),
            "cov_err_vs_fp64": cov_err,
            "tuned": {"cell_subdiv": info["cell_subdiv"], "cells_per_axis": info["cells_per_axis"],
                      "unit_chunk": info["unit_chunk"], "graph_replay": bool(info["graph_replay"])},
            "precision_config": prec_cfg,
            "smp_comparison": smp,
            "after_covariance": nxt,
            "batching_sample": bat,
            "scale_sample": scl,
            "roofline": {"bound": "alu", "achieved": achieved / 1e12, "peak": peak / 1e12, "unit": "Tlane-op/s",
                         "frac": achieved / peak, "traffic": measured_traffic(n_mock),
                         "traffic_note": "ncu DRAM bytes of 2 mocks scaled to the launch's mocks",
                         "frac_at_run_clock": achieved / (n_sm * LANES_PER_SM * f_run * 1e6),
                         "kernel": "paircount_kernel", "kernel_ms": k_ms,
                         "lane_ops_per_launch": lane_ops, "exact_rechecks": info["n_exact"]},
            "clocks": clocks,
            "e2e": {"value": e2e, "unit": "mocks/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": kernels_per_step * args.steps,
            "status": rc,
        }
        if cpu is not None:
            line["cpu_baseline"] = cpu
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
