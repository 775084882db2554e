#!/usr/bin/env python
"""Benchmark of the LC covariance hot path on the scale workload.

Headline workload (per GPU, weak scaling): 200 mocks in a periodic box
L = 2000 Mpc/h, N_d = 1e6 Neyman-Scott points (parents 2e-6 (Mpc/h)^-3,
sigma = 3 Mpc/h) and two uniform random subsets R1, R2 of N_d points each
(the M_a = 1 pair of the linear construction), 40 linear s bins on
[0, 200) Mpc/h x 10 mu bins with the x line of sight.

One step = the whole hot path: quantisation + chaining-mesh build + pair
counts DD, DR1, DR2, RR1, RR2 of every mock (one persistent launch) + split
Landy-Szalay for R1, R2 and R1 u R2 + the LC covariance (Eqs. R1R2, LCdef)
with M = 50.  `value` is mocks/s with inputs resident in HBM; `e2e` is the
same metric through the public API with the positions copied from pinned
host memory and C^LC copied back inside every step.  The xi and covariance
errors of the timed step are measured against the float64 oracle on the
same counts and the same xi rows.

Extra keys time the mid, batching (all 1000 uneven cut-sky mocks, midpoint
line of sight) and small workloads through the same whole step, each with
its own one-launch-per-mock-per-term comparison; the covariance-only
precision workload; the brute-force (Smp, M = 50) comparison; and the steps
after the covariance.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time
from concurrent.futures import ThreadPoolExecutor

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
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    p.add_argument("--workload", default="scale", choices=sorted(synth.WORKLOADS),
                   help="headline workload (the metric is quoted on scale)")
    p.add_argument("--mocks", type=int, default=0, help="mocks per GPU (0: the workload's count)")
    p.add_argument("--nd", type=int, default=0, help="data points per mock (0: the workload's N_d)")
    p.add_argument("--precision", default="tf32x3", choices=["fp64", "tf32x3", "bf16x3"])
    p.add_argument("--extras", default="mid,batching,small",
                   help="comma list of extra workloads timed through the whole step (empty: none)")
    p.add_argument("--batching-mocks", type=int, default=synth.BATCHING.n_mock)
    p.add_argument("--no-precision-config", action="store_true",
                   help="skip the covariance-only measurement on 3500 mocks x 200 bins")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--subdiv", type=int, default=0, help="pin the mesh subdivision (0: library choice)")
    p.add_argument("--pair-kernel", default="auto", choices=["auto", "direct", "general"],
                   help="pair counter (auto: the autotuner's choice)")
    p.add_argument("--cpu-seconds", type=float, default=12.0)
    p.add_argument("--smp-mocks", type=int, default=4,
                   help="mocks of the brute-force (Smp, M=50) comparison run; 0 skips it")
    p.add_argument("--cov-only", action="store_true",
                   help="two split-precision LC covariances of 3500 mocks x 200 bins, then exit (profiler captures)")
    p.add_argument("--count-only", action="store_true",
                   help="one warm-up and one batched tpcf_count of the headline workload, then exit "
                        "(profiler captures)")
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
# workloads
# ---------------------------------------------------------------------------

def host_cores():
    return len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)


def workload_desc(w, n_mock, n_d=0):
    """One wording of a workload, shared by both arms of the benchmark."""
    if w.shell is None:
        geo = f"periodic L={w.L:g} Mpc/h"
    else:
        geo = f"cut-sky octant shell {w.shell[0]:g}-{w.shell[1]:g} Mpc/h"
    if w.n_d_range is not None and not n_d:
        pts = f"N_d Poisson-scattered in {w.n_d_range[0]}-{w.n_d_range[1]}"
    else:
        pts = f"N_d={n_d or w.n_d}"
    return (f"{w.name}: {n_mock} mocks/GPU, {geo}, {pts} Neyman-Scott (n_p={w.n_parent:g}, sigma={w.sigma:g}), "
            f"R1+R2 uniform of N_d each, {w.n_s} s x {w.n_mu} mu bins to {w.s_max:g} Mpc/h, "
            f"{'midpoint' if w.los == 'midpoint' else 'x'} line of sight; LS (R1, R2, R1uR2) + LC covariance "
            f"(M={M_FINAL:g})")


def host_inputs(w, first, n_mock, n_d=0, pinned=False):
    """Positions of mocks first..first+n_mock-1 of workload w in one float64 [n][3] array (a pinned torch
    tensor when `pinned`), drawn by a thread pool; per mock (offset, (n_d, n_r1, n_r2, ...))."""
    import torch
    sizes = [n_d or w.n_d_of(m) for m in range(first, first + n_mock)]
    layout, off = [], 0
    for nd in sizes:
        layout.append((off, (nd,) * (1 + w.M)))
        off += nd * (1 + w.M)
    if pinned:
        buf = torch.empty((off, 3), dtype=torch.float64, pin_memory=True)
        arr = buf.numpy()
    else:
        arr = np.empty((off, 3), dtype=np.float64)
        buf = torch.from_numpy(arr)

    def fill(i):
        mk = w.make_mock(first + i, n_d=n_d or None)
        o, sz = layout[i]
        for part, n in zip([mk.data] + mk.randoms, sz):
            if len(part) != n:
                raise RuntimeError(f"mock {first + i}: catalogue of {len(part)} points, expected {n}")
            arr[o:o + n] = part
            o += n

    with ThreadPoolExecutor(max(1, min(32, host_cores()))) as ex:
        list(ex.map(fill, range(n_mock)))
    return buf, layout


def mock_views(pos, layout):
    mocks = []
    for off, sz in layout:
        nd, nr = sz[0], sz[1:]
        offs = [0]
        for n in nr:
            offs.append(offs[-1] + n)
        mocks.append({"data": pos[off:off + nd], "randoms": pos[off + nd:off + nd + offs[-1]], "offsets": offs})
    return mocks


def binning_of(tp, w):
    if w.geometry == "periodic":
        return tp.make_binning(w.s_edges, w.n_mu, tp.TPCF_PERIODIC, w.L)
    return tp.make_binning(w.s_edges, w.n_mu, tp.TPCF_OPEN, w.L, origin=w.origin,
                           los=tp.TPCF_LOS_MIDPOINT if w.los == "midpoint" else tp.TPCF_LOS_X, observer=w.observer)


class Job:
    """One workload resident on the device: the whole step (counts, three split LS estimates, LC covariance)."""

    SELS = {"a1": [0], "a2": [1], "b": [0, 1]}

    def __init__(self, tp, ctx, dev, w, pos, layout, prec, world):
        import torch
        self.tp, self.ctx, self.dev, self.w, self.prec, self.world = tp, ctx, dev, w, prec, world
        self.layout = layout
        self.mocks = mock_views(pos, layout)
        self.n_mock = len(layout)
        self.nd = [sz[0] for _, sz in layout]
        self.nr = [list(sz[1:]) for _, sz in layout]
        self.b = binning_of(tp, w)
        self.nbin = w.n_s * w.n_mu
        n, M, nbin = self.n_mock, w.M, self.nbin
        self.outc = {"dd": torch.empty((n, nbin), dtype=torch.int64, device=dev),
                     "dr": torch.empty((n, M, nbin), dtype=torch.int64, device=dev),
                     "rr": torch.empty((n, M, nbin), dtype=torch.int64, device=dev)}
        self.xi = {k: torch.empty((n, nbin), dtype=torch.float64, device=dev) for k in self.SELS}
        self.rows = self.xi

    def step(self, mode=None, mocks=None):
        from paper_2205_11852_gb300 import multi
        tp, ctx = self.tp, self.ctx
        ctx.tpcf_count(mocks or self.mocks, self.b, mode=tp.TPCF_BATCHED if mode is None else mode, out=self.outc)
        for k, sel in self.SELS.items():
            ctx.tpcf_ls(self.outc["dd"], self.outc["dr"], self.outc["rr"], self.nd, self.nr, sel, out=self.xi[k])
        self.rows = {k: multi.gather_rows(v, self.world) for k, v in self.xi.items()}
        return ctx.tpcf_lc_cov(self.rows["a1"], self.rows["a2"], self.rows["b"], 1, M_FINAL, self.prec,
                               want_parts=False)

    def errors(self, cov):
        """xi of the last step against the oracle's float64 LS on the same counts, |dxi| / (1 + |xi|), and
        C^LC against the oracle's float64 construction on the same xi rows, |dC| / sqrt(C^a_ii C^a_jj)."""
        import oracle
        dd, dr, rr = (self.outc[k].cpu().numpy() for k in ("dd", "dr", "rr"))
        rel, nan_mismatch = [], 0
        for k, sel in self.SELS.items():
            got = self.xi[k].cpu().numpy()
            for m in range(self.n_mock):
                ref = oracle.ls(dd[m], dr[m], rr[m], self.nd[m], self.nr[m], sel)
                nan_r, nan_g = np.isnan(ref), np.isnan(got[m])
                nan_mismatch += int(np.count_nonzero(nan_r != nan_g))
                ok = ~(nan_r | nan_g)
                rel.append(np.abs(got[m][ok] - ref[ok]) / (1.0 + np.abs(ref[ok])))
        rel = np.concatenate(rel)
        rows = {k: v.cpu().numpy() for k, v in self.rows.items()}
        ref = oracle.lc_cov(rows["a1"], rows["a2"], rows["b"], 1, M_FINAL)
        d = np.sqrt(np.abs(np.diag(ref["Ca"])))
        scale = np.outer(d, d)
        scale[scale == 0] = 1.0
        ce = np.abs(cov["C_lc"].cpu().numpy() - ref["C_lc"]) / scale
        return ({"max": float(rel.max()), "rms": float(np.sqrt(np.mean(rel * rel))), "nan_mismatch": nan_mismatch,
                 "definition": "|xi - oracle.ls(same counts)| / (1 + |xi|) over mocks, bins and R1, R2, R1uR2"},
                {"max": float(ce.max()), "rms": float(np.sqrt(np.mean(ce * ce))),
                 "definition": "|C - oracle.lc_cov(same xi)| / sqrt(C^a_ii C^a_jj) over all elements"})


def event_time(fn, n, sync):
    """ms per call of fn over n calls, CUDA events on the current stream, synchronised on both sides."""
    import torch
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sync()
    e0.record(stream)
    out = None
    for _ in range(n):
        out = fn()
    e1.record(stream)
    sync()
    return e0.elapsed_time(e1) / n, out


def kernel_code_hash(path):
    """sha256 prefix of a CUDA source with comments and blank space removed: it changes
    only when the code does (a profile taken before a comment edit still describes it)."""
    src = open(path, encoding="utf-8").read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    src = re.sub(r"//[^\n]*", "", src)
    src = "\n".join(line.strip() for line in src.splitlines() if line.strip())
    return hashlib.sha256(src.encode()).hexdigest()[:16]


def kernel_source(pair_kernel):
    return "pairdirect.cu" if pair_kernel == 1 else "paircount.cu"


def measured_traffic(workload, n_mock, pair_kernel):
    """DRAM bytes of one pair-count launch from the committed ncu summary of this workload, if it was taken
    on the current kernel code (else None)."""
    try:
        src = kernel_source(pair_kernel)
        rec = json.load(open(os.path.join(ROOT, "profiles", "paircount_traffic.json")))[workload][src]
        code = kernel_code_hash(os.path.join(ROOT, "paper_2205_11852_gb300", "csrc", src))
    except (OSError, KeyError, ValueError):
        return None
    if code != rec.get("kernel_code_sha256_prefix"):
        return None
    return rec["dram_bytes_per_mock"] * n_mock


# ---------------------------------------------------------------------------
# CPU oracle timing (bounded sample of the same workload)
# ---------------------------------------------------------------------------

def oracle_sample_rate(w, n_d, target_s, seed_mock=0):
    """Time the oracle's brute-force counts on a row sample of one mock of workload w.

    The five terms of one mock cost 3.5 N_d^2 pair tests (DD and RR_i: N_d^2/2
    each, DR_i: N_d^2 each, with N_r,i = N_d).  A sample of k a-rows against all
    b-points runs k N_d tests per term; the rate in mocks/s is the executed
    fraction of the mock's pair tests divided by the time taken.
    """
    import oracle
    mk = w.make_mock(seed_mock, n_d=n_d or None)
    n = len(mk.data)
    geo = oracle.PERIODIC if w.geometry == "periodic" else oracle.OPEN
    ob = oracle.Binning(w.s_edges, w.n_mu, geo, w.L, origin=w.origin,
                        los=oracle.LOS_MIDPOINT if w.los == "midpoint" else oracle.LOS_X, observer=w.observer)
    qd = oracle.quantize(mk.data, geo, w.L, w.origin)
    qr = [oracle.quantize(r, geo, w.L, w.origin) for r in mk.randoms]

    def run(k):
        t0 = time.perf_counter()
        tests = 0
        a = np.ascontiguousarray(qd[:, :k])
        oracle.count_pairs(a, qd, ob)      # DD rows against all points
        tests += k * n
        for r in qr:
            oracle.count_pairs(a, r, ob)   # DR_i rows
            tests += k * r.shape[1]
            ar = np.ascontiguousarray(r[:, :k])
            oracle.count_pairs(ar, r, ob)  # RR_i rows against all points
            tests += k * r.shape[1]
        return time.perf_counter() - t0, tests

    k = max(16, n // 20000)
    dt, tests = run(k)
    # grow the sample until it takes at least ~70% of the target time (or the whole mock)
    while dt < 0.7 * target_s and k < n:
        k = int(min(n, max(2 * k, k * 0.9 * target_s / max(dt, 1e-3))))
        dt, tests = run(k)
    full = 3.5 * float(n) * float(n)
    frac = tests / full
    return {"mocks_per_s": frac / dt, "seconds": dt, "rows": k, "fraction_of_mock": frac, "cores": host_cores(),
            "pair_tests_per_s": tests / dt}


def sample_text(r):
    return (f"brute-force counts of {r['rows']} a-rows of mock 0 against all points (DD, DR1, DR2, RR1, RR2), "
            f"{r['fraction_of_mock']:.4%} of one mock's pair tests, {r['seconds']:.1f} s")


def run_reference(args, rank, world):
    """--impl reference: the CPU oracle as it stands, on the host cores (rank 0 only)."""
    if rank != 0:
        return
    w = synth.WORKLOADS[args.workload]
    n_mock = args.mocks or w.n_mock
    rates = []
    for i in range(args.warmup + args.steps):
        r = oracle_sample_rate(w, args.nd, target_s=max(2.0, 60.0 / max(1, args.warmup + args.steps)))
        if i >= args.warmup:
            rates.append(r)
    v = statistics.median([r["mocks_per_s"] for r in rates])
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "mocks/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * statistics.median([r["seconds"] for r in rates]),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": {"workload": workload_desc(w, n_mock, args.nd), "global_batch": n_mock * world},
            "cpu_baseline": {"value": v, "unit": "mocks/s", "cores": rates[0]["cores"], "kind": "oracle",
                             "sample": sample_text(rates[0]) + " per step"},
            "e2e": {"value": v, "unit": "mocks/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# extra measurements
# ---------------------------------------------------------------------------

def smp_measure(tp, ctx, dev, prec, n_mock, M=50, reps=2):
    """Brute-force (Smp) path on the mid shape: every mock against all M random
    subsets in one batched launch, LS over all subsets, sample covariance
    (Eq. bruteforce).  Returns ms per step and the pair totals."""
    import torch
    w = synth.MID
    n_d = w.n_d
    mks = [w.make_mock(m, M=M) for m in range(n_mock)]
    dm = [{"data": torch.from_numpy(mk.data).to(dev),
           "randoms": torch.from_numpy(np.concatenate(mk.randoms)).to(dev),
           "offsets": [i * n_d for i in range(M + 1)]} for mk in mks]
    b = binning_of(tp, w)
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
    ctx.tpcf_set_timing(True)
    ms, _ = event_time(step, reps, torch.cuda.synchronize)
    info = ctx.tpcf_last_count_info()
    ctx.tpcf_set_timing(False)
    return {"ms": ms, "n_binned": info["n_binned"], "n_candidates": info["n_candidates"], "status": ctx.tpcf_sync()}


def extra_workload(tp, dev, w, n_mock, prec, reps=2):
    """One more workload through the whole step on its own context: batched and one-launch-per-mock-per-term
    rates, the pair-kernel rate, counts of the two paths compared on 2 mocks, xi and covariance errors."""
    import torch
    ctx = tp.Context(dev.index)
    try:
        pos, layout = host_inputs(w, 0, n_mock)
        pos = pos.to(dev)
        job = Job(tp, ctx, dev, w, pos, layout, prec, 1)
        chk_b = ctx.tpcf_count(job.mocks[:2], job.b, mode=tp.TPCF_BATCHED)
        chk_p = ctx.tpcf_count(job.mocks[:2], job.b, mode=tp.TPCF_PER_LAUNCH)
        same = all(torch.equal(chk_b[k], chk_p[k]) for k in ("dd", "dr", "rr"))
        job.step()
        ctx.tpcf_set_timing(True)
        ms, cov = event_time(job.step, reps, torch.cuda.synchronize)
        info = ctx.tpcf_last_count_info()
        ctx.tpcf_set_timing(False)
        xi_err, cov_err = job.errors(cov)
        k_ms = info["paircount_ms"] / max(1, info["timed_calls"])
        job.step(mode=tp.TPCF_PER_LAUNCH)
        ms_pl, _ = event_time(lambda: job.step(mode=tp.TPCF_PER_LAUNCH), 1, torch.cuda.synchronize)
        rc = ctx.tpcf_sync()
        return {"workload": workload_desc(w, n_mock), "value": n_mock / (ms * 1e-3), "unit": "mocks/s",
                "ms_per_step": ms, "steps": reps, "pair_kernel_ms": k_ms,
                "gpairs_binned_per_s": info["n_binned"] / (k_ms * 1e-3) / 1e9,
                "pairs_binned_per_step": info["n_binned"], "candidate_pairs_per_step": info["n_candidates"],
                "pair_kernel": info["pair_kernel"], "cell_subdiv": info["cell_subdiv"],
                "last_wave_idle_frac": info["idle_frac"],
                "per_launch": {"value": n_mock / (ms_pl * 1e-3), "unit": "mocks/s", "ms_per_step": ms_pl,
                               "batched_over_per_launch": ms_pl / ms},
                "batched_equals_per_launch": bool(same), "xi_err": xi_err, "cov_err": cov_err, "status": rc}
    finally:
        ctx.close()
        torch.cuda.empty_cache()


def precision_measure(tp, ctx, dev):
    """Covariance-only workload: 3500 mocks x 3 variants x 200 (s, mu) bins, float64 vs split precision on the
    tensor cores, error against the oracle."""
    import torch
    import oracle
    xs = synth.synthetic_xi_variants(3, 3500, 200)
    gx = [torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in xs]
    ref = oracle.lc_cov(*xs, 1, M_FINAL)
    d = np.sqrt(np.diag(ref["Ca"]))
    scale = np.outer(d, d)
    out = {"workload": "3500 mocks x 3 variants x 200 (s, mu) bins, LC covariance with M=50"}
    for name, pr in (("fp64", tp.TPCF_FP64), ("tf32x3", tp.TPCF_TF32X3), ("bf16x3", tp.TPCF_BF16X3)):
        fn = lambda pr=pr: ctx.tpcf_lc_cov(*gx, 1, M_FINAL, pr, want_parts=False)  # noqa: E731
        for _ in range(3):
            fn()
        ms, res = event_time(fn, 10, torch.cuda.synchronize)
        e = np.abs(res["C_lc"].cpu().numpy() - ref["C_lc"]) / scale
        out[name] = {"ms": ms, "max_err_vs_fp64_oracle": float(e.max()),
                     "rms_err_vs_fp64_oracle": float(np.sqrt(np.mean(e * e)))}
    return out


def next_rows_measure(tp, ctx, dev, reps=20):
    """Timings of the steps after the LC covariance, on the covariance workload shape: the brute-force
    sample covariance, the multipole projection, the covariance-of-covariance variances, the predicted
    chi^2 and the eigenvalue check."""
    import torch

    def timed(fn):
        for _ in range(3):
            fn()
        return event_time(fn, reps, torch.cuda.synchronize)[0]

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
    from paper_2205_11852_gb300 import multi

    dev = torch.device("cuda", local)
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

    w = synth.WORKLOADS[args.workload]
    n_mock = args.mocks or w.n_mock
    t_gen = time.perf_counter()
    pinned, layout = host_inputs(w, multi.mock_range(rank, n_mock).start, n_mock, args.nd, pinned=True)
    t_gen = time.perf_counter() - t_gen
    pos = pinned.to(dev)
    ctx = tp.Context(local)
    if args.subdiv:
        ctx.tpcf_set_cell_subdiv(args.subdiv)
    ctx.tpcf_set_option(tp.TPCF_OPT_KERNEL, {"auto": tp.TPCF_KERNEL_AUTO, "direct": tp.TPCF_KERNEL_DIRECT,
                                             "general": tp.TPCF_KERNEL_GENERAL}[args.pair_kernel])
    job = Job(tp, ctx, dev, w, pos, layout, prec, world)

    if args.count_only:
        for _ in range(2):
            ctx.tpcf_count(job.mocks, job.b, mode=tp.TPCF_BATCHED, out=job.outc)
        rc = ctx.tpcf_sync()
        info = ctx.tpcf_last_count_info()
        print(json.dumps({"count_only": True, "workload": w.name, "mocks": n_mock, "status": rc,
                          "n_candidates": info["n_candidates"], "n_binned": info["n_binned"],
                          "n_exact": info["n_exact"], "pair_kernel": info["pair_kernel"],
                          "cell_subdiv": info["cell_subdiv"]}))
        ctx.close()
        return

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    def max_over_ranks(ms):
        t = torch.tensor([ms], dtype=torch.float64, device=dev)
        if world > 1:
            import torch.distributed as dist
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    # correctness of the timed configuration: batched == per-launch on 2 mocks
    chk_b = ctx.tpcf_count(job.mocks[:2], job.b, mode=tp.TPCF_BATCHED)
    chk_p = ctx.tpcf_count(job.mocks[:2], job.b, mode=tp.TPCF_PER_LAUNCH)
    ctx.tpcf_sync()
    same = all(torch.equal(chk_b[k], chk_p[k]) for k in ("dd", "dr", "rr"))
    del chk_b, chk_p

    for _ in range(args.warmup):
        job.step()
    barrier()
    ctx.tpcf_set_timing(True)
    sampler = ClockSampler(local)
    torch.cuda.nvtx.range_push("timed_step")   # lets a profiler capture exactly the timed steps
    ms, cov = event_time(job.step, args.steps, barrier)
    torch.cuda.nvtx.range_pop()
    clocks = sampler.stop()
    rc = ctx.tpcf_sync()
    info = ctx.tpcf_last_count_info()
    ctx.tpcf_set_timing(False)
    ms = max_over_ranks(ms)
    mocks_total = n_mock * world
    value = mocks_total / (ms * 1e-3)
    xi_err, cov_err = job.errors(cov) if rank == 0 else (None, None)

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
    job.step(mode=tp.TPCF_PER_LAUNCH)
    n_pl = max(1, min(args.steps, 2))
    ms_pl, _ = event_time(lambda: job.step(mode=tp.TPCF_PER_LAUNCH), n_pl, barrier)
    ms_pl = max_over_ranks(ms_pl)
    per_launch = mocks_total / (ms_pl * 1e-3)

    # end to end through the public API: the positions are passed as pinned
    # HOST arrays (TPCF_HOST_INPUT: the library copies them in, in groups whose copies overlap the counting)
    # and C^LC is read back, every step
    del pos
    job.mocks = None
    torch.cuda.empty_cache()
    h2d = pinned.numel() * pinned.element_size()
    d2h = job.nbin * job.nbin * 8
    res_host = torch.empty((job.nbin, job.nbin), dtype=torch.float64).pin_memory()
    mocks_host = mock_views(pinned, layout)

    def e2e_step():
        c = job.step(mocks=mocks_host)
        res_host.copy_(c["C_lc"], non_blocking=True)
        return c

    # one untimed call first: its staged inputs sit at new device addresses,
    # so it builds a launch plan and graph
    e2e_step()
    n_e2e = max(1, min(args.steps, 3))
    ms_e2e, _ = event_time(e2e_step, n_e2e, barrier)
    ms_e2e = max_over_ranks(ms_e2e)
    e2e = mocks_total / (ms_e2e * 1e-3)
    kernels_per_step = info["n_kernels"] + 3 + 4   # count + 3 LS + 4 covariance kernels
    tuned = {"cell_subdiv": info["cell_subdiv"], "cells_per_axis": info["cells_per_axis"],
             "unit_chunk": info["unit_chunk"], "graph_replay": bool(info["graph_replay"]),
             "pair_kernel": info["pair_kernel"], "pair_blocks": info["pair_blocks"],
             "last_wave_idle_frac": info["idle_frac"]}
    ctx.close()
    del job, pinned, mocks_host
    torch.cuda.empty_cache()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        r = oracle_sample_rate(w, args.nd, args.cpu_seconds)
        cpu = {"value": r["mocks_per_s"], "unit": "mocks/s", "cores": r["cores"], "kind": "oracle",
               "sample": sample_text(r)}

    extras = {}
    if rank == 0 and world == 1:
        for name in [x for x in args.extras.split(",") if x]:
            ew = synth.WORKLOADS[name]
            extras[name] = extra_workload(tp, dev, ew, args.batching_mocks if name == "batching" else ew.n_mock,
                                          tp.TPCF_FP64 if name == "small" else prec)

    prec_cfg = nxt = smp = None
    if rank == 0 and world == 1:
        ctx2 = tp.Context(local)
        if not args.no_precision_config:
            prec_cfg = precision_measure(tp, ctx2, dev)
            nxt = next_rows_measure(tp, ctx2, dev)
        if args.smp_mocks >= 2:
            r = smp_measure(tp, ctx2, dev, prec, args.smp_mocks)
            smp_rate = args.smp_mocks / (r["ms"] * 1e-3)
            smp = {"workload": (f"{args.smp_mocks} mocks of the mid shape with M=50 random subsets of N_d each: "
                                "DD, DR_1..50, RR_1..50 in one batched launch, LS over all 50, sample covariance"),
                   "value": smp_rate, "unit": "mocks/s", "ms_per_step": r["ms"],
                   "pairs_binned_per_mock": r["n_binned"] / args.smp_mocks,
                   "paper_cost_ratio_1p3M_over_7": (1 + 3 * 50) / 7, "status": r["status"]}
            mid = extras.get("mid")
            if mid is not None:
                smp["lc_over_smp_speed_mid"] = mid["value"] / smp_rate
                smp["lc_over_smp_binned_pairs"] = ((r["n_binned"] / args.smp_mocks) /
                                                   (mid["pairs_binned_per_step"] / synth.MID.n_mock))
        ctx2.close()

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "mocks/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": {"workload": workload_desc(w, n_mock, args.nd), "global_batch": mocks_total,
                       "cov_precision": args.precision,
                       "l2": "inputs larger than L2 (positions and mesh > 129 MB)"},
            "gpairs_binned_per_s": gpairs,
            "pairs_binned_per_step": n_binned * world,
            "candidate_pairs_per_step": n_cand * world,
            "per_launch": {"value": per_launch, "unit": "mocks/s", "ms_per_step": ms_pl, "steps": n_pl,
                           "batched_over_per_launch": value / per_launch},
            "batched_equals_per_launch": bool(same),
            "xi_err": xi_err,
            "cov_err_vs_fp64": cov_err,
            "tuned": tuned,
            "host_input_generation_s": t_gen,
            "extra_workloads": extras,
            "precision_config": prec_cfg,
            "smp_comparison": smp,
            "after_covariance": nxt,
            "roofline": {"bound": "alu", "achieved": achieved / 1e12, "peak": peak / 1e12, "unit": "Tlane-op/s",
                         "frac": achieved / peak,
                         "traffic": measured_traffic(w.name, n_mock, info["pair_kernel"]),
                         "traffic_note": "ncu DRAM bytes of a 2-mock launch of this workload scaled to the mocks",
                         "frac_at_run_clock": achieved / (n_sm * LANES_PER_SM * f_run * 1e6),
                         "kernel": "pairdirect_kernel" if info["pair_kernel"] == 1 else "paircount_kernel",
                         "kernel_ms": k_ms, "lane_ops_per_launch": lane_ops, "exact_rechecks": info["n_exact"]},
            "clocks": clocks,
            "e2e": {"value": e2e, "unit": "mocks/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "ms_per_step": ms_e2e, "steps": n_e2e},
            "gpu_launches": kernels_per_step * args.steps,
            "status": rc,
        }
        if cpu is not None:
            line["cpu_baseline"] = cpu
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
