#!/usr/bin/env python
"""Throughput benchmark of the coupling-matrix library on GB300.

Workload (one "step"): the full spin-0 / spin-2 set -- TT, TE(=TB),
EE(=BB), EE->BB and EB -- at l_max = 3000 from three separate synthetic
windows W^TT, W^TP, W^PP (l <= 6000; power law (l+1)^-a, a ~ U(2,3), times a
Gaussian taper sigma_l ~ U(200, 800), W_0 = 4 pi fsky^2), plain FP64 path,
dense 2999 x 2999 output per spectrum.  One step = one cpl_build call.

Printed JSON line (rank 0):
  value        coupling elements/s = n_windows * n_spectra * 2999^2 / step time,
               inputs resident in HBM, CUDA events on the launching stream,
               L2 flushed between steps (outside the timed events)
  e2e          the same metric through cpl_build_host (pinned host windows in,
               pinned host matrix out; H2D and D2H copies inside the timed region)
  roofline     dominant kernel's algorithmic FLOP / its event-timed duration
               against the FP64 rate the library's FMA probe measures in the same
               run (fp64_peak; the nominal 2 FMA/clk/SM x 152 SMs x 2.07 GHz beside it)
  cpu_baseline the CPU oracle (Schulten-Gordon recursion + direct sum) on a
               bounded random sample of pairs of the same workload
  cov          cpl_cov_gaussian (TT + EE terms, l_max = 3000) with squared-mask
               spectra band-limited at L_cut = 16, 64, 512, FP64 and mixed kernels
  df32         the same workload with the contractions in double-float (CPL_DF32)
               and its error against the FP64 arm
  decouple     cpl_decouple on the binned matrices of 16 band-limited windows
               (l_max = 8000, 160 bins): event time per call for 1 and 32
               right-hand sides
  mixed        the same workload in mixed precision (tcgen05 limb GEMMs), its
               error against the FP64 arm, its own roofline and e2e
  batch        8 ragged jobs (l_max 1000 - 10000, 4 windows each) as one
               cpl_build_batch (a CUDA-graph replay) per step, mixed precision
  large_lmax   TT at l_max = 20000, FP64, with and without the operand tables
  threej_m11   (j1 j2 j3; 0 -1 1) rows for 4096 (j2, j3) pairs
Multi-GPU (torchrun): every rank builds an independent problem of the same
size (weak scaling; no data-path collective), the step time is the max over
ranks, and value counts the elements of all ranks.

--impl reference times the CPU oracle itself as the reference arm.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "M_l1l2 elements/s and 3j terms/s, lmax 3000-10000, batched vs plain FP64 on 1 GB300"
UNIT = "elements/s"
LMAX = 3000
SPEC_NAMES = ("TT", "TE", "EE", "EEBB", "EB")
# nominal FP64 pipe rate: 2 FLOP x 2 DFMA/clk/SM x 152 SMs x max clock (context only; the rooflines
# use the rate the library's FMA probe measures in the same run, FP64_PEAK below)
FP64_NOMINAL_TFLOPS = 2.0 * 2 * 152 * 2.070e9 / 1e12
FP64_PEAK = {"tflops": FP64_NOMINAL_TFLOPS, "source": "nominal (probe not run)"}
PROFILE_DIR = os.path.join(ROOT, "profiles")


def bf16_peak():
    """Measured dense BF16 tensor peak (TFLOP/s) of this machine, burst figure."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["bf16_tflops"]), "measured (MEASURED_PEAKS.json bf16_tflops, burst)"
    except (OSError, KeyError, ValueError):
        return 1900.0, "fallback 1.9 PFLOP/s"


def hbm_peak():
    """Measured HBM copy bandwidth (GB/s) of this machine."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs)"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback 6.8 TB/s"


def measure_fp64_peak(local, n_blocks=152 * 4, iters=200, steps=5):
    """The FP64 pipe's FMA rate on this GPU, measured with the library's probe
    (cpl_probe_fp64: independent FMA chains, no memory traffic): median of
    `steps` event-timed launches after three warm-ups, with the SM clock
    sampled during them.  Sets FP64_PEAK and returns the record."""
    import torch
    from paper_2602_15605_gb300 import coupling
    sink = torch.zeros(1, dtype=torch.float64, device="cuda:%d" % local)
    for _ in range(3):
        coupling.probe_fp64(n_blocks, iters, sink)
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    flop = 0.0
    for a, b in evs:
        a.record()
        flop = coupling.probe_fp64(n_blocks, iters, sink)
        b.record()
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = statistics.median(a.elapsed_time(b) for a, b in evs)
    tf = flop / (ms * 1e-3) / 1e12
    rec = {"tflops": tf, "ms_per_launch": ms, "flop_per_launch": flop, "clocks": clk,
           "nominal_tflops": FP64_NOMINAL_TFLOPS, "frac_of_nominal": tf / FP64_NOMINAL_TFLOPS,
           "kernel": "k_fp64_probe: %d blocks x 256 threads, 1024 x %d shared-memory-fed FMAs per thread" % (n_blocks, iters)}
    if clk and clk.get("sm_mhz"):
        rec["tflops_per_ghz"] = tf / (clk["sm_mhz"] / 1e3)
    FP64_PEAK["tflops"] = tf
    FP64_PEAK["source"] = ("measured in this run: FMA probe (cpl_probe_fp64) %.4f TFLOP/s at a median %s MHz; "
                           "nominal %.4f" % (tf, clk.get("sm_mhz") if clk else "?", FP64_NOMINAL_TFLOPS))
    return rec


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--cpu-seconds", type=float, default=15.0,
                    help="budget of the CPU-oracle baseline sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--lmax", type=int, default=3000,
                    help="smaller l_max for profiler captures only (the bench line uses 3000)")
    ap.add_argument("--precision", choices=["fp64", "mixed"], default="fp64",
                    help="arm of the headline value (the bench line uses fp64); the other arm is "
                         "reported in the 'mixed' / 'fp64' sub-object")
    ap.add_argument("--no-other", action="store_true", help="skip the other precision arm")
    ap.add_argument("--no-batch", action="store_true",
                    help="skip the ragged mixed-precision batch (8 jobs, l_max 1000-10000, 4 windows each)")
    ap.add_argument("--batch-steps", type=int, default=3)
    args = ap.parse_args()
    global LMAX
    LMAX = args.lmax
    return args


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", str(rank)))
    return rank, world, local


def windows_for_rank(rank):
    """W^TT, W^TP, W^PP of rank `rank`: seeds 2, 3, 4 on rank 0; independent
    seeds on the other ranks (each rank builds its own problem)."""
    from paper_2602_15605_gb300 import windows
    seeds = (2, 3, 4) if rank == 0 else tuple(1000 + 3 * rank + q for q in range(3))
    return tuple(windows.gaussian_taper(LMAX, s) for s in seeds)


def oracle_batch_extrapolation(jobs_w, seconds, seed=13):
    """The oracle on a sample of upper-triangle pairs of each ragged job (all
    its windows, all five spectra): 3j terms/s per job and the full-batch
    time extrapolated as terms / rate."""
    import numpy as np
    import oracle
    threads = os.cpu_count() or 1
    rng = np.random.default_rng(seed)

    def run(n):
        rates, wall = [], 0.0
        for lm, W in jobs_w:
            P = np.sort(rng.integers(2, lm + 1, size=(n, 2)), axis=1).astype(np.int32)
            t0 = time.perf_counter()
            oracle.coupling_pairs(P[:, 0], P[:, 1], W, W, W, 31, threads=threads)
            dt = max(time.perf_counter() - t0, 1e-6)
            m = P[:, 0].astype(np.float64)   # l3 range: m + 1 even-L and m odd-L terms
            terms = W.shape[0] * float(np.sum(4.0 * (m + 1) + 2.0 * m))
            rates.append(terms / dt)
            wall += dt
        return rates, wall

    n = 16 * threads
    _, w = run(n)                                        # also pays for thread start-up
    n = int(max(16 * threads, n * 0.25 * seconds / max(w, 1e-3)))
    _, w = run(n)
    n = int(max(16 * threads, n * seconds / max(w, 1e-3)))
    rates, wall = run(n)
    total_s = 0.0
    for (lm, W), r in zip(jobs_w, rates):
        _, t = work_counts(lm)
        total_s += W.shape[0] * sum(t.values()) / r
    return {"kind": "oracle", "cores": threads, "sample": "%d upper-triangle pairs per job, %.1f s" % (n, wall),
            "terms_per_s_by_job": rates, "extrapolated_batch_s": total_s, "label": "extrapolated"}


def ragged_seed0(rank):
    """First window seed of rank `rank`'s ragged batch (independent per rank)."""
    return 300 if rank == 0 else 300 + 1000 * rank


def max_over_ranks(x, world, device):
    """Max of a float over all ranks (the slowest rank's step time)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(world, units_per_rank, step_s):
    """Whole-job throughput: the units all ranks processed / the slowest rank's time."""
    return world * units_per_rank / step_s


def work_counts(lmax):
    """Per step: dense elements per spectrum and 3j terms per spectrum kernel
    (upper triangle l1 <= l2, parity-selected l3 counts)."""
    n = lmax - 1
    even = odd = 0
    for l1 in range(2, lmax + 1):
        npairs = lmax - l1 + 1
        # for l1 <= l2 the l3 range has 2 l1 + 1 values: l1 + 1 of even L, l1 of odd L
        even += npairs * (l1 + 1)
        odd += npairs * l1
    terms = {"TT": even, "TE": even, "EE": even, "EEBB": odd, "EB": even + odd}
    return n * n, terms


# ---------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.lines = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=5)
        mhz, maxes, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                mhz.append(float(parts[1]))
                maxes.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not mhz:
            return None
        return {"sm_mhz": statistics.median(mhz), "sm_max_mhz": max(maxes) if maxes else None,
                "samples": len(mhz), "reasons": sorted(reasons)}


# ---------------------------------------------------------------- CPU oracle
def oracle_rate(Wt, Wc, Wp, seconds, seed=7):
    """Oracle throughput in elements/s on a random sample of ordered pairs of
    the workload (uniform over the 2999 x 2999 square, all five spectra).
    Returns (elements/s, pairs, threads, wall seconds)."""
    import numpy as np
    import oracle
    threads = os.cpu_count() or 1
    rng = np.random.default_rng(seed)
    # two calibration passes (the first also pays for thread start-up, the
    # second runs about a second), then a sample sized for `seconds`
    def rate_of(n):
        cal = rng.integers(2, LMAX + 1, size=(n, 2)).astype(np.int32)
        t0 = time.perf_counter()
        oracle.coupling_pairs(cal[:, 0], cal[:, 1], Wt, Wc, Wp, 31, threads=threads)
        return n / max(time.perf_counter() - t0, 1e-6)
    r = rate_of(max(64, 8 * threads))
    r = rate_of(int(min(6_000_000, max(64, r * 1.0))))
    n = int(min(6_000_000, max(64, r * seconds)))
    P = rng.integers(2, LMAX + 1, size=(n, 2)).astype(np.int32)
    t0 = time.perf_counter()
    oracle.coupling_pairs(P[:, 0], P[:, 1], Wt, Wc, Wp, 31, threads=threads)
    wall = time.perf_counter() - t0
    return 5.0 * n / wall, n, threads, wall


def run_reference(args, rank, world):
    """The reference arm: the CPU oracle as it stands, timed on this host."""
    if rank != 0:
        return
    Wt, Wc, Wp = windows_for_rank(0)
    import numpy as np
    import oracle
    oracle.build()
    threads = os.cpu_count() or 1
    per_step = min(4.0, 120.0 / max(1, args.steps + args.warmup))
    rng = np.random.default_rng(11)
    cal = rng.integers(2, LMAX + 1, size=(max(64, 8 * threads), 2)).astype(np.int32)
    t0 = time.perf_counter()
    oracle.coupling_pairs(cal[:, 0], cal[:, 1], Wt, Wc, Wp, 31, threads=threads)
    dt = max(time.perf_counter() - t0, 1e-6)
    n = int(max(cal.shape[0], cal.shape[0] * per_step / dt))
    for _ in range(args.warmup):
        P = rng.integers(2, LMAX + 1, size=(n, 2)).astype(np.int32)
        oracle.coupling_pairs(P[:, 0], P[:, 1], Wt, Wc, Wp, 31, threads=threads)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        P = rng.integers(2, LMAX + 1, size=(n, 2)).astype(np.int32)
        oracle.coupling_pairs(P[:, 0], P[:, 1], Wt, Wc, Wp, 31, threads=threads)
    wall = time.perf_counter() - t0
    value = 5.0 * n * args.steps / wall
    sample = "%d random ordered (l1,l2) pairs per step of the l_max=3000 square, all 5 spectra" % n
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * wall / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(world),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def workload_config(world, precision="fp64"):
    return {"workload": "full spin-0/spin-2 set (TT, TE/TB, EE/BB, EE->BB, EB), %s, "
                        "l_max=%d, separate W^TT/W^TP/W^PP (l<=%d)"
                        % ("plain FP64" if precision == "fp64" else "mixed BF16 limbs", LMAX, 2 * LMAX),
            "lmax": LMAX, "lmin": 2, "n_windows": 1, "spectra": list(SPEC_NAMES), "precision": precision,
            "output": "dense 5 x %d x %d FP64 per rank" % (LMAX - 1, LMAX - 1), "parallelism": "independent problem per GPU"
            if world > 1 else "1 GPU", "l2": "flushed between steps (256 MiB write, outside the timed events)"}


# ---------------------------------------------------------------- profiles
def recorded_traffic(summary, source, key):
    """DRAM bytes per launch from a committed ncu summary under profiles/, or
    None if absent or taken on a different kernel source."""
    import hashlib
    path = os.path.join(PROFILE_DIR, summary)
    src = os.path.join(ROOT, "paper_2602_15605_gb300", "csrc", source)
    if not os.path.exists(path) or not os.path.exists(src):
        return None
    digest = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    vals = {}
    for line in open(path):
        if ":" in line:
            k, v = line.split(":", 1)
            vals[k.strip()] = v.strip()
    if vals.get("source_sha256_16") != digest:
        return None
    try:
        return float(vals[key].split()[0])
    except (KeyError, ValueError, IndexError):
        return None


# ---------------------------------------------------------------- ragged batch
def batch_arm(ctx, args, world, local, mixed_roofline):
    """The persistent ragged batch: 8 jobs, l_max in {1000, ..., 10000}, 4
    windows each (one pointer for all three roles), all five spectra, mixed
    precision, one cpl_build_batch per step (a CUDA graph replay after the
    first call).  Errors against the plain FP64 path for the jobs with
    l_max <= 4000 (the larger ones would take ~40 s in FP64)."""
    import torch
    from paper_2602_15605_gb300 import coupling, windows
    dev = lambda a: torch.as_tensor(a, dtype=torch.float64, device="cuda:%d" % local)
    jobs_w = windows.ragged_jobs(seed0=ragged_seed0(int(os.environ.get("RANK", "0"))))
    jobs = []
    n_el = 0
    terms = 0
    for lm, W in jobs_w:
        d = dev(W)
        jobs.append(dict(lmax=lm, W_tt=d, W_tp=d, W_pp=d, spectra=coupling.ALL, precision=coupling.MIXED_BF16))
        e, t = work_counts(lm)
        n_el += W.shape[0] * 5 * e
        terms += W.shape[0] * sum(t.values())
    t0 = time.perf_counter()
    outs = ctx.build_batch(jobs)            # plans, captures the graph and runs once
    torch.cuda.synchronize()
    ctx.sync()
    first_s = time.perf_counter() - t0
    for _ in range(max(args.warmup - 1, 1)):
        ctx.build_batch(jobs, outs=outs)
    torch.cuda.synchronize()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda:%d" % local)
    steps = max(1, args.batch_steps)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    before = ctx.stats()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    for q in range(steps):
        flush.fill_(q & 255)
        evs[q][0].record()
        ctx.build_batch(jobs, outs=outs)
        evs[q][1].record()
    torch.cuda.synchronize()
    clk = clocks.stop()
    ctx.sync()
    after = ctx.stats()
    per = [a.elapsed_time(b) for a, b in evs]
    ms = sum(per) / steps
    launches = sum(v["launches"] for v in after.values()) - sum(v["launches"] for v in before.values())
    ms = max_over_ranks(ms, world, "cuda:%d" % local)
    # one profiled (eager, not graph) step for the per-kernel breakdown
    ctx.profile(True)
    ctx.stats(reset=True)
    ctx.build_batch(jobs, outs=outs)
    torch.cuda.synchronize()
    st = ctx.stats(reset=True)
    ctx.profile(False)
    ctx.sync()
    err = {}
    for job, o in zip(jobs, outs):
        if job["lmax"] > 4000:
            continue
        ref = ctx.build(**dict(job, precision=coupling.FP64))
        torch.cuda.synchronize()
        for s_, nm in enumerate(SPEC_NAMES):
            a, b = o[:, s_], ref[:, s_]
            if nm in ("TT", "EE", "EEBB"):
                m = b.abs() > 1e-280
                e = float(((a - b).abs()[m] / b.abs()[m]).max())
            else:
                e = float((a - b).abs().max() / b.abs().max())
                nm = nm + "_normwise"
            err[nm] = max(err.get(nm, 0.0), e)
        del ref
    ctx.sync()
    return {"workload": "8 jobs, l_max in (1000,2000,3000,4000,6000,8000,9000,10000), 4 mask-like windows "
                        "each (one pointer for W^TT/W^TP/W^PP), all five spectra, mixed BF16 limbs (6), dense "
                        "FP64 output; one cpl_build_batch per step = one CUDA graph replay",
            "value": job_value(world, n_el, ms * 1e-3), "unit": UNIT,
            "terms_per_s": job_value(world, terms, ms * 1e-3),
            "ms_per_step": ms, "steps": steps, "first_call_s": first_s, "gpu_launches_per_step": launches / steps,
            "roofline": mixed_roofline(st),
            "kernels_profiled_step": {k: {"launches": v["launches"], "ms": v["ms"]} for k, v in st.items()},
            "max_rel_err_vs_fp64_lmax_le_4000": err, "clocks": clk,
            "spread": {"ms_median": statistics.median(per), "ms_min": min(per), "ms_max": max(per)},
            "cpu_extrapolated": (oracle_batch_extrapolation(jobs_w, args.cpu_seconds / 2)
                                 if world == 1 and not args.no_cpu_baseline else None),
            "l2": "flushed between steps (256 MiB write, outside the timed events)"}


def large_lmax_arm(ctx, local, flush, lmax=20000):
    """TT at a large l_max in plain FP64: the operand-table memory, which
    kernel ran (the tabled one builds its A blocks on every call, so a
    plain_tables_a launch marks it), the FP64 rate against the probe's peak,
    for the default choice and for the self-staging fallback."""
    import torch
    from paper_2602_15605_gb300 import coupling, windows
    W = torch.as_tensor(windows.mask_like(lmax, seed=41), dtype=torch.float64, device="cuda:%d" % local)
    out = torch.empty((1, 1, lmax - 1, lmax - 1), dtype=torch.float64, device="cuda:%d" % local)
    info = coupling.plan_info(lmax, 1, coupling.TT)
    res = {"workload": "TT, l_max = %d, one mask-like window, dense %d^2 FP64 output" % (lmax, lmax - 1),
           "table_bytes_b": info["table_bytes_b"], "table_bytes_a": info["table_bytes_a"],
           "algorithmic_flop": info["flop"]}
    prev = os.environ.get("CPL_PLAIN_TABLES")
    try:
        for name, env in (("tabled", None), ("self_staging", "0")):
            if env is None:
                os.environ.pop("CPL_PLAIN_TABLES", None)
            else:
                os.environ["CPL_PLAIN_TABLES"] = env
            t0 = time.perf_counter()
            ctx.build(lmax, W, None, None, coupling.TT, out=out)   # first call: tables for this size
            torch.cuda.synchronize()
            first_s = time.perf_counter() - t0
            free_b, total_b = torch.cuda.mem_get_info(local)
            flush.fill_(3)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            ctx.build(lmax, W, None, None, coupling.TT, out=out)
            b.record()
            torch.cuda.synchronize()
            ms = a.elapsed_time(b)
            # a profiled call for the per-kernel times
            flush.fill_(4)
            ctx.profile(True)
            ctx.stats(reset=True)
            ctx.build(lmax, W, None, None, coupling.TT, out=out)
            torch.cuda.synchronize()
            st = ctx.stats(reset=True)
            ctx.profile(False)
            ctx.sync()
            k = st.get("plain_fp64_tt", {"ms": 0.0, "flop": 0.0, "launches": 0})
            tf = k["flop"] / (k["ms"] * 1e-3) / 1e12 if k["ms"] else 0.0
            res[name] = {"ms": ms, "first_call_s": first_s, "elements_per_s": (lmax - 1) ** 2 / (ms * 1e-3),
                         "kernel": "k_plain_tab (operand tables)" if st.get("plain_tables_a", {}).get("launches")
                                   else "k_plain (self-staging)",
                         "kernel_ms": k["ms"], "fp64_tflops": tf, "frac_of_measured_fp64_peak": tf / FP64_PEAK["tflops"],
                         "kernels_profiled_call": {q: {"launches": v["launches"], "ms": v["ms"]}
                                                   for q, v in st.items() if v["launches"]},
                         "device_free_gb_after": free_b / 1e9, "device_total_gb": total_b / 1e9}
    finally:
        if prev is None:
            os.environ.pop("CPL_PLAIN_TABLES", None)
        else:
            os.environ["CPL_PLAIN_TABLES"] = prev
    del out, W
    return res


# ---------------------------------------------------------------- our arm
def run_ours(args, rank, world, local):
    import numpy as np
    import torch
    from paper_2602_15605_gb300 import build_ext, coupling, windows

    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend=backend)
    torch.cuda.set_device(local)
    if rank == 0:
        build_ext.build()
    if world > 1:
        dist.barrier()
    ctx = coupling.Context(local)
    # the mixed path's tile shapes come from the autotuner (measured on the
    # first request of each shape, outside every timed region)
    import tempfile
    tune_file = os.path.join(tempfile.mkdtemp(prefix="cpl_tune_"), "tune.jsonl")
    ctx.tune(True, tune_file)
    # the FP64 pipe's measured rate: the denominator of every FP64-bound roofline below
    fp64_peak = measure_fp64_peak(local)
    Wt, Wc, Wp = windows_for_rank(rank)
    dev = lambda a: torch.as_tensor(a, dtype=torch.float64, device="cuda:%d" % local)
    dWt, dWc, dWp = dev(Wt), dev(Wc), dev(Wp)
    n_el, terms = work_counts(LMAX)
    out = torch.empty((1, 5, LMAX - 1, LMAX - 1), dtype=torch.float64, device="cuda:%d" % local)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda:%d" % local)

    def timed_arm(prec, steps, warmup):
        """Times `steps` builds (L2 flushed between them, outside the events);
        returns (ms per step, per-kernel stats, sampled clocks, wall seconds)."""
        step = lambda: ctx.build(LMAX, dWt, dWc, dWp, coupling.ALL, out=out, precision=prec)
        first_ms = None
        for w in range(warmup):
            if w == 0:
                # the first call of this precision in the context: table build,
                # B-image cache and the autotuner's candidate runs included
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                step()
                torch.cuda.synchronize()
                first_ms = (time.perf_counter() - t0) * 1e3
            else:
                step()
        torch.cuda.synchronize()
        ctx.sync()
        ctx.profile(True)
        ctx.stats(reset=True)
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        clocks = ClockSampler(local)
        clocks.start()
        time.sleep(0.3)
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        t_wall = time.perf_counter()
        for q in range(steps):
            flush.fill_(q & 255)
            evs[q][0].record()
            step()
            evs[q][1].record()
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        t_wall = time.perf_counter() - t_wall
        clk = clocks.stop()
        per = [a.elapsed_time(b) for a, b in evs]
        ms = sum(per) / steps
        st = ctx.stats(reset=True)
        ctx.profile(False)
        ctx.sync()
        ms = max_over_ranks(ms, world, "cuda:%d" % local)
        spread = {"ms_median": statistics.median(per), "ms_min": min(per), "ms_max": max(per),
                  "first_call_ms": first_ms}
        return ms, st, clk, t_wall, spread

    def fp64_roofline(stats, clk):
        dom_name, dom = max(((k, v) for k, v in stats.items() if k.startswith("plain")), key=lambda kv: kv[1]["ms"])
        achieved = dom["flop"] / (dom["ms"] * 1e-3) / 1e12 if dom["ms"] > 0 else 0.0
        traffic = recorded_traffic("ncu_%s_full_spin_3000.txt" % dom_name, "plain_fp64.cu",
                                   "dram_bytes_per_launch_full_size") if LMAX == 3000 else None
        roof = {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK["tflops"], "unit": "TFLOP/s",
                "frac": achieved / FP64_PEAK["tflops"], "traffic": traffic, "kernel": dom_name,
                "kernel_ms_per_launch": dom["ms"] / max(dom["launches"], 1),
                "peak_source": FP64_PEAK["source"]}
        if clk and clk.get("sm_mhz"):
            roof["frac_of_nominal_at_sampled_clock"] = achieved / (2.0 * 2 * 152 * clk["sm_mhz"] * 1e6 / 1e12)
        roof["frac_of_nominal"] = achieved / FP64_NOMINAL_TFLOPS
        return roof

    def mixed_roofline(stats, traffic_summary=None):
        name, g = max(((k, v) for k, v in stats.items() if k.startswith("mixed_gemm")), key=lambda kv: kv[1]["ms"])
        traffic = (recorded_traffic(traffic_summary, "mixed_gemm.cu", "dram_bytes_per_launch")
                   if traffic_summary and LMAX == 3000 else None)
        peak, src = bf16_peak()
        issued = g["issued_flop"] / (g["ms"] * 1e-3) / 1e12 if g["ms"] > 0 else 0.0
        algo = g["flop"] / (g["ms"] * 1e-3) / 1e12 if g["ms"] > 0 else 0.0
        return {"bound": "tensor", "achieved": issued, "peak": peak, "unit": "TFLOP/s", "frac": issued / peak,
                "traffic": traffic, "kernel": name, "kernel_ms_per_launch": g["ms"] / max(g["launches"], 1),
                "algorithmic_tflops": algo, "peak_source": src,
                "achieved_counts": "BF16 limb-product FLOP issued by the tcgen05 MMAs (21 per contraction term "
                                   "at 6 limbs) / event-timed kernel duration; algorithmic_tflops counts 2 FLOP "
                                   "per window-term-contraction"}

    def mixed_error(prec=coupling.MIXED_BF16):
        """Relative error of another arm (mixed or double-float) against the plain
        FP64 arm on this workload."""
        ref = torch.empty_like(out)
        ctx.build(LMAX, dWt, dWc, dWp, coupling.ALL, out=ref)
        ctx.build(LMAX, dWt, dWc, dWp, coupling.ALL, out=out, precision=prec)
        torch.cuda.synchronize()
        ctx.sync()
        err = {}
        for s, nm in enumerate(SPEC_NAMES):
            a, b = out[0, s], ref[0, s]
            if nm in ("TT", "EE", "EEBB"):      # non-negative terms: |M| is the absolute-sum scale
                m = b.abs() > 1e-280
                err[nm] = float(((a - b).abs()[m] / b.abs()[m]).max())
            else:                               # signed terms: normwise
                err[nm + "_normwise"] = float((a - b).abs().max() / b.abs().max())
        return err

    head_prec = coupling.MIXED_BF16 if args.precision == "mixed" else coupling.FP64
    step_ms, stats, clk, t_wall, spread = timed_arm(head_prec, args.steps, args.warmup)
    launches = sum(v["launches"] for v in stats.values())
    MIXED_SUMMARY = "ncu_mixed_gemm_s6_full_spin_3000.txt"
    roofline = mixed_roofline(stats, MIXED_SUMMARY) if args.precision == "mixed" else fp64_roofline(stats, clk)
    other = None
    if not args.no_other:
        o_prec = coupling.FP64 if args.precision == "mixed" else coupling.MIXED_BF16
        o_steps = max(3, min(args.steps, 10))
        o_ms, o_stats, o_clk, _, o_spread = timed_arm(o_prec, o_steps, 2)
        other = {"value": job_value(world, 5 * n_el, o_ms * 1e-3), "unit": UNIT, "ms_per_step": o_ms, "steps": o_steps,
                 "precision": "fp64" if args.precision == "mixed" else "mixed_bf16 (6 limbs)",
                 "roofline": fp64_roofline(o_stats, o_clk) if args.precision == "mixed" else mixed_roofline(o_stats, MIXED_SUMMARY),
                 "kernels": {k: {"launches": v["launches"], "ms": v["ms"]} for k, v in o_stats.items()},
                 "clocks": o_clk, "spread": o_spread}
        other["max_rel_err_vs_fp64"] = mixed_error()
    # the plain path's contractions in double-float (CPL_DF32), same workload
    df32 = None
    if not args.no_other and args.precision == "fp64":
        d_steps = max(3, min(args.steps, 10))
        d_ms, d_stats, d_clk, _, d_spread = timed_arm(coupling.DF32, d_steps, 2)
        dk = max(((k, v) for k, v in d_stats.items() if k.startswith("plain_df") and v["launches"]),
                 key=lambda kv: kv[1]["ms"], default=None)
        df32 = {"value": job_value(world, 5 * n_el, d_ms * 1e-3), "unit": UNIT, "ms_per_step": d_ms,
                "steps": d_steps, "precision": "df32 (FP32 pairs on the FP32 pipe)",
                "kernels": {k: {"launches": v["launches"], "ms": v["ms"]} for k, v in d_stats.items()},
                "clocks": d_clk, "spread": d_spread}
        if dk is not None and dk[1]["ms"] > 0:
            eq = dk[1]["flop"] / (dk[1]["ms"] * 1e-3) / 1e12
            df32["roofline"] = {
                "bound": "alu", "kernel": dk[0], "achieved": eq, "peak": FP64_PEAK["tflops"], "unit": "TFLOP/s",
                "frac": eq / FP64_PEAK["tflops"], "traffic": None,
                "peak_source": FP64_PEAK["source"],
                "achieved_counts": "FP64-equivalent FLOP of the contractions (2 per term and contraction, as the "
                                   "FP64 kernel counts them) / event time: the fraction says how far the FP32-pair "
                                   "kernel runs past the FP64 pipe's peak; ncu: FMA-heavy pipe ~80% busy"}
        df32["max_rel_err_vs_fp64"] = mixed_error(coupling.DF32)

    # (j1 j2 j3; 0 -1 1) columns: 4096 pairs with j2, j3 in [1000, 3000]
    threej = None
    if not args.no_batch:
        rng = np.random.default_rng(31)
        j2 = rng.integers(1000, 3001, size=4096)
        j3 = rng.integers(1000, 3001, size=4096)
        stride = int(2 * np.minimum(j2, j3).max() + 1)
        tout = torch.empty((4096, stride), dtype=torch.float64, device="cuda:%d" % local)
        for _ in range(3):
            ctx.threej_m11(j2, j3, out=tout, stride=stride)
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(5)]
        ctx.sync()
        ctx.profile(True)
        ctx.stats(reset=True)
        for a, b in ev:
            flush.fill_(1)
            a.record()
            ctx.threej_m11(j2, j3, out=tout, stride=stride)
            b.record()
        torch.cuda.synchronize()
        ctx.sync()
        tj_st = ctx.stats(reset=True)
        ctx.profile(False)
        tms = statistics.median(a.elapsed_time(b) for a, b in ev)
        kst = tj_st.get("threej_m11", {"launches": 0, "ms": 0.0})
        kms = kst["ms"] / max(kst["launches"], 1)
        nsym = int(np.sum(2 * np.minimum(j2, j3) + 1))
        peak = hbm_peak()
        gbs = 4096 * stride * 8 / (kms * 1e-3) / 1e9 if kms > 0 else 0.0
        threej = {"workload": "4096 (j2, j3) pairs, j2, j3 uniform in [1000, 3000], rows padded to %d" % stride,
                  "symbols_per_s": nsym / (tms * 1e-3), "ms": tms, "kernel_ms": kms,
                  "kernels": {k: {"launches": v["launches"], "ms": v["ms"]} for k, v in tj_st.items() if v["launches"]},
                  "roofline": {"bound": "hbm", "achieved": gbs, "peak": peak[0], "unit": "GB/s",
                               "frac": gbs / peak[0], "traffic": None, "peak_source": peak[1],
                               "achieved_counts": "bytes of the written rows / event time of the row kernel "
                                                  "(k_threej_m11; ms is the whole call, with the index copies "
                                                  "and the per-row constants); the kernel is instruction-issue "
                                                  "bound (double-float products and the integer FP64 assembly), "
                                                  "not DRAM bound"}}
        del tout

    # mode decoupling (Eq. pseudo_cl): the binned matrices of 16 band-limited
    # windows at l_max = 8000 (Delta l = 50, 160 bins, all spectra)
    decouple = None
    if not args.no_batch:
        Wb, Lwb = windows.band_limited(8000, n_win=16)
        edges = np.arange(2, 8001, 50).tolist() + [8001]
        db = torch.as_tensor(Wb, dtype=torch.float64, device="cuda:%d" % local)
        Mb = ctx.build(8000, db, db, db, coupling.ALL, band_limit=Lwb, bin_edges=edges,
                       precision=coupling.MIXED_BF16)
        nb = len(edges) - 1
        decouple = {"workload": "16 windows x 5 systems (TT, TE, EE+EEBB, EE-EEBB, EB) of 160 x 160 binned "
                                "coupling matrices (band-limited l_max = 8000, Delta l = 50)"}
        rng = np.random.default_rng(77)
        for n_rhs in (1, 32):
            pcl = torch.as_tensor(rng.uniform(0.1, 1.0, size=(16, n_rhs, 5, nb)), device="cuda:%d" % local)
            dout = torch.empty_like(pcl)
            for _ in range(3):
                ctx.decouple(Mb, pcl, coupling.ALL, out=dout)
            torch.cuda.synchronize()
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(7)]
            for a, b in ev:
                flush.fill_(1)
                a.record()
                ctx.decouple(Mb, pcl, coupling.ALL, out=dout)
                b.record()
            torch.cuda.synchronize()
            ctx.sync()
            dms = statistics.median(a.elapsed_time(b) for a, b in ev)
            nsys = 16 * 5
            flop = nsys * ((nb - 1) * nb * (2 * nb - 1) / 3.0 + 2.0 * n_rhs * nb * (nb - 1))
            tf = flop / (dms * 1e-3) / 1e12
            decouple["n_rhs_%d" % n_rhs] = {
                "ms": dms, "systems_per_s": nsys / (dms * 1e-3),
                "solver": "fp32 blocked LU + fp64 iterative refinement" if 9 * n_rhs <= 2 * nb else "fp64 LU",
                "roofline": {"bound": "alu", "achieved": tf, "peak": FP64_PEAK["tflops"], "unit": "TFLOP/s",
                             "frac": tf / FP64_PEAK["tflops"], "traffic": None,
                             "peak_source": FP64_PEAK["source"],
                             "achieved_counts": "FP64-equivalent flops of the direct solve (2n^3/3 + 2 n^2 n_rhs "
                                                "per system) / median event time; the refined solver runs the "
                                                "factorisation in FP32 and the residuals at FP64 accuracy (from 8 "
                                                "right-hand sides the first on the FP64 and FP32 pipes, the later "
                                                "ones as double-float updates); one CTA per system (80 of 152 "
                                                "SMs), a chain of n dependent elimination steps"}}
            del pcl, dout
        del Mb, db

    # approximate covariance from squared-mask kernels (Sec. 4.3 band limits):
    # TT + EE Wick terms at l_max = 3000, L_cut in {16, 64, 512}, dense output
    cov = None
    if not args.no_batch:
        cov = {"workload": "Cov = Xi_TT(W~) C C' + Xi_EE(W~) E E' (2 Wick terms), l_max = 3000, dense "
                           "2999 x 2999, W~ band-limited at L_cut"}
        cv_l = 3000
        cv_ell = np.arange(cv_l + 1, dtype=np.float64)
        cv_ct = torch.as_tensor(1e3 / (cv_ell + 10.0) ** 2, device="cuda:%d" % local)
        cv_ce = torch.as_tensor(20.0 / (cv_ell + 10.0) ** 2, device="cuda:%d" % local)
        cv_out = torch.empty((cv_l - 1, cv_l - 1), dtype=torch.float64, device="cuda:%d" % local)
        for cv_cut in (16, 64, 512):
            cv_w = torch.as_tensor(windows.random_positive(cv_l, seed=90 + cv_cut, band=cv_cut),
                                   device="cuda:%d" % local)
            cv_terms = [(coupling.TT, cv_w, cv_cut, cv_ct, 2 * cv_ct), (coupling.EE, cv_w, cv_cut, cv_ce, 2 * cv_ce)]
            cv_entry = {}
            for cv_prec, cv_name in ((coupling.FP64, "fp64"), (coupling.MIXED_BF16, "mixed_bf16")):
                for _ in range(2):
                    ctx.cov_gaussian(cv_l, cv_terms, precision=cv_prec, out=cv_out)
                torch.cuda.synchronize()
                ctx.stats(reset=True)
                cv_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(5)]
                for a, b in cv_ev:
                    flush.fill_(1)
                    a.record()
                    ctx.cov_gaussian(cv_l, cv_terms, precision=cv_prec, out=cv_out)
                    b.record()
                torch.cuda.synchronize()
                ctx.sync()
                cv_ms = statistics.median(a.elapsed_time(b) for a, b in cv_ev)
                # per-kernel event times from a separate profiled pass
                ctx.stats(reset=True)
                ctx.profile(True)
                for _ in range(3):
                    flush.fill_(1)
                    ctx.cov_gaussian(cv_l, cv_terms, precision=cv_prec, out=cv_out)
                ctx.sync()
                ctx.profile(False)
                cv_st = {k: v for k, v in ctx.stats(reset=True).items() if v["launches"]}
                cv_cb = cv_st.get("cov_combine", {})
                cv_entry[cv_name] = {"ms": cv_ms, "elements_per_s": (cv_l - 1) ** 2 / (cv_ms * 1e-3),
                                     "kernels": {k: {"launches": v["launches"], "ms": v["ms"]} for k, v in cv_st.items()}}
                if cv_cb.get("ms"):
                    cv_tf = cv_cb["flop"] / (cv_cb["ms"] * 1e-3) / 1e12
                    cv_entry[cv_name]["combine_roofline"] = {
                        "bound": "alu", "achieved": cv_tf, "peak": FP64_PEAK["tflops"], "unit": "TFLOP/s",
                        "frac": cv_tf / FP64_PEAK["tflops"], "traffic": None,
                        "peak_source": FP64_PEAK["source"],
                        "achieved_counts": "2 FLOP x 3 FP64 operations per upper-triangle element and term / "
                                           "event time of the combine launches (profiled pass); the kernel is "
                                           "FP64-pipe bound, DRAM below a fifth of its peak"}
            cov["L_cut_%d" % cv_cut] = cv_entry
            del cv_w
        del cv_out, cv_ct, cv_ce

    batch = None
    if not args.no_batch:
        batch = batch_arm(ctx, args, world, local, mixed_roofline)

    # the plain path at a large l_max: TT at l_max = 20000 (one window), with the
    # operand tables (the default while they fit half of the free memory) and
    # with the self-staging kernel (CPL_PLAIN_TABLES=0, the fallback beyond that)
    large = None
    if not args.no_batch:
        large = large_lmax_arm(ctx, local, flush)

    # end to end through the public host-buffer call
    e2e = None
    if not args.no_e2e:
        # pinned host buffers: the windows in, the matrices out
        def pinned(shape):
            return torch.empty(shape, dtype=torch.float64, pin_memory=True).numpy()
        hW = []
        for W in (Wt, Wc, Wp):
            h = pinned(W.shape)
            h[...] = W
            hW.append(h)
        host_out = pinned((1, 5, LMAX - 1, LMAX - 1))
        ctx.build_host(LMAX, *hW, coupling.ALL, out=host_out, precision=head_prec)
        t0 = time.perf_counter()
        k_e2e = max(3, min(args.steps, 10))
        for _ in range(k_e2e):
            ctx.build_host(LMAX, *hW, coupling.ALL, out=host_out, precision=head_prec)
        dt = max_over_ranks((time.perf_counter() - t0) / k_e2e, world, "cuda:%d" % local)
        e2e = {"value": job_value(world, 5 * n_el, dt), "unit": UNIT, "h2d_bytes_per_step": int(3 * Wt.nbytes),
               "d2h_bytes_per_step": int(host_out.nbytes), "ms_per_step": dt * 1e3,
               "host_buffers": "pinned (page-locked) windows in and matrices out"}
        # the other precision arm end to end through the same call
        if other is not None:
            o_prec = coupling.FP64 if args.precision == "mixed" else coupling.MIXED_BF16
            ctx.build_host(LMAX, *hW, coupling.ALL, out=host_out, precision=o_prec)
            k_o = max(3, min(args.steps, 10))
            t0 = time.perf_counter()
            for _ in range(k_o):
                ctx.build_host(LMAX, *hW, coupling.ALL, out=host_out, precision=o_prec)
            dt_o = max_over_ranks((time.perf_counter() - t0) / k_o, world, "cuda:%d" % local)
            other["e2e"] = {"value": job_value(world, 5 * n_el, dt_o), "unit": UNIT,
                            "h2d_bytes_per_step": int(3 * Wt.nbytes), "d2h_bytes_per_step": int(host_out.nbytes),
                            "ms_per_step": dt_o * 1e3, "device_ms_per_step": other["ms_per_step"],
                            "exposed_transfer_ms": dt_o * 1e3 - other["ms_per_step"],
                            "host_buffers": "pinned (page-locked) windows in and matrices out"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, n, threads, wall = oracle_rate(Wt, Wc, Wp, args.cpu_seconds)
        cpu = {"value": rate, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": "%d random ordered (l1,l2) pairs of the l_max=3000 square, all 5 spectra, %.1f s"
                         % (n, wall)}

    if rank == 0:
        step_s = step_ms * 1e-3
        value = job_value(world, 5 * n_el, step_s)
        total_terms = sum(terms.values())
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "bf16-limbs/f32-acc/f64",
                "data": "synthetic", "config": workload_config(world, args.precision),
                "terms_per_s": world * total_terms / step_s,
                "terms_per_s_by_spectrum": {k: world * v / step_s for k, v in terms.items()},
                "roofline": roofline, "e2e": e2e, "cpu_baseline": cpu, "gpu_launches": int(launches),
                "kernels": {k: {"launches": v["launches"], "ms": v["ms"]} for k, v in stats.items()},
                "clocks": clk, "wall_s_timed": t_wall, "spread": spread, "fp64_peak": fp64_peak}
        if other is not None:
            line["mixed" if args.precision == "fp64" else "fp64"] = other
        if df32 is not None:
            line["df32"] = df32
        if batch is not None:
            line["batch"] = batch
        if large is not None:
            line["large_lmax"] = large
        if threej is not None:
            line["threej_m11"] = threej
        if decouple is not None:
            line["decouple"] = decouple
        if cov is not None:
            line["cov"] = cov
        try:
            line["tuner"] = [dict(lmax=e["key"][1], n_windows=e["key"][3], src=e["src"], order=e["order"],
                                  ms=e["ms"]) for e in map(json.loads, open(tune_file).read().splitlines())]
        except (OSError, ValueError, KeyError, IndexError):
            line["tuner"] = None
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        dist.destroy_process_group()


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    run_ours(args, rank, world, local)


if __name__ == "__main__":
    main()
