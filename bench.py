"""Benchmark: contraction throughput on one GB300 (or N replicas).

Headline workload (the larger permuted plain method): C[a,b,c] =
sum_{i,j} A[i,a,j] * B[j,b,i,c] with a = b = c = 512 and i = j = 16, dense
column-major, entries uniform in [-1, 1], in the paper's double precision.
One step = one tc_execute of the planner's GETT over inputs already resident
in HBM (1.6 GB in FP64, larger than the 129 MB L2, so no flush is needed
between steps).  The same line carries the same workload in FP32 and in the
chosen precision form (split-BF16 on the tensor cores, FP32 I/O) with its
measured error, and one object per other workload of the study:

  small      abc=ai,ibc a=b=c=64 i=8 FP64: every algorithm, microseconds
  ranking    abc=iaj,jbic n=128 i=j=16 FP64: predicted vs measured, all 177
  precision  abc=ai,ibc 512^3 i=64 and ab=aij,jib 4096^2 i=j=64: every
             precision form, time, roofline, error (uniform and lognormal)
  chain      abc=ai,ij,jbc a=b=c=512 i=j=16 FP64: every order / slicing of a
             three-operand chain, predicted vs measured
  batched    4096 x abc=ai,ibc (a,b,c log-uniform [8,128], i in {4,...,32})
  serving    Poisson request stream, 10 s after 1 s of warm-up, rate sweep

    python bench.py [--gpus N] [--steps K] [--warmup W] [--quick]
                    [--impl reference]

Prints one JSON line.  ``--impl reference`` times the FP64 CPU oracle on the
host cores instead (a bounded slab of the same workload per step).  The
oracle runs only in the CPU leg below (timing it, and computing expected
values for sampled outputs); the GPU numbers come from libtc.so alone.
"""
import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "contraction GFLOP/s & %roofline, chosen vs plain FP64 form; p50/p99 latency ms"
SPEC = "abc=iaj,jbic"
N_FREE, N_CONTR = 512, 16
EXTENTS = [N_FREE, N_FREE, N_FREE, N_CONTR, N_CONTR]
WORKLOAD = "abc=iaj,jbic a=b=c=512 i=j=16 uniform[-1,1], FP64 (the paper's precision)"


def set_free_extent(n):
    """Smaller cases of the same workload (profiling captures only)."""
    global N_FREE, EXTENTS, WORKLOAD
    N_FREE = n
    EXTENTS = [n, n, n, N_CONTR, N_CONTR]
    WORKLOAD = f"abc=iaj,jbic a=b=c={n} i=j=16 uniform[-1,1], FP64"


SMS = 152
SM_MAX_MHZ = 2070.0
TORCH_IN = {"f64": "float64", "f32": "float32", "tf32": "float32", "bf16x3": "float32", "tf32x3": "float32",
            "bf16": "bfloat16", "f16": "float16", "e4m3": "float32"}
TENSOR_FORMS = ("tf32", "bf16", "f16", "bf16x3", "tf32x3", "e4m3")


def flops_of(extents):
    f = 2.0
    for e in extents:
        f *= e
    return f


def source_sha(rel):
    with open(os.path.join(ROOT, rel), "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()


def captured_traffic(key, source):
    """DRAM bytes per launch from a committed ncu capture of this kernel,
    or None when there is none or the kernel's source changed since."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            entry = json.load(f).get(key)
    except (OSError, ValueError):
        return None
    if not entry or entry.get("source_sha256") != source_sha(source):
        return None
    return entry.get("bytes_per_launch")


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "fallback": True}


def alu_peak(dtype):
    """FP64 DFMA / FP32 FFMA peak (TFLOP/s) and where it comes from: the
    committed probe summary (profiles/alu_peaks.json, measured on this
    pool's GB300s), else the unit count x max clock."""
    try:
        with open(os.path.join(ROOT, "profiles", "alu_peaks.json")) as f:
            p = json.load(f)
        return float(p[dtype]["tflops"]), f"measured ({p[dtype]['how']})"
    except (OSError, ValueError, KeyError):
        per_clk = {"f64": 2 * 2, "f32": 128 * 2}[dtype]
        return SMS * per_clk * SM_MAX_MHZ * 1e6 / 1e12, "derived: 152 SMs x units x 2 x 2070 MHz"


class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "20", "-i", str(self.index)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.thread.join(timeout=2)

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 6:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[2:6]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def aggregate_over_ranks(total_ms, steps, flops, world, dist=None, device="cpu"):
    """Whole-job throughput of `world` replicas that each ran `steps` steps of
    `flops` FLOPs: the slowest rank's time (all-reduce MAX) divides the work
    of all ranks.  Returns (max total ms, ms per step, GFLOP/s)."""
    import torch
    if dist is not None and world > 1:
        t = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    return total_ms, total_ms / steps, flops * steps * world / (total_ms / 1e3) / 1e9


def event_median(fn, reps, stream, warm=1):
    """Median seconds of fn() between CUDA events on `stream`."""
    import torch
    for _ in range(warm):
        fn()
    out = []
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        e1.synchronize()
        out.append(e0.elapsed_time(e1) * 1e-3)
    return statistics.median(out)


def sample_points(spec, extents, count, seed):
    """Random C multi-indices and their linear (Fortran) offsets."""
    from paper_1409_8608_gb300 import synth
    c_modes = synth.spec_modes(spec)[0]
    e = dict(zip(synth.index_order(spec), [int(x) for x in extents]))
    rng = np.random.default_rng(seed)
    pts = np.stack([rng.integers(0, e[m], count) for m in c_modes], axis=1)
    lin = np.zeros(count, dtype=np.int64)
    mul = 1
    for k, m in enumerate(c_modes):
        lin += pts[:, k] * mul
        mul *= e[m]
    return pts, lin


# ---------------------------------------------------------------- CPU leg
# The only code here that runs the oracle: the CPU baseline (the FP64
# oracle timed on the host cores) and the expected values of sampled
# outputs, computed one by one.  Nothing on a GPU path calls these.

def cpu_oracle_slab(spec, extents, target_s, threads, seed=0):
    """Times the FP64 oracle on a slab of the last C mode sized for about
    target_s seconds; returns (GFLOP/s, threads, slab, total slices, s)."""
    from oracle import contraction as oc
    from paper_1409_8608_gb300 import synth
    if oc.max_threads() > 0:
        threads = min(threads, oc.max_threads())
    A, B, _ = synth.uniform_operands(spec, extents, seed=seed)
    nC = synth.dense_sizes(spec, extents)[0]
    C = np.zeros(nC)
    order = synth.index_order(spec)
    e = dict(zip(order, extents))
    last = e[synth.spec_modes(spec)[0][-1]]
    per = max(1, min(threads, last, int(max(1.0, 2e9 / (flops_of(extents) / last)))))
    t0 = time.perf_counter()
    oc.contract(spec, extents, A, B, C=C, outer_range=(0, per), threads=threads)
    t1 = max(time.perf_counter() - t0, 1e-6) / per
    nsl = int(max(1, min(last, target_s / t1)))
    t0 = time.perf_counter()
    oc.contract(spec, extents, A, B, C=C, outer_range=(0, nsl), threads=threads)
    dt = time.perf_counter() - t0
    f = flops_of(extents) * nsl / last
    return f / dt / 1e9, threads, nsl, last, dt


def cpu_baseline_line(spec, extents, seconds):
    """OpenMP over all cores (the value) and one thread beside it."""
    cores = len(os.sched_getaffinity(0))
    v, used, nsl, last, dt = cpu_oracle_slab(spec, extents, seconds, cores)
    v1, _, nsl1, _, dt1 = cpu_oracle_slab(spec, extents, seconds / 2, 1)
    return {"value": v, "unit": "GFLOP/s", "cores": used, "kind": "oracle",
            "sample": f"FP64 oracle (plain nested loops, OpenMP over the outermost free index) on a slab "
                      f"of {nsl} of {last} values of the last C index ({dt:.1f} s)",
            "single_thread": {"value": v1, "unit": "GFLOP/s", "cores": 1,
                              "sample": f"slab of {nsl1} of {last} ({dt1:.1f} s)"}}


def oracle_points(spec, extents, A, B, pts, threads):
    """Expected values and |A||B| scales at the sampled points (FP64)."""
    from oracle import contraction as oc
    want = oc.contract_points(spec, extents, A, B, pts, threads=threads)
    scale = oc.contract_points(spec, extents, np.abs(A), np.abs(B), pts, threads=threads)
    return want, scale


def oracle_full(spec, extents, A, B, threads):
    from oracle import contraction as oc
    want = oc.contract(spec, extents, A, B, threads=threads)
    scale = oc.contract(spec, extents, np.abs(A), np.abs(B), threads=threads)
    return want, scale


def max_rel_err(got, want, scale):
    return float(np.max(np.abs(np.asarray(got, dtype=np.float64) - want) / scale))


def cpu_batch_baseline(rows, seconds, threads):
    """FP64 oracle over the batched problems in list order until about
    `seconds` have passed."""
    from oracle import contraction as oc
    from paper_1409_8608_gb300 import synth
    spec = "abc=ai,ibc"
    done_f, t0, n = 0.0, time.perf_counter(), 0
    for ext in rows:
        A, B, _ = synth.uniform_operands(spec, ext, seed=n)
        oc.contract(spec, ext, A, B, threads=threads)
        done_f += flops_of(ext)
        n += 1
        if time.perf_counter() - t0 > seconds:
            break
    dt = time.perf_counter() - t0
    return {"value": done_f / dt / 1e9, "unit": "GFLOP/s", "cores": threads, "kind": "oracle",
            "sample": f"the first {n} of {len(rows)} problems, FP64 ({dt:.1f} s)"}


def cpu_serving_baseline(requests, seconds, threads):
    """FP64 oracle on a slab of each sampled request, about `seconds` in all
    (requests whose single slice of the last C index exceeds 2 GFLOP are
    left out: one slice is the smallest unit the slab timing runs)."""
    from paper_1409_8608_gb300 import synth
    keep = []
    for spec, ext in requests:
        e = dict(zip(synth.index_order(spec), ext))
        if flops_of(ext) / e[synth.spec_modes(spec)[0][-1]] <= 2e9:
            keep.append((spec, ext))
    if not keep:
        return None
    per = seconds / len(keep)
    gf, tt = 0.0, 0.0
    for spec, ext in keep:
        v, _, nsl, last, dt = cpu_oracle_slab(spec, ext, per, threads)
        gf += v * dt
        tt += dt
    return {"value": gf / tt, "unit": "GFLOP/s", "cores": threads, "kind": "oracle",
            "sample": f"slabs of {len(keep)} of {len(requests)} sampled requests "
                      f"(those with at most 2 GFLOP per slice; {tt:.1f} s)"}


# ---------------------------------------------------------------- GPU legs
def measure_form(args, dtype, spec, extents, A, B, dev, stream, dist, world, tc, steps,
                 alg_name="gett", products=6, e2e=True, sample_lin=None, clocks=True):
    """Times one form (dtype + algorithm) of a workload; returns its line."""
    import torch
    tin = getattr(torch, TORCH_IN[dtype])
    tout = torch.float64 if dtype == "f64" else torch.float32
    from paper_1409_8608_gb300 import synth
    nC = synth.dense_sizes(spec, extents)[0]

    def new_plan():
        pl = tc.Plan(spec, extents, dtype=dtype)
        if dtype == "bf16x3":
            pl.set_split(products)
        pl.select({a["name"]: a["id"] for a in pl.algorithms()}[alg_name])
        return pl

    plan = new_plan()
    alg = next(a for a in plan.algorithms() if a["name"] == alg_name)
    hA = torch.from_numpy(A).to(tin).pin_memory()
    hB = torch.from_numpy(B).to(tin).pin_memory()
    dA, dB = hA.to(dev), hB.to(dev)
    dC = torch.empty(nC, dtype=tout, device=dev)
    flops = plan.flops
    # GETT: one kernel, plus the pre-pass when the plan pre-converts its
    # smaller input (the only GETT workspace); nests: phases and copies
    if alg["kernel"] == "gett":
        # with a workspace: one pre-pass (the smaller input), or two (both
        # inputs: the default of the compensated split forms, K past the
        # 256-element chunk)
        K = plan.flops // (2 * nC)
        both = dtype in ("bf16x3", "tf32x3") and K > 256
        launches_per_step = 1 + (2 if both else 1) * int(plan.workspace(alg["id"]) > 0)
    else:
        launches_per_step = alg["n_phases"] * (1 + sum(1 for lv in alg["copy_level"] if lv != -2))

    def step():
        plan.execute(dA, dB, dC, alpha=1.0, beta=0.0, stream=stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    plan.device_status()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    est = event_median(step, 2, stream, warm=0)
    # untimed load around the timed region (about 0.3 s before and after),
    # so that the clock sampler sees the clocks the timed steps run at
    pad = max(1, int(0.3 / max(1e-4, est))) if clocks else 0
    sampler = ClockSampler(torch.cuda.current_device()) if clocks else None
    if sampler:
        sampler.__enter__()
    try:
        for _ in range(pad):
            step()
        t_begin = torch.cuda.Event(enable_timing=True)
        t_end = torch.cuda.Event(enable_timing=True)
        t_begin.record(stream)
        for k in range(steps):
            ev[k][0].record(stream)
            step()
            ev[k][1].record(stream)
        t_end.record(stream)
        for _ in range(pad):
            step()
        torch.cuda.synchronize()
    finally:
        if sampler:
            sampler.__exit__(None, None, None)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    plan.device_status()
    total_ms = t_begin.elapsed_time(t_end)
    step_ms = statistics.mean(a.elapsed_time(b) for a, b in ev)
    total_ms, ms_per_step, value = aggregate_over_ranks(total_ms, steps, flops, world, dist, dev)
    samples = dC[torch.from_numpy(sample_lin).to(dev)].double().cpu().numpy() if sample_lin is not None else None

    # end to end through tc_execute_host: pinned host inputs copied in, the
    # contraction, the result copied back, every step, inside one C ABI
    # call.  Two plans on two streams take alternate steps, so one step's
    # result copy overlaps the next step's input copies and kernels.
    e2e_line = None
    if e2e:
        lanes = []
        for _ in range(2):
            lanes.append((torch.cuda.Stream(device=dev), new_plan(), torch.empty(nC, dtype=tout).pin_memory()))
        for st, pl, hc in lanes:  # first call allocates the plan's device copies
            pl.execute_host(hA, hB, hc, stream=st)
        torch.cuda.synchronize()
        e2e_steps = max(4, steps)  # the timed steps' count: the pipeline's fill and drain spread over all of them
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for st, _, _ in lanes:
            st.wait_event(e0)
        for k in range(e2e_steps):
            st, pl, hc = lanes[k % 2]
            pl.execute_host(hA, hB, hc, stream=st)
        for st, _, _ in lanes:
            done = torch.cuda.Event()
            done.record(st)
            stream.wait_event(done)
        e1.record(stream)
        torch.cuda.synchronize()
        for _, pl, _ in lanes:
            pl.device_status()
            pl.close()
        e2e_ms = e0.elapsed_time(e1) / e2e_steps
        e2e_line = {"value": flops * world / (e2e_ms / 1e3) / 1e9, "unit": "GFLOP/s",
                    "h2d_bytes_per_step": int(hA.numel() * hA.element_size() + hB.numel() * hB.element_size()),
                    "d2h_bytes_per_step": int(nC * dC.element_size()),
                    "call": "tc_execute_host (pinned host buffers; copies in, contraction, copy out)",
                    "pipelining": "2 plans on 2 streams take alternate steps"}

    peaks = measured_peaks()
    launch_s = step_ms / 1e3  # every launch of a step: the pre-pass and the GETT, or the phases
    algorithmic_bytes = int(hA.numel() * hA.element_size() + hB.numel() * hB.element_size() + nC * dC.element_size())
    nkey = extents[0]
    if dtype in TENSOR_FORMS:
        prods = products if dtype == "bf16x3" else (3 if dtype == "tf32x3" else 1)
        work = flops * prods
        peak_tf = peaks["bf16_tflops"] * (0.5 if dtype in ("tf32", "tf32x3") else 1.0)
        achieved_tf = work / launch_s / 1e12
        tkey = f"gett_tc_kernel/{dtype}/{spec}/{nkey}" + (f"/p{prods}" if dtype == "bf16x3" else "")
        roofline = {"bound": "tensor", "achieved": achieved_tf, "peak": peak_tf, "unit": "TFLOP/s",
                    "frac": achieved_tf / peak_tf,
                    "traffic": captured_traffic(tkey, "paper_1409_8608_gb300/csrc/tc_gett.cu"),
                    "algorithmic_bytes": algorithmic_bytes,
                    "kernel": "gett_tc_kernel" + (" + pack_kernel (timed together)" if launches_per_step == 2 else
                                                  " + 2 x pack_kernel (timed together)" if launches_per_step == 3 else ""),
                    "work": f"{prods} slice products x 2*prod(extents) = {work / 1e9:.1f} GFLOP per step",
                    "peak_source": "MEASURED_PEAKS bf16_tflops (burst)" +
                    (" x 0.5 (TF32 nominal ratio)" if dtype in ("tf32", "tf32x3") else "") +
                    (" (fallback)" if peaks.get("fallback") else " (measured)")}
    else:
        achieved_tf = flops / launch_s / 1e12
        peak_tf, src = alu_peak(dtype)
        kern = "tile_kernel" if alg["kernel"] in ("gett", "gemm") else "elementwise_kernel"
        tkey = f"{kern}/{dtype}/{spec}/{nkey}"
        roofline = {"bound": "alu", "achieved": achieved_tf, "peak": peak_tf, "unit": "TFLOP/s",
                    "frac": achieved_tf / peak_tf,
                    "traffic": captured_traffic(tkey, "paper_1409_8608_gb300/csrc/tc_exec.cu"),
                    "algorithmic_bytes": algorithmic_bytes, "kernel": kern,
                    "work": f"2*prod(extents) = {flops / 1e9:.1f} GFLOP per step",
                    "peak_source": ("DFMA" if dtype == "f64" else "FFMA") + " " + src}
    line = {"value": value, "unit": "GFLOP/s", "ms_per_step": ms_per_step, "dtype": dtype,
            "algorithm": alg_name, "roofline": roofline, "e2e": e2e_line,
            "gpu_launches": int(steps * launches_per_step), "steps": steps,
            "clocks": sampler.summary() if sampler else None}
    plan.close()
    return line, samples


def run_small(tc, seed=0):
    """abc=ai,ibc a=b=c=64 i=8 FP64: every algorithm, microseconds each
    (L2-resident and latency-bound, so no roofline), predicted beside it."""
    from paper_1409_8608_gb300 import ranking
    r = ranking.study("abc=ai,ibc", [64, 64, 64, 8], "f64", seed=seed, reps=20, cap=1.0)
    algs = {a["name"]: round(a["measured_s"] * 1e6, 2) for a in r["algorithms"]}
    return {"workload": "abc=ai,ibc a=b=c=64 i=8 FP64 uniform[-1,1] seed 0",
            "us_per_algorithm": algs,
            "predicted_us": {a["name"]: round(a["predicted_s"] * 1e6, 2) for a in r["algorithms"]},
            "spearman": r["spearman"], "top1_regret": r["top1_regret"],
            "top_predicted": r["top_pred"], "top_measured": r["top_meas"]}


def run_ranking(tc, n=128, dtype="f64"):
    from paper_1409_8608_gb300 import ranking
    r = ranking.study(SPEC, [n, n, n, 16, 16], dtype, seed=0, reps=3, cap=1.0)
    return {"workload": f"{SPEC} a=b=c={n} i=j=16 {dtype.upper()}", "algorithms": len(r["algorithms"]),
            "spearman": r["spearman"], "kendall": r["kendall"], "top1_regret": r["top1_regret"],
            "top_predicted": r["top_pred"], "top_measured": r["top_meas"],
            "prediction_s": r["prediction_seconds"], "measurement_s": r["measurement_seconds"]}


CHAIN_WORKLOAD = ("abc=ai,ij,jbc", [512, 512, 512, 16, 16])  # a, b, c, i, j: the headline's shape as a chain


def run_chain(tc, dev, reps=3):
    """Section 3.2's several-kernel trees: every variant of a three-operand
    chain (pair order, sliced or not) predicted from its two steps'
    micro-benchmarks and measured whole, FP64."""
    import torch
    spec, ext = CHAIN_WORKLOAD
    from paper_1409_8608_gb300 import synth
    letters = []
    for ch in spec.replace("=", "").replace(",", ""):
        if ch not in letters:
            letters.append(ch)
    e = dict(zip(letters, ext))
    d, ops = spec.split("=")[0], spec.split("=")[1].split(",")
    size = lambda modes: int(np.prod([e[m] for m in modes]))
    g = torch.Generator(device=dev).manual_seed(0)
    X, Y, Z = (torch.rand(size(o), dtype=torch.float64, device=dev, generator=g) * 2 - 1 for o in ops)
    D = torch.empty(size(d), dtype=torch.float64, device=dev)
    ch = tc.Chain(spec, ext, "f64")
    st = torch.cuda.current_stream()
    t0 = time.perf_counter()
    ch.predict(all_algorithms=False, stream=st)
    t_pred = time.perf_counter() - t0
    rows = []
    for i, v in enumerate(ch.variants()):
        ch.select(i)
        ch.execute(X, Y, Z, D, stream=st)
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a0.record(st)
            ch.execute(X, Y, Z, D, stream=st)
            a1.record(st)
            a1.synchronize()
            ts.append(a0.elapsed_time(a1) * 1e-3)
        rows.append({"first": list(v["first"]), "sliced": v["sliced"], "slices": v["slices"],
                     "workspace_mb": v["workspace_bytes"] / 2**20, "gflop": v["flops"] / 1e9,
                     "predicted_ms": v["predicted_seconds"] * 1e3, "measured_ms": statistics.median(ts) * 1e3})
    ch.device_status()
    ch.select(-1)
    sel = ch.selected()
    best = min(r["measured_ms"] for r in rows)
    ch.close()
    return {"workload": f"{spec} a=b=c=512 i=j=16 FP64 (X: ai, Y: ij, Z: jbc)", "variants": rows,
            "selected": sel, "top1_regret": rows[sel]["measured_ms"] / best - 1.0, "prediction_s": t_pred}


PRECISION_WORKLOADS = (
    ("abc=ai,ibc", [512, 512, 512, 64], "hbm"),
    ("ab=aij,jib", [4096, 4096, 64, 64], "tensor"),
)
# (label, dtype, products, compensation chunk: None = the plan's default)
PRECISION_FORMS = (
    ("bf16x3 x6 (chosen)", "bf16x3", 6, None), ("bf16x3 x3", "bf16x3", 3, None),
    ("bf16x3 x9", "bf16x3", 9, None), ("bf16x3 x6 uncompensated", "bf16x3", 6, 0),
    ("tf32x3", "tf32x3", None, None),
    ("tf32", "tf32", None, None), ("bf16", "bf16", None, None), ("f16", "f16", None, None),
    ("fp8 e4m3 (power-of-two input scales)", "e4m3", None, None),
    ("f32 (SIMT)", "f32", None, None), ("f64 (plain)", "f64", None, None),
)


def run_precision(tc, dev, stream, points=3000, reps=5):
    """Every precision form on both precision workloads: time (GPU), sampled
    outputs (errors are computed in the CPU leg)."""
    import torch
    from paper_1409_8608_gb300 import synth
    peaks = measured_peaks()
    out = []
    for spec, ext, bound in PRECISION_WORKLOADS:
        nC, nA, nB = synth.dense_sizes(spec, ext)
        flops = flops_of(ext)
        pts, lin = sample_points(spec, ext, points, seed=7)
        dlin = torch.from_numpy(lin).to(dev)
        inputs = {}
        for dist_name, gen, seed in (("uniform", synth.uniform_operands, 0),
                                     ("lognormal", synth.lognormal_slice_operands, 1)):
            A, B, _ = gen(spec, ext, seed=seed)
            inputs[dist_name] = (A, B)
        rows = []
        for label, dtype, prods, comp in PRECISION_FORMS:
            if dtype == "f64" and bound == "tensor":
                reps_f = 2
            else:
                reps_f = reps
            tin = getattr(torch, TORCH_IN[dtype])
            tout = torch.float64 if dtype == "f64" else torch.float32
            plan = tc.Plan(spec, ext, dtype=dtype)
            if prods:
                plan.set_split(prods)
            if comp is not None:
                plan.set_compensation(comp)
            plan.select(0)
            row = {"form": label, "samples": {}}
            for dist_name, (A, B) in inputs.items():
                dA = torch.from_numpy(A).to(tin).to(dev)
                dB = torch.from_numpy(B).to(tin).to(dev)
                dC = torch.empty(nC, dtype=tout, device=dev)
                run1 = lambda: plan.execute(dA, dB, dC, stream=stream)
                if dist_name == "uniform":
                    t = event_median(run1, reps_f, stream)
                    row["ms"] = t * 1e3
                    row["gflops"] = flops / t / 1e9
                    esz = 8 if dtype == "f64" else 4
                    row["hbm_frac"] = (nA + nB) * dA.element_size() / t / 1e9 / peaks["hbm_gbs"] + \
                        nC * esz / t / 1e9 / peaks["hbm_gbs"]
                    if dtype in TENSOR_FORMS:
                        # tensor work: slice products x F (3 TF32 products for 3xTF32)
                        work = flops * (prods or (3 if dtype == "tf32x3" else 1))
                        # nominal ratios to the measured BF16 peak: TF32 0.5, FP8 2
                        pk = peaks["bf16_tflops"] * (0.5 if dtype in ("tf32", "tf32x3") else
                                                     (2.0 if dtype == "e4m3" else 1.0))
                        row["tensor_frac"] = work / t / 1e12 / pk
                else:
                    run1()
                torch.cuda.synchronize()
                plan.device_status()
                row["samples"][dist_name] = dC[dlin].double().cpu().numpy()
                del dA, dB, dC
            plan.close()
            torch.cuda.empty_cache()
            rows.append(row)
        out.append({"spec": spec, "extents": ext, "bound": bound, "points": pts, "inputs": inputs, "rows": rows})
    return out


def finish_precision(prec, threads):
    """CPU leg: errors of every form against the FP64 oracle at the sampled
    points.  The oracle runs on the data as the user holds it: FP64 for the
    FP64 form, the FP32 values for every other form (so rounding the inputs
    to BF16 / FP16 / TF32 counts as error)."""
    out = []
    for w in prec:
        spec, ext = w["spec"], w["extents"]
        ref = {}
        for dist_name, (A, B) in w["inputs"].items():
            A32, B32 = A.astype(np.float32).astype(np.float64), B.astype(np.float32).astype(np.float64)
            ref[dist_name] = {"f64": oracle_points(spec, ext, A, B, w["points"], threads),
                              "f32": oracle_points(spec, ext, A32, B32, w["points"], threads)}
        rows = []
        for row in w["rows"]:
            key = "f64" if row["form"].startswith("f64") else "f32"
            errs = {d: max_rel_err(row["samples"][d], *ref[d][key]) for d in row["samples"]}
            r = {k: v for k, v in row.items() if k != "samples"}
            r["max_rel_err"] = errs
            rows.append(r)
        chosen = rows[0]
        f64 = next(r for r in rows if r["form"].startswith("f64"))
        entry = {"workload": f"{spec} {ext}, inputs uniform[-1,1] (seed 0) and lognormal per-slice scales (seed 1)",
                 "bound": w["bound"], "forms": rows,
                 "chosen": {"form": chosen["form"], "ms": chosen["ms"], "gflops": chosen["gflops"],
                            "max_rel_err": chosen["max_rel_err"],
                            "speedup_vs_f64": f64["ms"] / chosen["ms"]}}
        if w["bound"] == "hbm":
            entry["chosen"]["roofline"] = {"bound": "hbm", "frac": chosen["hbm_frac"],
                                           "unit": "of MEASURED_PEAKS hbm_gbs (compulsory bytes A+B+C)"}
        else:
            entry["chosen"]["roofline"] = {"bound": "tensor", "frac": chosen["tensor_frac"],
                                           "unit": "of MEASURED_PEAKS bf16_tflops (6 products x F)"}
        out.append(entry)
    return out


def run_batched(args):
    from paper_1409_8608_gb300 import batch_report
    out = {}
    peak = measured_peaks()["hbm_gbs"]
    for bdt, label in (("f32", "FP32 SIMT"), ("bf16x3", "split-BF16 x6 on the tensor-core GETT tiles")):
        b = batch_report.run(4096, bdt, seed=0, reps=10, hbm_gbs=peak)
        t = b["tuned"]
        out[bdt] = {
            "workload": f"4096 x abc=ai,ibc, a,b,c log-uniform [8,128], i in {{4,8,16,32}}, {label}",
            "gflops": t["gflops"], "ms": t["ms"],
            "roofline": {"bound": "hbm", "achieved": t["gbs"], "peak": peak, "unit": "GB/s",
                         "frac": t["hbm_frac"], "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)",
                         "work": f"compulsory bytes A+B+C once = {b['compulsory_gb']:.2f} GB"},
            "tiles": t["tiles"], "fixed_tiles_ms": b["fixed"]["ms"], "rule_tiles_ms": b["rule"]["ms"],
            "autotuned_vs_fixed": b["fixed"]["ms"] / t["ms"], "tuning": b["tuning"],
            "graph_ms": b["graph"]["ms"], "launch_per_problem_ms": b["launch_per_problem"]["ms"],
            "e2e": {"value": b["e2e"]["gflops"], "unit": "GFLOP/s", "ms": b["e2e"]["ms"],
                    "h2d_bytes_per_step": b["e2e"]["h2d_bytes_per_step"],
                    "d2h_bytes_per_step": b["e2e"]["d2h_bytes_per_step"]}}
    return out


def run_serving(args):
    from paper_1409_8608_gb300 import serve_report
    main = serve_report.run(seconds=args.serve_seconds, warmup=1.0, rate=2000.0, seed=0, check_samples=8)
    sweep = []
    for rate in (500.0, 1000.0, 1500.0):
        r = serve_report.run(seconds=3.0, warmup=0.5, rate=rate, seed=1)
        sweep.append({k: r[k] for k in ("rate_per_s", "offered_gflops", "served_gflops", "p50_ms", "p99_ms",
                                        "failed")})
    sweep.append({k: main[k] for k in ("rate_per_s", "offered_gflops", "served_gflops", "p50_ms", "p99_ms",
                                       "failed")})
    sustainable = max([s["rate_per_s"] for s in sweep if s["served_gflops"] >= 0.95 * s["offered_gflops"]
                       and s["failed"] == 0] or [0.0])
    main["rate_sweep"] = sweep
    main["sustainable_rate_per_s"] = sustainable
    return main


def run_gpu(args):
    import torch
    import __graft_entry__
    from paper_1409_8608_gb300 import synth, tc

    world, rank, local = dist_setup()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
        dist = None
    if rank == 0 or world == 1:
        __graft_entry__.build_library()
    if dist is not None:
        dist.barrier()
    tc.load()
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.Stream(device=dev)

    if args.only:  # one form alone (for profiler captures)
        spec, ext, form, wl = SPEC, EXTENTS, args.only, WORKLOAD
        if args.only == "bf16x3_4096":  # the chosen form of the tensor-bound precision workload
            spec, ext = PRECISION_WORKLOADS[1][:2]
            form, wl = "bf16x3", f"{spec} {ext}"
        A, B, _ = synth.uniform_operands(spec, ext, seed=rank)
        with torch.cuda.stream(stream):
            one, _ = measure_form(args, form, spec, ext, A, B, dev, stream, dist, world, tc,
                                  args.steps, e2e=False, clocks=False)
        if rank == 0:
            print(json.dumps(dict(one, metric=METRIC, config={"workload": wl, "only": args.only})), flush=True)
        return 0
    A, B, _ = synth.uniform_operands(SPEC, EXTENTS, seed=rank)
    pts, lin = sample_points(SPEC, EXTENTS, 4000, seed=11)
    with torch.cuda.stream(stream):
        head, head_samples = measure_form(args, "f64", SPEC, EXTENTS, A, B, dev, stream, dist, world, tc,
                                          args.steps, sample_lin=lin)
        forms = {}
        samples = {}
        if not args.quick:
            for dt in ("f32", "bf16x3", "tf32x3"):
                forms[dt], samples[dt] = measure_form(
                    args, dt, SPEC, EXTENTS, A, B, dev, stream, dist, world, tc, min(args.steps, 10),
                    e2e=(dt == "bf16x3"), sample_lin=lin, clocks=(dt == "bf16x3"))
    extras = {}
    if rank == 0 and world == 1 and not args.quick:
        with torch.cuda.stream(stream):
            extras["small"] = run_small(tc)
            extras["ranking"] = run_ranking(tc)
            extras["chain"] = run_chain(tc, dev)
            prec = run_precision(tc, dev, stream)
        torch.cuda.synchronize()
        extras["batched"] = run_batched(args)
        extras["serving"] = run_serving(args)
    if rank == 0:
        line = {"metric": METRIC, "value": head["value"], "unit": "GFLOP/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": head["ms_per_step"],
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic",
                "config": {"workload": WORKLOAD, "algorithm": "gett (SIMT DFMA tiles)",
                           "parallelism": f"replicas x{world}",
                           "l2": "inputs larger than L2 (no flush needed)"},
                "roofline": head["roofline"], "e2e": head["e2e"], "gpu_launches": head["gpu_launches"],
                "clocks": head["clocks"]}
        threads = len(os.sched_getaffinity(0))
        if not args.no_cpu and world == 1:
            # CPU leg: expected values of sampled outputs, then the baselines
            A32 = A.astype(np.float32).astype(np.float64)
            B32 = B.astype(np.float32).astype(np.float64)
            ref64 = oracle_points(SPEC, EXTENTS, A, B, pts, threads)
            line["max_rel_err"] = max_rel_err(head_samples, *ref64)
            if forms:
                ref32 = oracle_points(SPEC, EXTENTS, A32, B32, pts, threads)
                for dt in forms:
                    forms[dt]["max_rel_err"] = max_rel_err(samples[dt], *ref32)
            line["cpu_baseline"] = cpu_baseline_line(SPEC, EXTENTS, args.cpu_seconds)
        else:
            line["cpu_baseline"] = None
        if forms:
            forms["bf16x3"]["form"] = "chosen: split-BF16 x6 slice products on tcgen05, FP32 I/O"
            forms["bf16x3"]["speedup_vs_f64"] = forms["bf16x3"]["value"] / head["value"]
            forms["f32"]["form"] = "FP32 SIMT (FFMA tiles)"
            forms["tf32x3"]["form"] = "3xTF32: hi.hi + hi.lo + lo.hi on tcgen05 kind::tf32, FP32 I/O"
            forms["tf32x3"]["speedup_vs_f64"] = forms["tf32x3"]["value"] / head["value"]
            line["forms"] = forms
        if extras:
            if not args.no_cpu:
                extras["precision"] = finish_precision(prec, threads)
                extras["batched"]["cpu_baseline"] = cpu_batch_baseline(
                    __import__("paper_1409_8608_gb300.batch_report", fromlist=["problems"]).problems(4096, 0),
                    min(8.0, args.cpu_seconds), threads)
                extras["serving"]["cpu_baseline"] = cpu_serving_baseline(
                    extras["serving"].pop("sampled_requests", []), min(8.0, args.cpu_seconds), threads)
            line.update(extras)
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def run_reference(args):
    from oracle import contraction as oc
    from paper_1409_8608_gb300 import synth
    world, rank, _ = dist_setup()
    if rank != 0:
        return 0
    cores = len(os.sched_getaffinity(0))
    if oc.max_threads() > 0:
        cores = min(cores, oc.max_threads())
    target = max(2.0, 60.0 / max(1, args.steps + args.warmup))
    _, _, nsl, last, _ = cpu_oracle_slab(SPEC, EXTENTS, target, cores)
    A, B, _ = synth.uniform_operands(SPEC, EXTENTS, seed=0)
    C = np.zeros(synth.dense_sizes(SPEC, EXTENTS)[0])
    f_slab = flops_of(EXTENTS) * nsl / last
    for _ in range(args.warmup):
        oc.contract(SPEC, EXTENTS, A, B, C=C, outer_range=(0, nsl), threads=cores)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oc.contract(SPEC, EXTENTS, A, B, C=C, outer_range=(0, nsl), threads=cores)
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = f_slab * args.steps / total / 1e9
    sample = f"c-slab of {nsl} of {last} slices ({f_slab / 1e9:.2f} GFLOP) per step"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "GFLOP/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "form": "FP64 CPU oracle (plain nested loops, OpenMP)",
                   "l2": "n/a (host)"},
        "cpu_baseline": {"value": value, "unit": "GFLOP/s", "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "GFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--quick", action="store_true", help="the headline form only (no other forms or workloads)")
    ap.add_argument("--only", default=None, choices=["f64", "f32", "bf16x3", "tf32x3", "bf16x3_4096"],
                    help="profiling captures: one form of the headline workload alone, its line only")
    ap.add_argument("--serve-seconds", type=float, default=10.0)
    ap.add_argument("--impl", default="tc", choices=["tc", "reference"])
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--n", type=int, default=512, help="free extent a=b=c (512 = the workload)")
    args = ap.parse_args()
    if args.n != 512:
        set_free_extent(args.n)
    if args.warmup < 3 and args.impl == "tc":
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
