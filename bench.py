"""Benchmark: contraction throughput on one GB300 (or N replicas).

Workload: C[a,b,c] = sum_{i,j} A[i,a,j] * B[j,b,i,c] with a = b = c = 512 and
i = j = 16 (the permuted plain workload, dense column-major, entries uniform
in [-1, 1]).  One step = one tc_execute of the selected algorithm over
inputs already resident in HBM (1.6 GB in FP64, larger than the 129 MB L2,
so no flush is needed between steps).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--dtype f64|f32]
                    [--alg gett|<name>] [--impl reference]

Prints one JSON line.  ``--impl reference`` times the FP64 CPU oracle on the
host cores instead (a bounded slab of the same workload per step).
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

SPEC = "abc=iaj,jbic"
N_FREE, N_CONTR = 512, 16
EXTENTS = [N_FREE, N_FREE, N_FREE, N_CONTR, N_CONTR]
WORKLOAD = "abc=iaj,jbic a=b=c=512 i=j=16 uniform[-1,1]"
METRIC = "contraction GFLOP/s (abc=iaj,jbic, a=b=c=512, i=j=16)"


def set_free_extent(n):
    """Smaller cases of the same workload (profiling captures only)."""
    global N_FREE, EXTENTS, WORKLOAD
    N_FREE = n
    EXTENTS = [n, n, n, N_CONTR, N_CONTR]
    WORKLOAD = f"abc=iaj,jbic a=b=c={n} i=j=16 uniform[-1,1]"
SMS = 152
SM_MAX_MHZ = 2070.0
# FP64: 2 DFMA per SM per clock (measured 1.20 TFLOP/s at 1.97 GHz); FP32: 128 FFMA.
ALU_PEAK_TFLOPS = {"f64": SMS * 2 * 2 * SM_MAX_MHZ * 1e6 / 1e12,
                   "f32": SMS * 128 * 2 * SM_MAX_MHZ * 1e6 / 1e12}


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


def cpu_oracle_sample(target_s=12.0, threads=None):
    """Times the FP64 oracle on a slab of the workload (last C mode c)."""
    from oracle import contraction as oc
    from paper_1409_8608_gb300 import synth
    cores = threads or len(os.sched_getaffinity(0))
    cores = min(cores, oc.max_threads()) if oc.max_threads() > 0 else cores
    A, B, _ = synth.uniform_operands(SPEC, EXTENTS, seed=0)
    C = np.zeros(N_FREE ** 3)
    # calibrate on one c slice, then size the slab for ~target_s
    t0 = time.perf_counter()
    oc.contract(SPEC, EXTENTS, A, B, C=C, outer_range=(0, cores), threads=cores)
    t1 = time.perf_counter() - t0
    per_slice = max(t1 / cores, 1e-5)
    nsl = int(max(cores, min(N_FREE, target_s / per_slice)))
    nsl = min(N_FREE, max(1, nsl))
    return A, B, C, cores, nsl


def run_reference(args):
    from oracle import contraction as oc
    world, rank, _ = dist_setup()
    if rank != 0:
        return 0
    target = max(2.0, 60.0 / max(1, args.steps + args.warmup))
    A, B, C, cores, nsl = cpu_oracle_sample(target_s=target)
    f_slab = flops_of([N_FREE, N_FREE, nsl, N_CONTR, N_CONTR])
    for _ in range(args.warmup):
        oc.contract(SPEC, EXTENTS, A, B, C=C, outer_range=(0, nsl), threads=cores)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oc.contract(SPEC, EXTENTS, A, B, C=C, outer_range=(0, nsl), threads=cores)
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = f_slab * args.steps / total / 1e9
    sample = f"c-slab of {nsl} of {N_FREE} slices ({f_slab / 1e9:.2f} GFLOP) per step"
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

    A, B, _ = synth.uniform_operands(SPEC, EXTENTS, seed=rank)
    res = measure_form(args, args.dtype, args.alg, A, B, dev, stream, dist, world, tc)
    plain = None
    if args.dtype != "f64" and not args.no_plain:
        plain = measure_form(args, "f64", "gett", A, B, dev, stream, dist, world, tc,
                             steps=min(args.steps, 5), e2e=False)
    if rank == 0:
        line = dict(res["line"])
        line["n_gpus"] = world
        if plain is not None:
            pl = plain["line"]
            line["plain_f64"] = {"value": pl["value"], "unit": "GFLOP/s", "algorithm": "gett",
                                 "ms_per_step": pl["ms_per_step"], "roofline": pl["roofline"],
                                 "speedup_of_chosen": line["value"] / pl["value"]}
        if world == 1 and not args.no_extras:
            from paper_1409_8608_gb300 import batch_report, serve_report
            torch.cuda.synchronize()
            line["batched"] = {}
            for bdt, label in (("bf16x3", "split-BF16 x6 (tensor-core GETT tiles)"), ("f32", "FP32 (SIMT)")):
                b = batch_report.run(4096, bdt, seed=0, reps=10, hbm_gbs=measured_peaks()["hbm_gbs"])
                line["batched"][bdt] = {
                    "workload": f"4096 x abc=ai,ibc, a,b,c log-uniform [8,128], i in {{4,8,16,32}}, {label}",
                    "gflops": b["tuned"]["gflops"], "ms": b["tuned"]["ms"],
                    "hbm_frac": b["tuned"]["hbm_frac"], "untuned_ms": b["untuned"]["ms"],
                    "graph_ms": b["graph"]["ms"], "launch_per_problem_ms": b["launch_per_problem"]["ms"]}
            sv = serve_report.run(seconds=args.serve_seconds, rate=2000.0, seed=0)
            line["serving"] = {"workload": "Poisson 2000 req/s, specs ai,ibc / iaj,jbic / aij,jib, FP64:FP32:BF16X3 = 1:2:2, 40 GB",
                               "seconds_of_arrivals": args.serve_seconds, "requests": sv["requests"],
                               "p50_ms": sv["p50_ms"], "p99_ms": sv["p99_ms"],
                               "served_gflops": sv["served_gflops"], "offered_gflops": sv["offered_gflops"],
                               "failed": sv["failed"], "admission_stalls": sv["admission_stalls"]}
        if world == 1 and not args.no_cpu:
            from oracle import contraction as oc
            A64, B64, C64, cores, nsl = cpu_oracle_sample(target_s=args.cpu_seconds)
            t0 = time.perf_counter()
            oc.contract(SPEC, EXTENTS, A64, B64, C=C64, outer_range=(0, nsl), threads=cores)
            dt = time.perf_counter() - t0
            fs = flops_of([N_FREE, N_FREE, nsl, N_CONTR, N_CONTR])
            line["cpu_baseline"] = {
                "value": fs / dt / 1e9, "unit": "GFLOP/s", "cores": cores, "kind": "oracle",
                "sample": f"FP64 oracle on a slab of c = {nsl} of {N_FREE} ({fs / 1e9:.2f} GFLOP, {dt:.1f} s)"}
        else:
            line["cpu_baseline"] = None
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def launch_estimate(plan, step, stream):
    """Seconds per step from two timed warm steps."""
    import torch
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    step()
    step()
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1) / 2e3


TORCH_IN = {"f64": "float64", "f32": "float32", "tf32": "float32", "bf16x3": "float32",
            "bf16": "bfloat16", "f16": "float16"}
TENSOR_FORMS = ("tf32", "bf16", "f16", "bf16x3")


def measure_form(args, dtype, alg_name, A, B, dev, stream, dist, world, tc, steps=None, e2e=True):
    """Times one form (dtype + algorithm) of the workload; returns its line."""
    import torch
    steps = steps or args.steps
    tin = getattr(torch, TORCH_IN[dtype])
    tout = torch.float64 if dtype == "f64" else torch.float32
    nC = N_FREE ** 3
    plan = tc.Plan(SPEC, EXTENTS, dtype=dtype)
    if dtype == "bf16x3":
        plan.set_split(args.products)
    if dtype in TENSOR_FORMS and args.bn:
        plan.set_gett_tile(args.bn)
    algs = {a["name"]: a for a in plan.algorithms()}
    alg = algs[alg_name]
    plan.select(alg["id"])
    hA = torch.from_numpy(A).to(tin).pin_memory()
    hB = torch.from_numpy(B).to(tin).pin_memory()
    hC = torch.empty(nC, dtype=tout).pin_memory()
    dA = hA.to(dev)
    dB = hB.to(dev)
    dC = torch.empty(nC, dtype=tout, device=dev)
    flops = plan.flops
    # GETT: one kernel, plus the pre-pass when the plan pre-converts its
    # smaller input (the only GETT workspace)
    launches_per_step = 1 + (plan.workspace(alg["id"]) > 0) if alg["kernel"] == "gett" else alg["n_phases"] + sum(
        1 for lv in alg["copy_level"] if lv != -2) * alg["n_phases"]

    def step():
        plan.execute(dA, dB, dC, alpha=1.0, beta=0.0, stream=stream)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
    args_steps = steps
    torch.cuda.synchronize()
    plan.device_status()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args_steps)]
    # untimed load around the timed region (about 0.3 s before and after),
    # so that the clock sampler sees the clocks the timed steps run at
    pad = max(1, int(0.3 / max(1e-4, launch_estimate(plan, step, stream))))
    with ClockSampler(torch.cuda.current_device()) as clk:
        for _ in range(pad):
            step()
        t_begin = torch.cuda.Event(enable_timing=True)
        t_end = torch.cuda.Event(enable_timing=True)
        t_begin.record(stream)
        for k in range(args_steps):
            ev[k][0].record(stream)
            step()
            ev[k][1].record(stream)
        t_end.record(stream)
        for _ in range(pad):
            step()
        torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    plan.device_status()
    total_ms = t_begin.elapsed_time(t_end)
    per_launch_ms = statistics.mean(a.elapsed_time(b) for a, b in ev) / max(1, launches_per_step)
    total_ms, ms_per_step, value = aggregate_over_ranks(total_ms, args_steps, flops, world, dist, dev)

    # end to end through the public call: pinned host inputs -> device,
    # execute, result back to pinned host memory, every step.  Two streams
    # with their own device buffers take alternate steps, so one step's
    # result copy overlaps the next step's input copies and execute (each
    # step still copies all of its inputs and its whole result).
    e2e_steps = max(4, min(args_steps, 8)) if e2e else 0
    lanes = [(stream, dA, dB, dC, hC, plan)]
    if e2e_steps:
        # the second stream gets its own plan (a plan's workspace serves one
        # stream at a time), set up and run once outside the timed region
        plan2 = tc.Plan(SPEC, EXTENTS, dtype=dtype)
        if dtype == "bf16x3":
            plan2.set_split(args.products)
        if dtype in TENSOR_FORMS and args.bn:
            plan2.set_gett_tile(args.bn)
        plan2.select(alg["id"])
        lanes.append((torch.cuda.Stream(device=dev), torch.empty_like(dA), torch.empty_like(dB),
                      torch.empty_like(dC), torch.empty_like(hC).pin_memory(), plan2))
        with torch.cuda.stream(lanes[1][0]):
            plan2.execute(dA, dB, lanes[1][3], alpha=1.0, beta=0.0, stream=lanes[1][0])
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for st, *_ in lanes[1:]:
        st.wait_event(e0)
    for k in range(e2e_steps):
        st, a, b, c, hc, pl = lanes[k % len(lanes)]
        with torch.cuda.stream(st):
            a.copy_(hA, non_blocking=True)
            b.copy_(hB, non_blocking=True)
            pl.execute(a, b, c, alpha=1.0, beta=0.0, stream=st)
            hc.copy_(c, non_blocking=True)
    for st, *_ in lanes[1:]:
        done = torch.cuda.Event()
        done.record(st)
        stream.wait_event(done)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_value = None
    if e2e_steps:
        e2e_ms = e0.elapsed_time(e1) / e2e_steps
        e2e_value = flops * world / (e2e_ms / 1e3) / 1e9
        lanes[1][5].close()

    peaks = measured_peaks()
    launch_s = per_launch_ms * launches_per_step / 1e3
    if dtype in TENSOR_FORMS:
        products = args.products if dtype == "bf16x3" else 1
        work = flops * products
        peak_tf = peaks["bf16_tflops"] * (0.5 if dtype == "tf32" else 1.0)
        achieved_tf = work / launch_s / 1e12
        tkey = f"gett_tc_kernel/{dtype}/{SPEC}/{N_FREE}" + (f"/p{products}" if dtype == "bf16x3" else "")
        roofline = {"bound": "tensor", "achieved": achieved_tf, "peak": peak_tf, "unit": "TFLOP/s",
                    "frac": achieved_tf / peak_tf,
                    "traffic": captured_traffic(tkey, "paper_1409_8608_gb300/csrc/tc_gett.cu"),
                    "algorithmic_bytes": int(hA.numel() * hA.element_size() + hB.numel() * hB.element_size()
                                             + hC.numel() * hC.element_size()),
                    # with the pre-pass the events time both kernels of the step
                    "kernel": "gett_tc_kernel" + (" + pack_kernel (timed together)" if launches_per_step == 2 else ""),
                    "work": f"{products} slice products x 2*prod(extents) = {work / 1e9:.1f} GFLOP per launch",
                    "peak_source": "MEASURED_PEAKS bf16_tflops (burst)" + (" x 0.5 (TF32 nominal ratio)" if dtype == "tf32" else "")
                    + (" (fallback)" if peaks.get("fallback") else " (measured)")}
    else:
        achieved_tf = flops / launch_s / 1e12
        peak_tf = ALU_PEAK_TFLOPS[dtype]
        tkey = f"tile_kernel/{dtype}/{SPEC}/{N_FREE}"
        roofline = {"bound": "alu", "achieved": achieved_tf, "peak": peak_tf, "unit": "TFLOP/s",
                    "frac": achieved_tf / peak_tf,
                    "traffic": captured_traffic(tkey, "paper_1409_8608_gb300/csrc/tc_exec.cu"),
                    "kernel": "tile_kernel" if alg["kernel"] in ("gett", "gemm") else "elementwise_kernel",
                    "peak_source": f"derived: 152 SMs x {'2 DFMA' if dtype == 'f64' else '128 FFMA'}/clk x 2 x 2070 MHz"}
    line = {
        "metric": METRIC, "value": value, "unit": "GFLOP/s", "n_gpus": world,
        "steps": args_steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": dtype, "data": "synthetic",
        "config": {"workload": WORKLOAD, "algorithm": alg["name"],
                   "form": ("split-BF16 x%d products, FP32 I/O" % args.products) if dtype == "bf16x3" else f"{dtype}",
                   "parallelism": f"replicas x{world}",
                   "l2": "inputs larger than L2 (no flush needed)"},
        "roofline": roofline,
        "e2e": None if e2e_value is None else {
            "value": e2e_value, "unit": "GFLOP/s",
            "h2d_bytes_per_step": int(hA.numel() * hA.element_size() + hB.numel() * hB.element_size()),
            "d2h_bytes_per_step": int(hC.numel() * hC.element_size()),
            "pipelining": "2 streams, alternate steps, own device buffers"},
        "gpu_launches": int(args_steps * launches_per_step),
        "clocks": clk.summary(),
    }
    plan.close()
    return {"line": line}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--dtype", default="bf16x3", choices=["f64", "f32", "tf32", "bf16", "f16", "bf16x3"])
    ap.add_argument("--products", type=int, default=6)
    ap.add_argument("--bn", type=int, default=0, help="tensor-core GETT tile width (0: auto)")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the batched and serving measurements")
    ap.add_argument("--serve-seconds", type=float, default=1.0)
    ap.add_argument("--alg", default="gett")
    ap.add_argument("--impl", default="tc", choices=["tc", "reference"])
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
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
