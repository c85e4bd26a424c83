"""Ranking study: predicted vs measured time for every algorithm of one
contraction (the experiments of Sections 3-4, on the device).

    python -m paper_1409_8608_gb300.ranking --spec abc=iaj,jbic \\
        --extents 256,256,256,16,16 --dtype f64 [--json out.json] [--classes]
        [--execute name,name,...]

Reports per algorithm the predicted and the measured seconds, and over all
of them Spearman's rho and Kendall's tau of the two rankings, the top-1
regret (measured time of the top-ranked algorithm over the measured best,
minus one) and the time spent predicting against the time spent measuring
(the efficiency study of Section 4).  Measurement: CUDA events around one
tc_execute, after an L2 flush, median of `reps` runs; an algorithm whose
first run exceeds `cap` seconds is measured once and marked capped (the
paper stops slow algorithms the same way).
"""
import argparse
import json
import time

import numpy as np

from . import synth, tc


def ranks(x):
    """Average ranks (1 = smallest), ties share their mean rank."""
    x = np.asarray(x, dtype=np.float64)
    order = np.argsort(x, kind="stable")
    r = np.empty(len(x))
    r[order] = np.arange(1, len(x) + 1)
    for v in np.unique(x):
        idx = np.flatnonzero(x == v)
        if len(idx) > 1:
            r[idx] = r[idx].mean()
    return r


def spearman(a, b):
    ra, rb = ranks(a), ranks(b)
    ra -= ra.mean()
    rb -= rb.mean()
    den = np.sqrt((ra * ra).sum() * (rb * rb).sum())
    return float((ra * rb).sum() / den) if den > 0 else 0.0


def kendall(a, b):
    a, b = np.asarray(a), np.asarray(b)
    n, s = len(a), 0
    for i in range(n):
        s += int(np.sum(np.sign(a[i] - a[i + 1:]) * np.sign(b[i] - b[i + 1:])))
    pairs = n * (n - 1) / 2
    return float(s / pairs) if pairs else 0.0


def measure(plan, ids, dA, dB, dC, flush, reps=5, cap=2.0):
    import torch
    out, capped = [], []
    stream = torch.cuda.current_stream()
    for aid in ids:
        plan.select(aid)
        plan.execute(dA, dB, dC, stream=stream)  # warm-up (allocates copy workspace)
        torch.cuda.synchronize()
        times = []
        for r in range(reps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            plan.execute(dA, dB, dC, stream=stream)
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1) * 1e-3)
            if times[0] > cap:
                break
        plan.device_status()
        out.append(float(np.median(times)))
        capped.append(times[0] > cap)
    return out, capped


def study(spec, extents, dtype="f64", seed=0, reps=5, cap=2.0, ids=None):
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    tdt = {"f64": torch.float64, "f32": torch.float32}.get(dtype, torch.float32)
    A, B, _ = synth.uniform_operands(spec, extents, seed=seed)
    nC = synth.dense_sizes(spec, extents)[0]
    dA = torch.from_numpy(A).to(tdt).to(dev)
    dB = torch.from_numpy(B).to(tdt).to(dev)
    dC = torch.zeros(nC, dtype=tdt, device=dev)
    plan = tc.Plan(spec, extents, dtype=dtype)
    algs = plan.algorithms()
    if ids is None:
        ids = [a["id"] for a in algs]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    pred = plan.predict(ids, dA, dB, dC)
    t_pred = time.perf_counter() - t0
    runnable = [i for i, p in zip(ids, pred) if p > 0]
    flush = torch.empty(int(256 << 20) // 4, dtype=torch.float32, device=dev)
    t0 = time.perf_counter()
    meas, capped = measure(plan, runnable, dA, dB, dC, flush, reps=reps, cap=cap)
    t_meas = time.perf_counter() - t0
    pmap = dict(zip(ids, pred))
    p = [pmap[i] for i in runnable]
    best_pred = runnable[int(np.argmin(p))]
    best_meas = runnable[int(np.argmin(meas))]
    mmap = dict(zip(runnable, meas))
    rows = [{"id": i, "name": algs[i]["name"], "predicted_s": pmap[i], "measured_s": mmap[i],
             "capped": c} for i, c in zip(runnable, capped)]
    plan.close()
    return {
        "spec": spec, "extents": list(extents), "dtype": dtype, "algorithms": rows,
        "spearman": spearman(p, meas), "kendall": kendall(p, meas),
        "top_pred": algs[best_pred]["name"], "top_meas": algs[best_meas]["name"],
        "top1_regret": mmap[best_pred] / mmap[best_meas] - 1.0,
        "prediction_seconds": t_pred, "measurement_seconds": t_meas,
    }


def class_study(spec, extents, dtype="f32", seed=0, reps=5, top=3, hbm_gbs=None):
    """Per kernel class (Table 1: dot, axpy, gemv, ger, gemm): predict every
    algorithm of the class, measure the `top` best predicted, and report the
    class's best measured time with its compulsory traffic (A, B, C read
    once, C written once) as GB/s -- the classes' own access patterns at a
    size past L2."""
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    tdt = {"f64": torch.float64, "f32": torch.float32}[dtype]
    esz = 8 if dtype == "f64" else 4
    A, B, _ = synth.uniform_operands(spec, extents, seed=seed)
    nC, nA, nB = synth.dense_sizes(spec, extents)
    dA = torch.from_numpy(A).to(tdt).to(dev)
    dB = torch.from_numpy(B).to(tdt).to(dev)
    dC = torch.zeros(nC, dtype=tdt, device=dev)
    plan = tc.Plan(spec, extents, dtype=dtype)
    algs = plan.algorithms()
    flops = 2.0 * float(np.prod([float(e) for e in extents]))
    nbytes = (nA + nB + 2 * nC) * esz
    flush = torch.empty(int(256 << 20) // 4, dtype=torch.float32, device=dev)
    out = {}
    for kind in ("dot", "axpy", "gemv", "ger", "gemm"):
        ids = [a["id"] for a in algs if a["kernel"] == kind]
        if not ids:
            continue
        pred = plan.predict(ids, dA, dB, dC)
        order = [i for _, i in sorted(zip(pred, ids)) if _ > 0][:top]
        meas, _ = measure(plan, order, dA, dB, dC, flush, reps=reps, cap=5.0)
        j = int(np.argmin(meas))
        t = meas[j]
        row = {"algorithms": len(ids), "measured": len(order), "best": algs[order[j]]["name"],
               "ms": t * 1e3, "gflops": flops / t / 1e9, "compulsory_gbs": nbytes / t / 1e9,
               "top_predicted": algs[order[0]]["name"], "top_predicted_ms": meas[0] * 1e3}
        if hbm_gbs:
            row["hbm_frac"] = row["compulsory_gbs"] / hbm_gbs
        out[kind] = row
    plan.close()
    return {"spec": spec, "extents": list(extents), "dtype": dtype, "gflop": flops / 1e9,
            "compulsory_gb": nbytes / 1e9, "classes": out}


def execute_named(spec, extents, dtype, names, runs=2):
    """Runs the named algorithms `runs` times each on uniform inputs."""
    import torch
    tdt = {"f64": torch.float64, "f32": torch.float32}[dtype]
    A, B, _ = synth.uniform_operands(spec, extents, seed=0)
    dA, dB = torch.from_numpy(A).to(tdt).cuda(), torch.from_numpy(B).to(tdt).cuda()
    dC = torch.zeros(synth.dense_sizes(spec, extents)[0], dtype=tdt, device="cuda")
    plan = tc.Plan(spec, extents, dtype=dtype)
    ids = {a["name"]: a["id"] for a in plan.algorithms()}
    for n in names:
        plan.select(ids[n])
        for _ in range(runs):
            plan.execute(dA, dB, dC)
        torch.cuda.synchronize()
    plan.device_status()
    plan.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--spec", default="abc=iaj,jbic")
    ap.add_argument("--extents", default="128,128,128,16,16")
    ap.add_argument("--dtype", default="f64")
    ap.add_argument("--reps", type=int, default=5)
    ap.add_argument("--cap", type=float, default=2.0)
    ap.add_argument("--json", default=None)
    ap.add_argument("--classes", action="store_true", help="per-kernel-class study instead")
    ap.add_argument("--execute", default=None,
                    help="comma-separated algorithm names: run each twice, nothing else (profiler captures)")
    args = ap.parse_args()
    ext = [int(x) for x in args.extents.split(",")]
    if args.execute:
        execute_named(args.spec, ext, args.dtype, args.execute.split(","))
        return
    if args.classes:
        print(json.dumps(class_study(args.spec, ext, args.dtype, reps=args.reps)))
        return
    r = study(args.spec, ext, args.dtype, reps=args.reps, cap=args.cap)
    summary = {k: v for k, v in r.items() if k != "algorithms"}
    print(json.dumps(summary))
    if args.json:
        with open(args.json, "w") as f:
            json.dump(r, f, indent=1)


if __name__ == "__main__":
    main()
