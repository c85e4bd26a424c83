"""Batched-form measurement: 4096 independent C[a,b,c] = sum_i A[a,i] B[i,b,c]
with a, b, c log-uniform in [8, 128] and i drawn from {4, 8, 16, 32},
entries uniform in [-1, 1], seed 0.

    python -m paper_1409_8608_gb300.batch_report [--count 4096] [--dtype f32]

Times (CUDA events, median of `reps`, inputs resident, beta = 0): the
single persistent launch with per-problem tiles ("tuned"), the same with
64x64 tiles everywhere ("untuned"), the tuned launch replayed from a CUDA
graph, and one launch per problem.  Reports GFLOP/s and the compulsory
bytes (A, B, C once) over time against the measured HBM bandwidth.
"""
import argparse
import json
import statistics

import numpy as np

from . import synth, tc

SPEC = "abc=ai,ibc"


def problems(count, seed=0):
    rng = np.random.default_rng(seed)
    a, b, c = (synth.log_uniform_int(rng, 8, 128, count) for _ in range(3))
    i = rng.choice([4, 8, 16, 32], count)
    return [[int(x) for x in r] for r in zip(a, b, c, i)]


def _time(fn, reps, stream):
    import torch
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


def run(count=4096, dtype="f32", seed=0, reps=10, hbm_gbs=6758.5):
    import torch
    rows = problems(count, seed)
    tdt = {"f32": torch.float32, "f64": torch.float64, "bf16x3": torch.float32}[dtype]
    rng = torch.Generator(device="cuda").manual_seed(seed)
    As, Bs, Cs = [], [], []
    for a, b, c, i in rows:
        As.append(torch.rand(a * i, dtype=tdt, device="cuda", generator=rng) * 2 - 1)
        Bs.append(torch.rand(i * b * c, dtype=tdt, device="cuda", generator=rng) * 2 - 1)
        Cs.append(torch.empty(a * b * c, dtype=tdt, device="cuda"))
    batch = tc.Batch(SPEC, rows, dtype)
    batch.set_operands(As, Bs, Cs)
    stream = torch.cuda.Stream()
    info = batch.info()
    res = {"problems": count, "dtype": dtype, "gflop": info["flops"] / 1e9,
           "compulsory_gb": info["bytes"] / 1e9}
    with torch.cuda.stream(stream):
        for policy, key in ((1, "tuned"), (0, "untuned")):
            batch.set_tiles(policy)
            batch.prepare()
            batch.execute(stream=stream)  # warm-up
            t = _time(lambda: batch.execute(stream=stream), reps, stream)
            res[key] = {"ms": t * 1e3, "gflops": info["flops"] / t / 1e9,
                        "gbs": info["bytes"] / t / 1e9, "hbm_frac": info["bytes"] / t / 1e9 / hbm_gbs,
                        "tiles": batch.info()["tiles"]}
        batch.set_tiles(1)
        batch.prepare()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            batch.execute(stream=stream)
        g.replay()
        t = _time(g.replay, reps, stream)
        res["graph"] = {"ms": t * 1e3, "gflops": info["flops"] / t / 1e9}
        batch.execute(per_problem=True, stream=stream)
        t = _time(lambda: batch.execute(per_problem=True, stream=stream), max(2, reps // 3), stream)
        res["launch_per_problem"] = {"ms": t * 1e3, "gflops": info["flops"] / t / 1e9, "launches": count}
    torch.cuda.synchronize()
    batch.device_status()
    batch.close()
    return res


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--count", type=int, default=4096)
    ap.add_argument("--dtype", default="f32")
    ap.add_argument("--reps", type=int, default=10)
    args = ap.parse_args()
    print(json.dumps(run(args.count, args.dtype, reps=args.reps)))


if __name__ == "__main__":
    main()
