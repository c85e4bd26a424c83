"""Batched-form measurement: 4096 independent C[a,b,c] = sum_i A[a,i] B[i,b,c]
with a, b, c log-uniform in [8, 128] and i drawn from {4, 8, 16, 32},
entries uniform in [-1, 1], seed 0.

    python -m paper_1409_8608_gb300.batch_report [--count 4096] [--dtype f32]

The problems' operands are consecutive slices of three device buffers (one
each for all A, all B and all C, every slice starting on a 16-byte
boundary).  Times (CUDA events, median of `reps`, inputs resident,
beta = 0): the single persistent launch with fixed tiles ("fixed"), with
the rule's tiles ("rule"), and with the autotuner's ("tuned"; the tuner's
per-class table is summarised), the tuned launch replayed from a CUDA
graph, one launch per problem, and end to end ("e2e": the host-to-device
copy of all A and B from pinned memory, the tuned launch, the
device-to-host copy of all C).  Reports GFLOP/s and the compulsory bytes
(A, B, C once) over time against the measured HBM bandwidth.
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


def _slices(sizes, esz):
    # offsets of consecutive slices, each rounded up to 16 bytes
    per = 16 // esz
    offs, o = [], 0
    for n in sizes:
        offs.append(o)
        o += (n + per - 1) // per * per
    return offs, o


def run(count=4096, dtype="f32", seed=0, reps=10, hbm_gbs=6758.5, tune_reps=5):
    import torch
    rows = problems(count, seed)
    tdt = {"f32": torch.float32, "f64": torch.float64, "bf16x3": torch.float32}[dtype]
    esz = 8 if dtype == "f64" else 4
    sizes = [synth.dense_sizes(SPEC, r) for r in rows]  # (C, A, B) elements
    offA, nA = _slices([s[1] for s in sizes], esz)
    offB, nB = _slices([s[2] for s in sizes], esz)
    offC, nC = _slices([s[0] for s in sizes], esz)
    gen = torch.Generator(device="cuda").manual_seed(seed)
    dA = torch.rand(nA, dtype=tdt, device="cuda", generator=gen) * 2 - 1
    dB = torch.rand(nB, dtype=tdt, device="cuda", generator=gen) * 2 - 1
    dC = torch.empty(nC, dtype=tdt, device="cuda")
    As = [dA[o:o + s[1]] for o, s in zip(offA, sizes)]
    Bs = [dB[o:o + s[2]] for o, s in zip(offB, sizes)]
    Cs = [dC[o:o + s[0]] for o, s in zip(offC, sizes)]
    batch = tc.Batch(SPEC, rows, dtype)
    batch.set_operands(As, Bs, Cs)
    stream = torch.cuda.Stream()
    info = batch.info()
    res = {"problems": count, "dtype": dtype, "gflop": info["flops"] / 1e9,
           "compulsory_gb": info["bytes"] / 1e9}

    def leg(key):
        batch.prepare()
        batch.execute(stream=stream)  # warm-up
        t = _time(lambda: batch.execute(stream=stream), reps, stream)
        res[key] = {"ms": t * 1e3, "gflops": info["flops"] / t / 1e9,
                    "gbs": info["bytes"] / t / 1e9, "hbm_frac": info["bytes"] / t / 1e9 / hbm_gbs,
                    "tiles": batch.info()["tiles"]}

    with torch.cuda.stream(stream):
        for policy, key in ((0, "fixed"), (1, "rule")):
            batch.set_tiles(policy)
            leg(key)
        table = batch.autotune(stream=stream, reps=tune_reps)
        cfg = batch.config()
        leg("tuned")
        timed = [r for r in table if r["candidates"] > 0]
        res["tuning"] = {
            "classes": len(table), "candidates_timed": sum(r["candidates"] for r in table),
            "stages": cfg["stages"], "tile_n": cfg["tile_n"],
            # sum over classes of the class alone at its best / rule / fixed
            # configuration (classes alone do not fill the GPU as the mix does)
            "sum_best_ms": 1e3 * sum(r["seconds_best"] for r in timed),
            "sum_rule_ms": 1e3 * sum(r["seconds_rule"] for r in timed),
            "sum_fixed_ms": 1e3 * sum(r["seconds_fixed"] for r in timed),
            "choices": {f"{r['tile_m']}x{r['tile_n']}/k{r['k_chunk']}":
                        sum(x["problems"] for x in table if (x["tile_m"], x["tile_n"], x["k_chunk"]) ==
                            (r["tile_m"], r["tile_n"], r["k_chunk"])) for r in table}}
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            batch.execute(stream=stream)
        g.replay()
        t = _time(g.replay, reps, stream)
        res["graph"] = {"ms": t * 1e3, "gflops": info["flops"] / t / 1e9}
        batch.execute(per_problem=True, stream=stream)
        t = _time(lambda: batch.execute(per_problem=True, stream=stream), max(2, reps // 3), stream)
        res["launch_per_problem"] = {"ms": t * 1e3, "gflops": info["flops"] / t / 1e9, "launches": count}
        # end to end: inputs from pinned host memory, results back
        hA = torch.empty(nA, dtype=tdt, pin_memory=True)
        hB = torch.empty(nB, dtype=tdt, pin_memory=True)
        hC = torch.empty(nC, dtype=tdt, pin_memory=True)
        hA.copy_(dA)
        hB.copy_(dB)

        def e2e():
            dA.copy_(hA, non_blocking=True)
            dB.copy_(hB, non_blocking=True)
            batch.execute(stream=stream)
            hC.copy_(dC, non_blocking=True)

        e2e()
        t = _time(e2e, max(3, reps // 2), stream)
        res["e2e"] = {"ms": t * 1e3, "gflops": info["flops"] / t / 1e9,
                      "h2d_bytes_per_step": (nA + nB) * esz, "d2h_bytes_per_step": nC * esz}
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
