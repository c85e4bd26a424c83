"""Serving measurement: a Poisson stream of contraction requests through
tc_server (continuous batching).

    python -m paper_1409_8608_gb300.serve_report [--seconds 10] [--rate 2000]

Requests: specs abc=ai,ibc / abc=iaj,jbic / ab=aij,jib (one third each);
free extents log-uniform in [16, 384], contracted extents log-uniform in
[8, 128]; dtypes FP64 : FP32 : split-BF16 = 1 : 2 : 2; 40 GB admission
budget; seeded.  Inputs are pinned host memory (views into a pool of
uniform [-1, 1] values per element type; an operand larger than the pool is
redrawn); the result stays on the device (latency = submission to result
ready).  Reports p50/p99 latency, served and offered GFLOP/s, admission
stalls.
"""
import argparse
import json
import math
import time

import numpy as np

from . import synth, tc

SPECS = ("abc=ai,ibc", "abc=iaj,jbic", "ab=aij,jib")
DTYPES = ("f64", "f32", "bf16x3")
DTYPE_P = (0.2, 0.4, 0.4)


def draw_request(rng):
    spec = SPECS[rng.integers(0, 3)]
    dtype = DTYPES[rng.choice(3, p=DTYPE_P)]
    order = synth.index_order(spec)
    c, a, b = synth.spec_modes(spec)
    ext = []
    for x in order:
        contracted = x in a and x in b and x not in c
        lo, hi = (8, 128) if contracted else (16, 384)
        ext.append(int(synth.log_uniform_int(rng, lo, hi)))
    return spec, ext, dtype


def run(seconds=2.0, rate=2000.0, seed=0, budget=40 << 30, slots=64, streams=16, pool_bytes=4 << 30):
    import torch
    rng = np.random.default_rng(seed)
    pools = {}
    for dt, tdt in (("f64", torch.float64), ("f32", torch.float32)):
        n = pool_bytes // (8 if dt == "f64" else 4)
        pool = torch.empty(n, dtype=tdt).pin_memory()
        pool.uniform_(-1.0, 1.0, generator=torch.Generator().manual_seed(seed))
        pools[dt] = pool
    pools["bf16x3"] = pools["f32"]
    server = tc.Server(budget, slots, streams)
    arrivals, t = [], 0.0
    while True:
        t += rng.exponential(1.0 / rate)
        if t >= seconds:
            break
        arrivals.append(t)
    reqs, offered = [], 0.0
    for _ in arrivals:
        while True:
            spec, ext, dtype = draw_request(rng)
            esz = 8 if dtype == "f64" else 4
            nc, na, nb = synth.dense_sizes(spec, ext)
            if max(na, nb) * esz <= pool_bytes:
                break
        pool = pools[dtype]
        limit = pool.numel()
        oa = int(rng.integers(0, (limit - na) // 64 + 1)) * 64  # 256-byte aligned views
        ob = int(rng.integers(0, (limit - nb) // 64 + 1)) * 64
        base = pool.data_ptr()
        reqs.append((spec, ext, dtype, base + oa * esz, base + ob * esz))
        offered += 2.0 * math.prod(ext)
    ids = []
    t0 = time.perf_counter()
    for ta, (spec, ext, dtype, pa, pb) in zip(arrivals, reqs):
        while time.perf_counter() - t0 < ta:
            pass
        ids.append(server.submit(spec, ext, dtype, pa, pb, None))
    for rid, (spec, ext, dtype, _, _) in zip(ids, reqs):
        try:
            server.wait(rid, timeout=600.0)
        except tc.TcError as e:
            raise RuntimeError(f"request {rid} ({spec} {ext} {dtype}) failed: {e}") from e
    wall = time.perf_counter() - t0
    st = server.stats()
    server.close()
    return {
        "requests": len(ids), "seconds_of_arrivals": seconds, "rate_per_s": rate,
        "offered_gflops": offered / seconds / 1e9,
        "served_gflops": st["flops_served"] / wall / 1e9,
        "p50_ms": st["p50_seconds"] * 1e3, "p99_ms": st["p99_seconds"] * 1e3,
        "max_ms": st["max_seconds"] * 1e3, "admission_stalls": st["admission_stalls"],
        "peak_inflight": st["peak_inflight"], "completed": st["completed"], "failed": st["failed"],
        "wall_s": wall,
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--seconds", type=float, default=10.0)
    ap.add_argument("--rate", type=float, default=2000.0)
    ap.add_argument("--seed", type=int, default=0)
    args = ap.parse_args()
    print(json.dumps(run(args.seconds, args.rate, args.seed)))


if __name__ == "__main__":
    main()
