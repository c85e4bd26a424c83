"""Serving measurement: a Poisson stream of contraction requests through
tc_server (continuous batching).

    python -m paper_1409_8608_gb300.serve_report [--seconds 10] [--warmup 1] [--rate 2000]

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


def run(seconds=2.0, rate=2000.0, seed=0, budget=40 << 30, slots=64, streams=16, pool_bytes=4 << 30,
        warmup=0.0, check_samples=0):
    """Submits a Poisson stream for warmup + seconds of arrivals.  Requests
    arriving during the warm-up are served but not counted; the rest form
    the measured window: offered and served GFLOP/s (served = their flops
    over first measured arrival to last measured completion), latency
    percentiles overall and per dtype.  check_samples requests of the
    window also copy their result to host memory and are then run again
    alone on the idle server: both results must be the same bits."""
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
    total = warmup + seconds
    arrivals, t = [], 0.0
    while True:
        t += rng.exponential(1.0 / rate)
        if t >= total:
            break
        arrivals.append(t)
    reqs = []
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
    window = [q for q, ta in enumerate(arrivals) if ta >= warmup]
    checks = {}
    if check_samples and window:
        for q in window[:: max(1, len(window) // check_samples)][:check_samples]:
            spec, ext, dtype, _, _ = reqs[q]
            tdt = torch.float64 if dtype == "f64" else torch.float32
            checks[q] = torch.full((synth.dense_sizes(spec, ext)[0],), float("nan"), dtype=tdt).pin_memory()
    ids, t_sub = [], []
    t0 = time.perf_counter()
    for q, (ta, (spec, ext, dtype, pa, pb)) in enumerate(zip(arrivals, reqs)):
        while time.perf_counter() - t0 < ta:
            pass
        t_sub.append(time.perf_counter() - t0)
        ids.append(server.submit(spec, ext, dtype, pa, pb, checks.get(q)))
    for rid, (spec, ext, dtype, _, _) in zip(ids, reqs):
        try:
            server.wait(rid, timeout=600.0)
        except tc.TcError as e:
            raise RuntimeError(f"request {rid} ({spec} {ext} {dtype}) failed: {e}") from e
    lat = [server.poll(rid)[1] for rid in ids]
    st = server.stats()
    # alone: each checked request again, one at a time, on the idle server
    alone_equal = 0
    for q, hc in checks.items():
        spec, ext, dtype, pa, pb = reqs[q]
        again = torch.full_like(hc, float("nan")).pin_memory()
        server.wait(server.submit(spec, ext, dtype, pa, pb, again), timeout=600.0)
        alone_equal += int(torch.equal(again, hc))
    server.close()

    def pct(v, qq):
        v = sorted(v)
        return v[min(len(v) - 1, int(qq * (len(v) - 1) + 0.5))] * 1e3 if v else None

    def summarize(sel):
        fl = [2.0 * math.prod(reqs[q][1]) for q in sel]
        if not sel:
            return {"requests": 0}
        t_first = min(arrivals[q] for q in sel)
        t_done = max(t_sub[q] + lat[q] for q in sel)
        return {"requests": len(sel), "offered_gflops": sum(fl) / seconds / 1e9,
                "served_gflops": sum(fl) / max(1e-9, t_done - t_first) / 1e9,
                "p50_ms": pct([lat[q] for q in sel], 0.50), "p99_ms": pct([lat[q] for q in sel], 0.99)}

    out = summarize(window)
    out.update({"seconds_of_arrivals": seconds, "warmup_seconds": warmup, "rate_per_s": rate,
                "max_ms": max(lat[q] for q in window) * 1e3 if window else None,
                "admission_stalls": st["admission_stalls"], "peak_inflight": st["peak_inflight"],
                "completed": st["completed"], "failed": st["failed"],
                "by_dtype": {dt: summarize([q for q in window if reqs[q][2] == dt]) for dt in DTYPES}})
    if checks:
        out["alone_vs_mix"] = {"checked": len(checks), "bitwise_equal": alone_equal}
        out["sampled_requests"] = [(reqs[q][0], reqs[q][1]) for q in checks]
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--seconds", type=float, default=10.0)
    ap.add_argument("--rate", type=float, default=2000.0)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--warmup", type=float, default=1.0)
    args = ap.parse_args()
    r = run(args.seconds, args.rate, args.seed, warmup=args.warmup, check_samples=8)
    r.pop("sampled_requests", None)
    print(json.dumps(r))


if __name__ == "__main__":
    main()
