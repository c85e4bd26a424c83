"""Precision-form measurement: error against the FP64 oracle and speed of the
tensor-core forms on the precision workloads.

    python -m paper_1409_8608_gb300.precision_report [--points 4000]

Workloads: C[a,b,c] = sum_i A[a,i] B[i,b,c] with a=b=c=512, i=64, and
C[a,b] = sum_{i,j} A[a,i,j] B[j,i,b] with a=b=4096, i=j=64; inputs uniform
in [-1, 1] (seed 0) and uniform times a lognormal scale per index value of
each operand's last mode (seed 1).  Forms: plain FP64 and FP32, TF32, BF16,
FP16 and split-BF16 with 3, 6 and 9 slice products (FP32 inputs rounded to
the form's input type first for BF16/FP16); split-BF16 with 6 products also
without compensated accumulation ("c0") and with 64-element chunks ("c64").  Error: the largest
componentwise |c_hat - c| / (|A||B|) over sampled outputs, each computed one
by one by the oracle in FP64 from the user's data (FP64 for the FP64 form,
the FP32 values for every other form, so that rounding the inputs to BF16,
FP16 or TF32 counts as error).  Time: CUDA events, median of 5 after a warm-up.
"""
import argparse
import json
import statistics

import numpy as np

from . import synth, tc

WORKLOADS = (("abc=ai,ibc", [512, 512, 512, 64]), ("ab=aij,jib", [4096, 4096, 64, 64]))
# (dtype, slice products, compensation chunk: None = the plan's default)
FORMS = (("f64", None, None), ("f32", None, None), ("tf32", None, None), ("bf16", None, None),
         ("f16", None, None), ("bf16x3", 3, None), ("bf16x3", 6, 0), ("bf16x3", 6, None),
         ("bf16x3", 6, 64), ("bf16x3", 9, None))


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


def run(points=4000, reps=5):
    import torch
    from oracle import contraction as oc  # the checker; measurement only
    rows = []
    stream = torch.cuda.current_stream()
    for spec, ext in WORKLOADS:
        for dist, gen in (("uniform", synth.uniform_operands), ("lognormal", synth.lognormal_slice_operands)):
            A, B, _ = gen(spec, ext, seed=0 if dist == "uniform" else 1)
            nC = synth.dense_sizes(spec, ext)[0]
            order = synth.index_order(spec)
            cmodes = synth.spec_modes(spec)[0]
            rng = np.random.default_rng(7)
            e = dict(zip(order, ext))
            pts = np.stack([rng.integers(0, e[m], points) for m in cmodes], axis=1)
            lin = np.zeros(points, dtype=np.int64)
            mul = 1
            for k, m in enumerate(cmodes):
                lin += pts[:, k] * mul
                mul *= e[m]
            for dtype, prod, comp in FORMS:
                tin = {"f64": torch.float64, "bf16": torch.bfloat16, "f16": torch.float16}.get(dtype, torch.float32)
                tout = torch.float64 if dtype == "f64" else torch.float32
                dA = torch.from_numpy(A).to(tin).cuda()
                dB = torch.from_numpy(B).to(tin).cuda()
                dC = torch.empty(nC, dtype=tout, device="cuda")
                plan = tc.Plan(spec, ext, dtype=dtype)
                if prod:
                    plan.set_split(prod)
                if comp is not None:
                    plan.set_compensation(comp)
                plan.select(0)
                run1 = lambda: plan.execute(dA, dB, dC, stream=stream)
                run1()
                t = _time(run1, reps, stream)
                got = dC[torch.from_numpy(lin).cuda()].double().cpu().numpy()
                # reference: the user's data -- FP64 for the FP64 form, the
                # FP32 values for every other form (so input rounding to
                # BF16 / FP16 / TF32 counts as error)
                if dtype == "f64":
                    Ar, Br = A, B
                else:
                    Ar = A.astype(np.float32).astype(np.float64)
                    Br = B.astype(np.float32).astype(np.float64)
                want = oc.contract_points(spec, ext, Ar, Br, pts, threads=8)
                scale = oc.contract_points(spec, ext, np.abs(Ar), np.abs(Br), pts, threads=8)
                err = float(np.max(np.abs(got - want) / scale))
                flops = plan.flops
                plan.close()
                rows.append({"workload": f"{spec} {ext}", "inputs": dist,
                             "form": dtype + (f"x{prod}" if prod else "") + (f"c{comp}" if comp is not None else ""), "max_err": err,
                             "ms": t * 1e3, "gflops": flops / t / 1e9})
                del dA, dB, dC
                torch.cuda.empty_cache()
    return rows


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--points", type=int, default=4000)
    ap.add_argument("--json", default=None)
    args = ap.parse_args()
    rows = run(args.points)
    for r in rows:
        print(json.dumps(r))
    if args.json:
        with open(args.json, "w") as f:
            json.dump(rows, f, indent=1)


if __name__ == "__main__":
    main()
