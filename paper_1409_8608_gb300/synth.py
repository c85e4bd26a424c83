"""Seeded synthetic inputs shared by the tests, the benchmark and the smoke
check.  This module only draws random numbers; it holds none of the
contraction's arithmetic and imports neither the library nor the oracle.

Conventions: ``numpy.random.default_rng(seed)``; operands are drawn in FP64
as flat arrays in the order A, then B, then C (only when requested);
extents drawn log-uniformly are ``round(exp(U(ln lo, ln hi)))``.
"""
import math

import numpy as np


def spec_modes(spec):
    lhs, rhs = spec.replace(" ", "").split("=")
    a, b = rhs.split(",")
    return lhs, a, b


def index_order(spec):
    seen = []
    for ch in "".join(spec_modes(spec)):
        if ch not in seen:
            seen.append(ch)
    return seen


def dense_sizes(spec, extents):
    """Element counts of C, A, B stored contiguously."""
    ext = dict(zip(index_order(spec), [int(e) for e in extents]))
    out = []
    for modes in spec_modes(spec):
        n = 1
        for m in modes:
            n *= ext[m]
        out.append(n)
    return tuple(out)


def uniform_operands(spec, extents, seed=0, with_c=False, lo=-1.0, hi=1.0):
    """Entries uniform in [lo, hi]: returns (A, B, C or None), FP64 flat."""
    rng = np.random.default_rng(seed)
    nc, na, nb = dense_sizes(spec, extents)
    A = rng.uniform(lo, hi, na)
    B = rng.uniform(lo, hi, nb)
    C = rng.uniform(lo, hi, nc) if with_c else None
    return A, B, C


def integer_operands(spec, extents, seed=0, with_c=False, bound=8):
    """Integers in [-bound, bound] stored as FP64: every product and partial
    sum is exact in FP64, in FP32 while sums stay below 2**24, and every
    value is exact in BF16, FP16 and TF32."""
    rng = np.random.default_rng(seed)
    nc, na, nb = dense_sizes(spec, extents)
    A = rng.integers(-bound, bound + 1, na).astype(np.float64)
    B = rng.integers(-bound, bound + 1, nb).astype(np.float64)
    C = rng.integers(-bound, bound + 1, nc).astype(np.float64) if with_c else None
    return A, B, C


def lognormal_slice_operands(spec, extents, seed=1, sigma=4.0 * math.log(10.0) / 3.0,
                             clip=1e4):
    """Uniform [-1, 1] entries times one lognormal scale per index value of
    each operand's last mode, exp(N(0, sigma)) clipped to [1/clip, clip]."""
    rng = np.random.default_rng(seed)
    ext = dict(zip(index_order(spec), [int(e) for e in extents]))
    _, ma, mb = spec_modes(spec)
    out = []
    for modes in (ma, mb):
        n = 1
        for m in modes:
            n *= ext[m]
        x = rng.uniform(-1.0, 1.0, n)
        last = ext[modes[-1]]
        scale = np.clip(np.exp(rng.normal(0.0, sigma, last)), 1.0 / clip, clip)
        x = x.reshape(last, n // last) * scale[:, None]  # last mode slowest
        out.append(x.reshape(-1))
    return out[0], out[1], None


def log_uniform_int(rng, lo, hi, size=None):
    v = np.exp(rng.uniform(math.log(lo), math.log(hi), size))
    return np.rint(v).astype(np.int64)
