"""Oracle (test infrastructure, not product code) for algorithm generation.

Restates Section 2 ("Algorithm Generation") in plain Python:

* Table 1 fixes, per BLAS kernel, how many contracted and free indices the
  kernel itself handles: dot 1 contracted / 0 free; axpy 0 contracted / one
  free index in exactly one of A, B; gemv 1 contracted / one free index in
  exactly one of A, B; ger 0 contracted / one free index in A and one in B;
  gemm 1 contracted / one free in A and one free in B.  Every other index is
  sliced, i.e. becomes a loop around the kernel.
* All kernels, all admissible choices of kernel indices and all permutations
  of the sliced loops are generated (Section 2, last paragraph).
* A matrix operand of gemv, ger or gemm needs one unit-stride dimension; a
  matrix slice without one is first copied into a contiguous temporary.  The
  copy sits in the body of the innermost loop whose index the slice depends
  on (the listings of "i'c-gemm" and "ci'-gemm" in the Test 3 algorithms).
* Names are the sliced loop indices in nest order, an apostrophe after the
  loop that holds a copy, then "-" and the kernel (footnote to the gemm
  example of Section 2).

Enumeration order (the paper numbers its plots but states no rule; this
order reproduces the numbering of the case-study and Test 3 legends): kernels
dot, axpy, gemv, ger, gemm; then kernel-index choices with the free index of
A outermost, then the free index of B, then the contracted index; then the
loop permutations in lexicographic order of the sliced indices, which are
ranked by first appearance in the spec string.

A reading where the paper is silent: a C slice without a unit-stride mode is
also given a copy (computed into a zeroed temporary and added back).

Only ``tests/`` may import this module.
"""
import itertools

from .contraction import fortran_strides, index_order, parse_spec

KERNELS = ("dot", "axpy", "gemv", "ger", "gemm")


def classify(spec):
    """Contracted, free-in-A and free-in-B indices, in first-appearance order."""
    c, a, b = parse_spec(spec)
    order = index_order(spec)
    contracted = [x for x in order if x in a and x in b and x not in c]
    free_a = [x for x in order if x in a and x not in b and x in c]
    free_b = [x for x in order if x in b and x not in a and x in c]
    return contracted, free_a, free_b


def kernel_index_choices(kernel, contracted, free_a, free_b):
    """Table 1: admissible sets of kernel indices, in enumeration order."""
    if kernel == "dot":
        return [(k,) for k in contracted]
    if kernel == "axpy":
        return [(f,) for f in free_a] + [(f,) for f in free_b]
    if kernel == "gemv":
        return [(f, k) for f in free_a + free_b for k in contracted]
    if kernel == "ger":
        return [(fa, fb) for fa in free_a for fb in free_b]
    if kernel == "gemm":
        return [(fa, fb, k) for fa in free_a for fb in free_b
                for k in contracted]
    raise ValueError(kernel)


def _strides_by_operand(spec, extents, strides):
    c, a, b = parse_spec(spec)
    order = index_order(spec)
    ext = dict(zip(order, extents))
    if strides is None:
        sc, sa, sb = (fortran_strides(m, ext) for m in (c, a, b))
    else:
        sc = list(strides[:len(c)])
        sa = list(strides[len(c):len(c) + len(a)])
        sb = list(strides[len(c) + len(a):])
    return {"C": dict(zip(c, sc)), "A": dict(zip(a, sa)),
            "B": dict(zip(b, sb))}


def enumerate_algorithms(spec, extents=None, strides=None):
    """All algorithms of Section 2 for ``spec``.

    Each algorithm is a dict with ``name``, ``kernel``, ``kernel_indices``,
    ``loops`` (sliced indices, outermost first), per operand the kernel modes
    of its slice (``slice_modes``, storage order) and the copies
    (``copies``: operand -> position of the loop that holds the copy, -1 for
    a copy before every loop).
    """
    c, a, b = parse_spec(spec)
    order = index_order(spec)
    if extents is None:
        extents = [2] * len(order)
    by_op = _strides_by_operand(spec, list(extents), strides)
    modes = {"A": a, "B": b, "C": c}
    contracted, free_a, free_b = classify(spec)
    algs = []
    for kernel in KERNELS:
        for kidx in kernel_index_choices(kernel, contracted, free_a, free_b):
            sliced = [x for x in order if x not in kidx]
            for loops in itertools.permutations(sliced):
                slice_modes = {op: [m for m in modes[op] if m in kidx]
                               for op in ("A", "B", "C")}
                copies = {}
                for op in ("A", "B", "C"):
                    km = slice_modes[op]
                    if len(km) != 2:
                        continue  # scalars and vectors take any stride
                    if any(by_op[op][m] == 1 for m in km):
                        continue
                    deps = [p for p, l in enumerate(loops) if l in modes[op]]
                    copies[op] = max(deps) if deps else -1
                name = "'" * sum(1 for v in copies.values() if v == -1)
                for p, l in enumerate(loops):
                    name += l + "'" * sum(1 for v in copies.values() if v == p)
                algs.append({
                    "id": len(algs),
                    "name": name + "-" + kernel,
                    "kernel": kernel,
                    "kernel_indices": tuple(kidx),
                    "loops": tuple(loops),
                    "slice_modes": slice_modes,
                    "copies": copies,
                })
    return algs


def count_by_kernel(algs):
    out = {k: 0 for k in KERNELS}
    for alg in algs:
        out[alg["kernel"]] += 1
    return out
