"""Oracle (test infrastructure, not product code) for contraction chains.

Section 3.2 ("Operand Access Distance") states that the method is general
enough for abstract syntax trees with several kernels, not only a single
kernel inside a loop nest.  A chain of three operands is the simplest such
tree: ``D = X Y Z`` is computed as one contraction into an intermediate and
a second one out of it.  Whatever the order, the result is fixed by the
notation of Section 1: every entry of D is the sum, over all indices that
do not appear in D, of the product of the three operands' entries.

``contract3`` writes that definition out directly -- every operand is
broadcast onto the full index space, multiplied, and the indices outside D
are summed -- so it is independent of the pairwise contraction and of any
contraction order.  It is only for small index spaces (the full product is
materialised).

Spec convention (the library's): ``"D=X,Y,Z"`` with one letter per index;
extents follow the order of first appearance in the spec string; operands
are flat FP64 arrays stored first index fastest.

Only ``tests/``, the smoke check and the benchmark's CPU-baseline leg may
import this module.
"""
import numpy as np

MAX_TERMS = 1 << 25  # the materialised product's element count


def parse_chain(spec):
    """``"ad=ab,bc,cd"`` -> ("ad", ["ab", "bc", "cd"])."""
    s = spec.replace(" ", "")
    lhs, rhs = s.split("=")
    ops = rhs.split(",")
    if len(ops) != 3:
        raise ValueError("a chain has three operands")
    return lhs, ops


def chain_index_order(spec):
    """Distinct letters in order of first appearance in the spec string."""
    d, ops = parse_chain(spec)
    seen = []
    for ch in d + "".join(ops):
        if ch not in seen:
            seen.append(ch)
    return seen


def chain_sizes(spec, extents):
    """Element counts of D, X, Y, Z stored densely."""
    d, ops = parse_chain(spec)
    ext = dict(zip(chain_index_order(spec), [int(e) for e in extents]))
    return tuple(int(np.prod([ext[m] for m in modes])) if modes else 1 for modes in [d] + ops)


def _on_full_space(flat, modes, letters, ext):
    # the operand as an array over every index (first index fastest in
    # storage), with axes of length 1 for the indices it does not carry
    arr = np.asarray(flat, dtype=np.float64).reshape([ext[m] for m in modes], order="F") if modes else \
        np.asarray(flat, dtype=np.float64).reshape(())
    # order its axes by position in `letters`, then insert the missing ones
    present = [m for m in letters if m in modes]
    arr = np.transpose(arr, [modes.index(m) for m in present]) if modes else arr
    shape = [ext[m] if m in modes else 1 for m in letters]
    return arr.reshape(shape)


def contract3(spec, extents, X, Y, Z):
    """D of ``spec`` in FP64, by the definition (small index spaces only)."""
    d, ops = parse_chain(spec)
    letters = chain_index_order(spec)
    ext = dict(zip(letters, [int(e) for e in extents]))
    total = int(np.prod([ext[m] for m in letters]))
    if total > MAX_TERMS:
        raise ValueError("index space too large for the direct sum")
    for m in letters:
        if m not in d and sum(m in o for o in ops) < 2:
            raise ValueError(f"index {m} appears in one operand only and not in D")
    prod = np.ones([1] * len(letters))
    for flat, modes in zip((X, Y, Z), ops):
        prod = prod * _on_full_space(flat, modes, letters, ext)
    summed = tuple(i for i, m in enumerate(letters) if m not in d)
    out = prod.sum(axis=summed) if summed else prod
    kept = [m for m in letters if m in d]  # axes left, in `letters` order
    out = np.transpose(out, [kept.index(m) for m in d]) if d else out
    return np.asarray(out).reshape(-1, order="F").copy()


def chain_flops(spec, extents, first):
    """Multiply-add count (x2) of contracting operands `first` (a pair of
    positions) first and the result with the third: each pairwise step
    costs 2 x the product of the extents of the indices its operands carry."""
    d, ops = parse_chain(spec)
    ext = dict(zip(chain_index_order(spec), [int(e) for e in extents]))
    p, q = first
    r = 3 - p - q
    step1 = set(ops[p]) | set(ops[q])
    t = [m for m in step1 if m in d or m in ops[r]]
    step2 = set(t) | set(ops[r])
    return 2 * int(np.prod([ext[m] for m in step1])) + 2 * int(np.prod([ext[m] for m in step2]))
