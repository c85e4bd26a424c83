"""Oracle (test infrastructure, not product code) for the cache analysis of
Section 3 ("Performance Prediction").

It restates, for one algorithm (a loop nest around one kernel, as produced by
``oracle.algorithms``), the integer part of the predictor:

* Section 3.2, access distance: for each kernel operand, walk from the
  kernel up through the surrounding loops.  (1) If the operand, joined along
  the loops passed so far, does not vary across the next loop, stop.  (2) If
  it varies, the collected set M becomes every kernel operand joined along
  all loops passed so far plus this one; go up one level.  (3) At the root,
  keep the M collected so far (the contraction is assumed to run
  repeatedly).  The distance is the summed size of the regions in M.
* Section 3.2, setup list: operands by decreasing distance, each followed by
  a remote region so that everything to an operand's right sums to its
  distance; the front of the list is cut so that it totals at most 5/4 of
  the cache size.
* Section 3.3, line sharing / prefetch: an operand is prefetched when it
  varies across the innermost loop and that loop indexes its first
  dimension, or its second dimension while the first is covered entirely by
  the slice or fits in one cache line.  A prefetched operand is accessed
  right before the kernel (prefetch distance 0), limited to one cache line
  along its first dimension.  A setup that touches only operands is omitted.
* Section 3.4, prefetch failures: operands that share lines along their first
  dimension miss once per cache line; a second case without the prefetch
  accesses covers those invocations.
* Section 3.5, first iterations: the first iteration of the innermost loop
  (and of any outer loop entered more than 1% as often as the kernel runs)
  is a case of its own, whose walk starts at that loop with every kernel
  region already joined across it and the loops inside it.
* Weighted sum: each case carries the number of invocations it stands for.

Readings where the paper is silent (each stated in the design notes):
remote regions that would be negative are dropped (size 0); equal distances
keep the order of the plain access distances (larger first), then operand
order C, A, B; a truncated operand turns into a remote region of the size
left; misses are counted as the iterations 1.. n-1 of the innermost loop
that start a new line, i.e. floor((n - 1) / line_elems) per traversal.

Sizes are in elements times ``elem_bytes`` (pass 1 to count elements as the
paper's worked example does, in doubles).  Only ``tests/`` imports this.
"""
from .contraction import parse_spec

OPERANDS = ("C", "A", "B")


def _modes(spec):
    c, a, b = parse_spec(spec)
    return {"C": c, "A": a, "B": b}


def region_size(spec, ext, alg, op, joined):
    """Size (elements) of ``op``'s kernel slice joined along ``joined``."""
    size = 1
    for m in _modes(spec)[op]:
        if m in alg["kernel_indices"] or m in joined:
            size *= ext[m]
    return size


def access_distance(spec, ext, alg, op, start_depth=None):
    """Section 3.2 walk for one operand.

    ``start_depth=None`` starts at the kernel.  ``start_depth=d`` starts at
    loop d for the first-iteration case of Section 3.5: M then already holds
    every kernel region joined along loops d..n-1.
    Returns (distance, M) with M a list of (operand, sorted joined indices).
    """
    loops = list(alg["loops"])
    modes = _modes(spec)
    if start_depth is None:
        joined, level = set(), len(loops) - 1
        M = []
    else:
        joined = set(loops[start_depth:])
        level = start_depth - 1
        M = [(x, tuple(sorted(joined & set(modes[x])))) for x in OPERANDS]
    while level >= 0:
        l = loops[level]
        if l not in modes[op]:
            break  # case 1: invariant across the surrounding loop
        joined.add(l)  # case 2: varies, join every operand along it
        M = [(x, tuple(sorted(joined & set(modes[x])))) for x in OPERANDS]
        level -= 1
    # case 3 (root) keeps M as collected
    dist = sum(region_size(spec, ext, alg, x, set(j)) for x, j in M)
    return dist, M


def prefetched(spec, ext, alg, op, line_elems):
    """Section 3.3 conditions.  Returns None, "first" (line sharing along the
    first dimension, which also fails once per line) or "second"."""
    loops = alg["loops"]
    if not loops:
        return None
    l = loops[-1]
    m = _modes(spec)[op]
    if l not in m:
        return None
    if m[0] == l:
        return "first"
    if len(m) > 1 and m[1] == l:
        d0 = m[0]
        if d0 in alg["kernel_indices"] or ext[d0] <= line_elems:
            return "second"
    return None


def prefetch_access_size(spec, ext, alg, op, line_elems):
    """Prefetch access: the slice, limited to one line along dimension 1."""
    m = _modes(spec)[op]
    size = 1
    for k, x in enumerate(m):
        if x in alg["kernel_indices"]:
            size *= min(ext[x], line_elems) if k == 0 else ext[x]
    return size


def build_setup(entries):
    """entries: (operand, size, distance, tie_key) -> setup list.

    The list holds ("op", name, size) and ("remote", size) items, first
    accessed first.  Returns the list before truncation.
    """
    order = sorted(entries, key=lambda e: (-e[2], e[3]))
    out = []
    # walk from the back: each operand's distance is what follows it
    tail = 0
    rev = []
    for name, size, dist, _ in reversed(order):
        remote = max(dist - tail, 0)
        rev.append(("remote", remote))
        rev.append(("op", name, size))
        tail += remote + size
    for item in reversed(rev):
        if item[0] == "remote" and item[1] == 0:
            continue
        out.append(item)
    return out


def truncate(setup, limit):
    """Cut the front of the list so that it totals at most ``limit``."""
    kept, total = [], 0
    for item in reversed(setup):
        size = item[-1]
        if total + size <= limit:
            kept.append(item)
            total += size
            continue
        left = limit - total
        if left > 0:
            kept.append(("remote", left))
        break
    return list(reversed(kept))


def only_operands(setup):
    return all(item[0] == "op" for item in setup)


def steady_setups(spec, ext, alg, cache_elems, line_elems):
    """Setup lists of the steady-state cases: (hit list, miss list or None).

    The hit list applies the prefetch emulation; the miss list (Section 3.4)
    drops it for operands that share lines along their first dimension.
    """
    limit = cache_elems * 5 // 4
    plain = {op: access_distance(spec, ext, alg, op)[0] for op in OPERANDS}
    size = {op: region_size(spec, ext, alg, op, set()) for op in OPERANDS}
    tie = {op: (-plain[op], OPERANDS.index(op)) for op in OPERANDS}
    kinds = {op: prefetched(spec, ext, alg, op, line_elems)
             for op in OPERANDS}

    def entries(with_prefetch):
        out = []
        for op in OPERANDS:
            if with_prefetch and kinds[op] is not None:
                out.append((op, prefetch_access_size(spec, ext, alg, op,
                                                     line_elems), 0, tie[op]))
            else:
                out.append((op, size[op], plain[op], tie[op]))
        return out

    hit = truncate(build_setup(entries(True)), limit)
    miss = None
    if any(k == "first" for k in kinds.values()):
        miss = truncate(build_setup(entries(False)), limit)
    return hit, miss, plain, kinds


def first_iteration_setup(spec, ext, alg, depth, cache_elems):
    """Section 3.5 case for the first iteration of loop ``depth``."""
    limit = cache_elems * 5 // 4
    dist = {op: access_distance(spec, ext, alg, op, start_depth=depth)[0]
            for op in OPERANDS}
    size = {op: region_size(spec, ext, alg, op, set()) for op in OPERANDS}
    ents = [(op, size[op], dist[op], (-dist[op], OPERANDS.index(op)))
            for op in OPERANDS]
    return truncate(build_setup(ents), limit), dist


def first_iteration_loops(alg, ext, threshold=0.01):
    """Loops benchmarked for their first iteration: the innermost one and
    every loop entered more than ``threshold`` times the invocation count."""
    loops = alg["loops"]
    n = len(loops)
    if n == 0:
        return []
    total = 1
    for l in loops:
        total *= ext[l]
    out = []
    entered = 1
    for d in range(n):
        if d == n - 1 or entered > threshold * total:
            out.append(d)
        entered *= ext[loops[d]]
    return out


def case_counts(alg, ext, line_elems, has_miss):
    """Invocation counts per case: {"hit": .., "miss": .., ("first", d): ..}.

    They sum to the product of the loop extents (one invocation when the
    algorithm has no loops, counted as "hit")."""
    loops = alg["loops"]
    n = len(loops)
    total = 1
    for l in loops:
        total *= ext[l]
    if n == 0:
        return {"hit": 1}
    entered = [1]
    for l in loops:
        entered.append(entered[-1] * ext[l])  # entered[d] = prod_{k<d} n_k
    counts = {}
    prev = 0
    for d in first_iteration_loops(alg, ext):
        counts[("first", d)] = entered[d] - prev
        prev = entered[d]
    steady = total - entered[n - 1]
    misses = 0
    if has_miss:
        misses = entered[n - 1] * ((ext[loops[-1]] - 1) // line_elems)
    counts["hit"] = steady - misses
    if has_miss:
        counts["miss"] = misses
    return counts
