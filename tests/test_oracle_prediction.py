"""Pins for the oracle's cache analysis (Section 3) against the worked
example printed in Sections 3.2-3.4 and against counting identities."""
import json
import os

import pytest

from oracle import algorithms as oa
from oracle import prediction as op


@pytest.fixture(scope="module")
def example(golden_dir):
    with open(os.path.join(golden_dir, "worked_example_ca_gemv.json")) as f:
        return json.load(f)


def _alg(spec, name):
    return next(a for a in oa.enumerate_algorithms(spec) if a["name"] == name)


def _as_lists(setup):
    return [list(x) for x in setup]


def test_access_distances(example):
    alg = _alg(example["spec"], example["algorithm"])
    ext = example["extents"]
    for name, want in example["operands"].items():
        assert op.region_size(example["spec"], ext, alg, name, set()) == want["size"]
        dist, M = op.access_distance(example["spec"], ext, alg, name)
        assert dist == want["distance"], name
        assert sorted([x, list(j)] for x, j in M) == sorted(want["M"]), name


def test_setup_list_and_truncation(example):
    alg = _alg(example["spec"], example["algorithm"])
    spec, ext = example["spec"], example["extents"]
    ents = []
    for name in ("C", "A", "B"):
        d = op.access_distance(spec, ext, alg, name)[0]
        ents.append((name, op.region_size(spec, ext, alg, name, set()), d,
                     (-d, 0)))
    full = op.build_setup(ents)
    assert _as_lists(full) == example["setup_full"]
    limit = example["cache_elems"] * 5 // 4
    assert limit == example["limit"]
    assert _as_lists(op.truncate(full, limit)) == example["setup_truncated"]
    # what follows each operand sums to its distance (Section 3.2)
    tail = 0
    for item in reversed(full):
        if item[0] == "op":
            assert tail == example["operands"][item[1]]["distance"]
        tail += item[-1]


def test_prefetch_and_failure_cases(example):
    alg = _alg(example["spec"], example["algorithm"])
    hit, miss, plain, kinds = op.steady_setups(
        example["spec"], example["extents"], alg, example["cache_elems"],
        example["line_elems"])
    assert kinds == {"C": "first", "A": "first", "B": None}
    assert _as_lists(hit) == example["setup_prefetch"]
    assert op.only_operands(hit) == example["setup_prefetch_omitted"]
    assert _as_lists(miss) == example["setup_prefetch_failure"]


def test_bi_ger_prefetch_conditions():
    # Section 3.3 example: in bi-ger both A[:,i] (second dimension, first
    # covered entirely) and B[i,b,:] (first dimension) are prefetched
    spec = "abc=ai,ibc"
    ext = {"a": 400, "b": 400, "c": 400, "i": 8}
    alg = _alg(spec, "bi-ger")
    assert op.prefetched(spec, ext, alg, "A", 8) == "second"
    assert op.prefetched(spec, ext, alg, "B", 8) == "first"
    assert op.prefetched(spec, ext, alg, "C", 8) is None


def test_ci_ger_first_iteration():
    # Section 3.5 example: in ci-ger the first i iteration (a new c) finds
    # C[:,:,c] at a new location (distance: everything), while A's previous
    # access lies one full i-traversal back
    spec = "abc=ai,ibc"
    ext = {"a": 64, "b": 64, "c": 64, "i": 8}
    alg = _alg(spec, "ci-ger")
    # loop c is entered once (< 1% of 512 invocations): only i is benchmarked
    assert op.first_iteration_loops(alg, ext) == [1]
    setup, dist = op.first_iteration_setup(spec, ext, alg, 1, 10 ** 9)
    whole = 64 * 8 + 8 * 64 * 64 + 64 ** 3
    assert dist["C"] == whole and dist["B"] == whole
    assert dist["A"] == 64 * 8 + 8 * 64 + 64 * 64
    # steady state: C is invariant across i
    assert op.access_distance(spec, ext, alg, "C")[0] == 0


@pytest.mark.parametrize("spec,ext", [
    ("abc=ai,ibc", {"a": 64, "b": 64, "c": 64, "i": 8}),
    ("abc=iaj,jbic", {"a": 24, "b": 20, "c": 16, "i": 16, "j": 16}),
    ("a=iaj,ji", {"a": 100, "i": 30, "j": 50}),
])
def test_case_counts_sum_to_invocations(spec, ext):
    for alg in oa.enumerate_algorithms(spec):
        total = 1
        for l in alg["loops"]:
            total *= ext[l]
        for has_miss in (False, True):
            counts = op.case_counts(alg, ext, 8, has_miss)
            assert sum(counts.values()) == total, alg["name"]
            assert all(v >= 0 for v in counts.values())


def test_distances_never_exceed_the_joined_tensors():
    spec = "abc=iaj,jbic"
    ext = {"a": 24, "b": 20, "c": 16, "i": 16, "j": 16}
    whole = 24 * 16 * 16 + 16 * 20 * 16 * 16 + 24 * 20 * 16
    for alg in oa.enumerate_algorithms(spec):
        for name in ("A", "B", "C"):
            d, _ = op.access_distance(spec, ext, alg, name)
            assert 0 <= d <= whole
            # an operand that varies across the innermost loop was last
            # touched at least one kernel invocation ago
            if alg["loops"] and alg["loops"][-1] in {"A": "iaj", "B": "jbic", "C": "abc"}[name]:
                assert d > 0


def _counts(spec, ext, name, cache_elems, line_elems):
    alg = _alg(spec, name)
    _, miss, _, _ = op.steady_setups(spec, ext, alg, cache_elems, line_elems)
    return op.case_counts(alg, ext, line_elems, miss is not None)


def test_case_counts_ca_gemv_worked_example():
    # Section 3.4 on the worked example (ca-gemv, a=b=c=400, i=8, 8 doubles
    # per line): A[a,:] and C[a,:,c] share lines along a, so the prefetch
    # fails once every 8 iterations of the innermost loop a.  Written out by
    # hand: the loop nest runs 400 (c) x 400 (a) = 160,000 gemv calls.
    #  * first a iteration of each c (Section 3.5, its own case): 400 calls;
    #  * the other 399 a values of a traversal start a new line at
    #    a = 8, 16, ..., 392: 49 per traversal, 400 * 49 = 19,600 misses;
    #  * the rest hit: 400 * (399 - 49) = 140,000.
    spec, ext = "abc=ai,ibc", {"a": 400, "b": 400, "c": 400, "i": 8}
    got = _counts(spec, ext, "ca-gemv", 786432, 8)
    assert got == {("first", 1): 400, "miss": 19600, "hit": 140000}


def test_case_counts_ci_ger():
    # ci-ger (Section 3.5 example), a=b=c=64, i=8: 64 (c) x 8 (i) = 512 ger
    # calls.  Loop c is entered once, below 1 % of 512, so only the first
    # i iteration of each c is its own case: 64 calls.  B[i,:,c] is
    # prefetched along its first dimension i, but a traversal of i (8
    # values) never leaves its first 8-double line: 0 misses; 448 hits.
    spec, ext = "abc=ai,ibc", {"a": 64, "b": 64, "c": 64, "i": 8}
    got = _counts(spec, ext, "ci-ger", 786432, 8)
    assert got == {("first", 1): 64, "miss": 0, "hit": 448}


def test_case_counts_two_first_iteration_levels():
    # bci-axpy with a=64, b=c=i=8: 8 x 8 x 8 = 512 axpy calls.  Loop c is
    # entered 8 times (> 1 % of 512 = 5.12), so its first iteration is a
    # case: once per b, 8 calls.  The innermost loop i is entered 64 times;
    # its first iterations that are not already first c iterations: 64 - 8
    # = 56.  B[i,b,c] shares lines along i (8 doubles per line, 8 values of
    # i): no miss after the first iteration.  Hits: 512 - 64 = 448.
    spec, ext = "abc=ai,ibc", {"a": 64, "b": 8, "c": 8, "i": 8}
    got = _counts(spec, ext, "bci-axpy", 786432, 8)
    assert got == {("first", 1): 8, ("first", 2): 56, "miss": 0, "hit": 448}


def test_case_counts_misses_on_a_longer_innermost_loop():
    # bci-axpy with a=64, b=c=8, i=20 and 8 doubles per line: 8 x 8 x 20 =
    # 1280 calls.  Loop c is entered 8 times, below 1 % of 1280 = 12.8, so
    # only the innermost loop i has first iterations: 64.  Each traversal
    # of i leaves a line at i = 8 and i = 16: 2 misses, 64 * 2 = 128.
    # Hits: 1280 - 64 - 128 = 1088.
    spec, ext = "abc=ai,ibc", {"a": 64, "b": 8, "c": 8, "i": 20}
    got = _counts(spec, ext, "bci-axpy", 786432, 8)
    assert got == {("first", 2): 64, "miss": 128, "hit": 1088}


def test_case_counts_without_line_sharing():
    # bc-gemv (loops b, c around gemv over a and i), a=b=c=400, i=8: the
    # innermost loop c is no operand's first dimension, and neither A's nor
    # B's nor C's second dimension with the first covered (B[:, b, c] has
    # i first, then b), so no prefetch and no miss case: 400 first
    # iterations of c, 160,000 - 400 = 159,600 hits.
    spec, ext = "abc=ai,ibc", {"a": 400, "b": 400, "c": 400, "i": 8}
    got = _counts(spec, ext, "bc-gemv", 786432, 8)
    assert got == {("first", 1): 400, "hit": 159600}


def test_first_iteration_distances_bci_axpy():
    # Section 3.5 walk for the first iteration of loop c in bci-axpy (a=64,
    # b=c=i=8; loops b, c, i; kernel axpy along a).  Starting at loop c,
    # every kernel region is already joined along c and i:
    #   A[:, i]      joined on i      -> 64 * 8          = 512
    #   B[i, b, c]   joined on i, c   -> 8 * 8           = 64
    #   C[:, b, c]   joined on c      -> 64 * 8          = 512
    # Loop b is next: A does not vary with b (walk stops: distance
    # 512 + 64 + 512 = 1088); B and C vary with b, so everything joins
    # along b too: A 512 + B 8*8*8 + C 64*8*8 = 512 + 512 + 4096 = 5120.
    spec, ext = "abc=ai,ibc", {"a": 64, "b": 8, "c": 8, "i": 8}
    alg = _alg(spec, "bci-axpy")
    _, dist = op.first_iteration_setup(spec, ext, alg, 1, 10 ** 9)
    assert dist == {"A": 1088, "B": 5120, "C": 5120}
