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
