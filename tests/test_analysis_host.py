"""The library's cache analysis (Section 3) against the oracle's and the
paper's worked example (integer work, no GPU)."""
import json
import os

import pytest

import __graft_entry__
from oracle import algorithms as oa
from oracle import prediction as op
from paper_1409_8608_gb300 import tc


@pytest.fixture(scope="module")
def lib():
    __graft_entry__.build_library()
    return tc.load()


def _as_lists(setup):
    return [list(x) for x in setup]


def test_worked_example(lib, golden_dir):
    with open(os.path.join(golden_dir, "worked_example_ca_gemv.json")) as f:
        ex = json.load(f)
    ext = [ex["extents"][k] for k in "abci"]
    plan = tc.Plan(ex["spec"], ext)
    alg = next(a for a in plan.algorithms() if a["name"] == ex["algorithm"])
    dist = tc.tc_access_distances(plan.handle, alg["id"], 0, 1)
    for name, want in ex["operands"].items():
        assert dist[name] == want["distance"], name
    cases = tc.tc_prediction_cases(plan.handle, alg["id"], 0, 1, ex["cache_elems"], ex["line_elems"])
    assert [c["kind"] for c in cases] == ["steady", "miss", "first"]
    hit = tc.tc_setup_list(plan.handle, alg["id"], 0, 0, 1, ex["cache_elems"], ex["line_elems"])
    miss = tc.tc_setup_list(plan.handle, alg["id"], 1, 0, 1, ex["cache_elems"], ex["line_elems"])
    assert _as_lists(hit) == ex["setup_prefetch"] and cases[0]["omit"] == ex["setup_prefetch_omitted"]
    assert _as_lists(miss) == ex["setup_prefetch_failure"]
    plan.close()


def _oracle_cases(spec, ext, alg, cache, line):
    hit, miss, plain, kinds = op.steady_setups(spec, ext, alg, cache, line)
    counts = op.case_counts(alg, ext, line, miss is not None)
    out = [("steady", -1, counts["hit"], hit)]
    if miss is not None:
        out.append(("miss", -1, counts["miss"], miss))
    for d in op.first_iteration_loops(alg, ext):
        setup, _ = op.first_iteration_setup(spec, ext, alg, d, cache)
        out.append(("first", d, counts[("first", d)], setup))
    if not alg["loops"]:
        out = [("steady", -1, 1, hit)]
    return out


@pytest.mark.parametrize("spec,extents,cache,line", [
    ("abc=ai,ibc", [400, 400, 400, 8], 786432, 8),
    ("abc=ai,ibc", [64, 48, 32, 8], 20000, 8),
    ("abc=iaj,jbic", [24, 20, 16, 16, 16], 50000, 16),
    ("a=iaj,ji", [100, 30, 50], 4096, 8),
    ("ab=aij,jib", [40, 30, 8, 6], 3000, 4),
    ("habc=hai,hibc", [6, 40, 30, 20, 8], 20000, 8),   # a batch index, always a loop
])
def test_every_case_matches_oracle(lib, spec, extents, cache, line):
    plan = tc.Plan(spec, extents)
    order = [x for x in dict.fromkeys(spec.replace("=", "").replace(",", ""))]
    ext = dict(zip(order, extents))
    for alg in oa.enumerate_algorithms(spec, extents):
        aid = alg["id"] + 1
        want = _oracle_cases(spec, ext, alg, cache, line)
        got = tc.tc_prediction_cases(plan.handle, aid, 0, 1, cache, line)
        assert [(c["kind"], c["depth"], c["count"]) for c in got] == [w[:3] for w in want], alg["name"]
        for k, w in enumerate(want):
            lst = tc.tc_setup_list(plan.handle, aid, k, 0, 1, cache, line)
            assert _as_lists(lst) == [list(x) for x in w[3]], (alg["name"], k)
        dist = tc.tc_access_distances(plan.handle, aid, 0, 1)
        for name in "ABC":
            assert dist[name] == op.access_distance(spec, ext, alg, name)[0]
    plan.close()


def test_device_granularity_is_the_phase_nest(lib):
    # granularity 1 analyses the device phases: the contracted loops that
    # enclose a free loop, around one phase launch whose operand slices
    # span every other index; same walk, byte units
    spec, extents = "abc=iaj,jbic", [64, 64, 64, 16, 16]
    ext = dict(zip("abcij", extents))
    plan = tc.Plan(spec, extents)
    for alg in oa.enumerate_algorithms(spec, extents):
        loops = list(alg["loops"])
        q = -1
        for pos, l in enumerate(loops):
            if l in "ij" and any(x in "abc" for x in loops[pos + 1:]):
                q = pos
        phase = [l for pos, l in enumerate(loops) if pos <= q and l in "ij"]
        pseudo = {"loops": tuple(phase), "kernel_indices": tuple(x for x in "abcij" if x not in phase)}
        got = tc.tc_access_distances(plan.handle, alg["id"] + 1, 1, 8)
        for name in "ABC":
            assert got[name] == 8 * op.access_distance(spec, ext, pseudo, name)[0], alg["name"]
        cases = tc.tc_prediction_cases(plan.handle, alg["id"] + 1, 1, 8, 126 << 20, 128)
        nph = 1
        for l in phase:
            nph *= ext[l]
        assert sum(c["count"] for c in cases) == nph
    plan.close()
