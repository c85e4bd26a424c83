"""Pins for the oracle's algorithm generator (Section 2 and Table 1) against
the counts, names, plot numbering and listings the paper prints."""
import json
import os

import pytest

from oracle import algorithms as oa
from oracle.contraction import index_order


def _golden(golden_dir):
    with open(os.path.join(golden_dir, "paper_algorithms.json")) as f:
        return json.load(f)["contractions"]


@pytest.fixture(scope="module")
def golden(golden_dir):
    return _golden(golden_dir)


def test_counts_per_kernel(golden):
    for entry in golden:
        algs = oa.enumerate_algorithms(entry["spec"])
        assert oa.count_by_kernel(algs) == entry["counts"], entry["spec"]
        assert len(algs) == sum(entry["counts"].values())


def test_plot_numbering(golden):
    for entry in golden:
        algs = oa.enumerate_algorithms(entry["spec"])
        for k, name in entry["numbered"].items():
            assert algs[int(k)]["name"] == name, (entry["spec"], k)


def test_listings(golden):
    for entry in golden:
        algs = {a["name"]: a for a in oa.enumerate_algorithms(entry["spec"])}
        for lst in entry["listings"]:
            alg = algs[lst["name"]]
            assert sorted(alg["kernel_indices"]) == sorted(lst["kernel_indices"])
            assert list(alg["loops"]) == lst["loops"]
            for op in ("A", "B", "C"):
                assert alg["slice_modes"][op] == lst["slices"][op], (lst["name"], op)
            assert alg["copies"] == lst.get("copy", {}), lst["name"]


def test_copy_totals():
    # Section 4.3: every gemm algorithm of Test 3 copies; Section 4.2: only
    # i'-gemv copies; the case study needs no copy at all.
    t3 = oa.enumerate_algorithms("abc=ija,jbic")
    assert all(a["copies"] for a in t3 if a["kernel"] == "gemm")
    t2 = oa.enumerate_algorithms("a=iaj,ji")
    assert [a["name"] for a in t2 if a["copies"]] == ["i'-gemv"]
    assert not any(a["copies"] for a in oa.enumerate_algorithms("abc=ai,ibc"))


def test_permuted_test3_layout_keeps_counts_and_copies():
    # the same contraction with A stored as (i, a, j): 176 algorithms, every
    # gemm algorithm and half of the gemv algorithms copy
    algs = oa.enumerate_algorithms("abc=iaj,jbic")
    assert len(algs) == 176
    assert sum(1 for a in algs if a["kernel"] == "gemm" and a["copies"]) == 8
    assert sum(1 for a in algs if a["kernel"] == "gemv" and a["copies"]) == 18


def test_every_algorithm_is_a_partition_of_the_indices():
    for spec in ("abc=ai,ibc", "abc=iaj,jbic", "ab=aij,jib", "a=iaj,ji"):
        order = index_order(spec)
        names = set()
        for alg in oa.enumerate_algorithms(spec):
            assert sorted(alg["loops"] + alg["kernel_indices"]) == sorted(order)
            names.add(alg["name"])
        assert len(names) == len(oa.enumerate_algorithms(spec))


def test_strides_decide_copies():
    # C_ab = A_ai B_ib with A stored i-fastest but padded so that neither
    # mode of A has unit stride: the gemm must copy A, before every loop
    algs = oa.enumerate_algorithms("ab=ai,ib", [4, 5, 3],
                                   strides=[1, 4, 2, 8, 1, 3])
    gemm = [a for a in algs if a["kernel"] == "gemm"]
    assert len(gemm) == 1 and gemm[0]["copies"] == {"A": -1}
    assert gemm[0]["name"] == "'-gemm"


@pytest.mark.parametrize("spec", ["habc=hai,hibc", "abh=aih,ibh", "hab=ha,hb", "gha=giah,hig"])
def test_batch_indices_counts_and_roles(spec):
    # Table 1 read with batch indices (in A, B and C; beyond the paper's
    # notation): they fit no kernel role, so they are sliced in every
    # algorithm.  Per kernel the count is then (kernel-index choices) x
    # (number of sliced indices)!, written out here from the role counts of
    # Table 1, not from the generator.
    import math
    c, a, b = (s for s in spec.replace(" ", "").replace("=", ",").split(","))
    order = index_order(spec)
    n = len(order)
    K = [x for x in order if x in a and x in b and x not in c]
    FA = [x for x in order if x in a and x in c and x not in b]
    FB = [x for x in order if x in b and x in c and x not in a]
    H = [x for x in order if x in a and x in b and x in c]
    assert H
    f = math.factorial
    want = {"dot": len(K) * f(n - 1), "axpy": (len(FA) + len(FB)) * f(n - 1),
            "gemv": (len(FA) + len(FB)) * len(K) * f(n - 2) if n >= 2 else 0,
            "ger": len(FA) * len(FB) * f(n - 2) if n >= 2 else 0,
            "gemm": len(FA) * len(FB) * len(K) * f(n - 3) if n >= 3 else 0}
    algs = oa.enumerate_algorithms(spec)
    assert oa.count_by_kernel(algs) == want
    for alg in algs:
        assert set(H) <= set(alg["loops"]) and not set(H) & set(alg["kernel_indices"]), alg["name"]
