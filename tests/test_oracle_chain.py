"""Pins of the chain oracle (oracle/chain.py): the direct sum over the
whole index space, checked against values that do not come from it."""
import numpy as np
import pytest

from oracle import chain as och
from oracle import contraction as oc


def rand(n, seed):
    return np.random.default_rng(seed).uniform(-1, 1, n)


def test_matrix_chain_against_matmul():
    # D = X Y Z for matrices: numpy's matrix product (a library routine the
    # oracle does not use)
    a, b, c, d = 5, 7, 3, 6
    X, Y, Z = rand(a * b, 1), rand(b * c, 2), rand(c * d, 3)
    got = och.contract3("ad=ab,bc,cd", [a, d, b, c], X, Y, Z)
    Xm, Ym, Zm = (v.reshape(s, order="F") for v, s in ((X, (a, b)), (Y, (b, c)), (Z, (c, d))))
    want = (Xm @ Ym @ Zm).reshape(-1, order="F")
    assert np.allclose(got, want, rtol=1e-13, atol=1e-13)


def test_brute_force_loops():
    # every entry as an explicit triple loop on a tiny case with an index
    # in all three operands (i) and an index in two inputs (j)
    spec, ext = "ab=ai,ij,jbi", [3, 2, 4, 2]  # a, b, i, j
    a, b, i, j = ext
    X, Y, Z = rand(a * i, 4), rand(i * j, 5), rand(j * b * i, 6)
    got = och.contract3(spec, ext, X, Y, Z).reshape((a, b), order="F")
    Xa = X.reshape((a, i), order="F")
    Ya = Y.reshape((i, j), order="F")
    Za = Z.reshape((j, b, i), order="F")
    for aa in range(a):
        for bb in range(b):
            s = 0.0
            for ii in range(i):
                for jj in range(j):
                    s += Xa[aa, ii] * Ya[ii, jj] * Za[jj, bb, ii]
            assert abs(got[aa, bb] - s) <= 1e-14 * (1 + abs(s))


def test_every_pairwise_order_agrees():
    # associativity: each order of two pairwise contractions (the separately
    # pinned FP64 pairwise oracle) gives the direct sum
    spec, ext = "abc=ai,ij,jbc", [4, 3, 5, 6, 2]  # a, b, c, i, j
    a, b, c, i, j = ext
    X, Y, Z = rand(a * i, 7), rand(i * j, 8), rand(j * b * c, 9)
    direct = och.contract3(spec, ext, X, Y, Z)
    T1 = oc.contract("aj=ai,ij", [a, j, i], X, Y)              # (X Y) first
    via1 = oc.contract("abc=aj,jbc", [a, b, c, j], T1, Z)
    T2 = oc.contract("ibc=ij,jbc", [i, b, c, j], Y, Z)         # (Y Z) first
    via2 = oc.contract("abc=ai,ibc", [a, b, c, i], X, T2)
    for v in (via1, via2):
        assert np.allclose(v, direct, rtol=1e-12, atol=1e-13)


def test_closed_forms():
    # all-ones operands: every entry is the product of the summed extents
    spec, ext = "ab=aij,jk,kib", [3, 4, 2, 5, 6]  # a, b, i, j, k
    sizes = och.chain_sizes(spec, ext)
    got = och.contract3(spec, ext, *(np.ones(n) for n in sizes[1:]))
    assert np.all(got == 2 * 5 * 6)
    # identity in the middle: X I Z = X Z
    a, n, d = 4, 5, 3
    X, Z = rand(a * n, 10), rand(n * d, 11)
    got = och.contract3("ad=ab,bc,cd", [a, d, n, n], X, np.eye(n).reshape(-1), Z)
    want = (X.reshape((a, n), order="F") @ Z.reshape((n, d), order="F")).reshape(-1, order="F")
    assert np.allclose(got, want, rtol=1e-13, atol=1e-13)


def test_rejects_an_index_summed_within_one_operand():
    with pytest.raises(ValueError):
        och.contract3("ad=abe,bc,cd", [2, 2, 2, 2, 2], np.ones(8), np.ones(4), np.ones(4))


def test_chain_flops_classic_order_choice():
    # X: 512 x 8, Y: 8 x 512, Z: 512 x 8: (Y Z) first costs 64x fewer flops
    spec, ext = "ad=ab,bc,cd", [512, 8, 8, 512]  # a, d, b, c
    xy = och.chain_flops(spec, ext, (0, 1))
    yz = och.chain_flops(spec, ext, (1, 2))
    assert xy == 2 * 512 * 8 * 512 + 2 * 512 * 512 * 8
    assert yz == 2 * 8 * 512 * 8 + 2 * 512 * 8 * 8
    assert xy == 64 * yz
