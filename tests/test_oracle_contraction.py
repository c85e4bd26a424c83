"""Pins for the FP64 oracle of the contraction (Section 1, "Tensor Notation").

None of these retypes the oracle's loop: each checks it against a library
routine (numpy.matmul, numpy.einsum), a closed form, an exact integer
identity or an invariant of the definition, so that a dropped term, a wrong
index, a transposed operand or a misread stride fails at least one test.
"""
import numpy as np
import pytest

from oracle import contraction as oc
from paper_1409_8608_gb300 import synth

SPECS = [
    ("abc=ai,ibc", [5, 3, 4, 7]),      # a b c i
    ("abc=iaj,jbic", [3, 4, 5, 2, 3]),  # a b c i j
    ("ab=aij,jib", [6, 5, 3, 4]),       # a b i j
    ("a=iaj,ji", [4, 3, 5]),            # a i j
    ("abc=ija,jbic", [3, 2, 4, 3, 2]),
    ("ab=ai,ib", [7, 6, 5]),
    # batch (Hadamard) indices, in A, B and C: beyond the paper's notation;
    # the definition extends with f_A and f_B sharing the batch index
    ("habc=hai,hibc", [3, 4, 3, 5, 2]),
    ("abh=aih,ibh", [4, 5, 3, 2]),
    ("hab=ha,hb", [3, 4, 5]),
    ("gha=giah,hig", [2, 3, 4, 5]),
]


def _nd(flat, modes, ext):
    """View a Fortran-contiguous flat buffer as an n-d array (first index
    fastest) for the library cross-checks."""
    shape = [ext[m] for m in modes]
    return flat.reshape(shape, order="F") if modes else flat.reshape(())


def _einsum(spec, extents, A, B):
    c, a, b = oc.parse_spec(spec)
    ext = dict(zip(oc.index_order(spec), extents))
    out = np.einsum(f"{a},{b}->{c}", _nd(A, a, ext), _nd(B, b, ext))
    return np.asarray(out).reshape(-1, order="F")


def test_matrix_product_matches_numpy_matmul():
    # C_ab = A_ai B_ib is the matrix product (Section 1, parenthetical)
    a, b, i = 37, 29, 11
    rng = np.random.default_rng(3)
    A = rng.uniform(-1, 1, a * i)
    B = rng.uniform(-1, 1, i * b)
    C = oc.contract("ab=ai,ib", [a, b, i], A, B)
    ref = A.reshape(a, i, order="F") @ B.reshape(i, b, order="F")
    np.testing.assert_allclose(C.reshape(a, b, order="F"), ref, rtol=1e-13,
                               atol=1e-13)


@pytest.mark.parametrize("spec,extents", SPECS)
def test_matches_einsum_uniform(spec, extents):
    A, B, _ = synth.uniform_operands(spec, extents, seed=11)
    C = oc.contract(spec, extents, A, B)
    np.testing.assert_allclose(C, _einsum(spec, extents, A, B), rtol=1e-12,
                               atol=1e-13)


@pytest.mark.parametrize("spec,extents", SPECS)
def test_matches_einsum_exactly_on_integers(spec, extents):
    A, B, _ = synth.integer_operands(spec, extents, seed=5)
    C = oc.contract(spec, extents, A, B)
    assert np.array_equal(C, _einsum(spec, extents, A, B))


def test_all_ones_closed_form():
    # every C entry sums prod(contracted extents) products 1*1
    spec, ext = "abc=iaj,jbic", [3, 4, 2, 5, 6]
    nc, na, nb = synth.dense_sizes(spec, ext)
    C = oc.contract(spec, ext, np.ones(na), np.ones(nb))
    assert np.all(C == 5 * 6)


def test_one_hot_operand_selects_a_slice():
    # A = e_(a0, i0): C[a,b,c] = [a == a0] * B[i0, b, c]
    spec, (a, b, c, i) = "abc=ai,ibc", (4, 3, 5, 6)
    a0, i0 = 2, 4
    A = np.zeros(a * i)
    A[a0 + a * i0] = 1.0
    _, B, _ = synth.uniform_operands(spec, [a, b, c, i], seed=2)
    C = oc.contract(spec, [a, b, c, i], A, B).reshape(a, b, c, order="F")
    Bn = B.reshape(i, b, c, order="F")
    for aa in range(a):
        expect = Bn[i0] if aa == a0 else np.zeros((b, c))
        assert np.array_equal(C[aa], expect)


def test_identity_operand_returns_the_other():
    # B = I in C_ab = A_ai B_ib gives C = A
    a, i = 6, 6
    A = np.arange(1.0, a * i + 1)
    C = oc.contract("ab=ai,ib", [a, i, i], A, np.eye(i).reshape(-1, order="F"))
    assert np.array_equal(C, A)


def test_bilinearity_exact():
    spec, ext = "abc=iaj,jbic", [3, 5, 2, 4, 3]
    A1, B, _ = synth.integer_operands(spec, ext, seed=1)
    A2, B2, _ = synth.integer_operands(spec, ext, seed=2)
    lhs = oc.contract(spec, ext, A1 + A2, B - 2 * B2)
    rhs = (oc.contract(spec, ext, A1, B) + oc.contract(spec, ext, A2, B)
           - 2 * oc.contract(spec, ext, A1, B2)
           - 2 * oc.contract(spec, ext, A2, B2))
    assert np.array_equal(lhs, rhs)


def test_summed_output_equals_contraction_of_summed_operands():
    # sum_abc C = sum_i (sum_a A[a,i]) (sum_bc B[i,b,c])
    spec, (a, b, c, i) = "abc=ai,ibc", (5, 4, 3, 6)
    A, B, _ = synth.integer_operands(spec, [a, b, c, i], seed=9)
    C = oc.contract(spec, [a, b, c, i], A, B)
    sa = A.reshape(a, i, order="F").sum(axis=0)
    sb = B.reshape(i, b * c, order="F").sum(axis=1)
    assert C.sum() == float(np.dot(sa, sb))


def test_swapping_the_inputs():
    # C_abc = A_ai B_ibc written as C_abc = B_ibc A_ai
    ext = [4, 3, 5, 6]
    A, B, _ = synth.uniform_operands("abc=ai,ibc", ext, seed=4)
    C1 = oc.contract("abc=ai,ibc", ext, A, B)
    C2 = oc.contract("abc=ibc,ai", ext, B, A)
    np.testing.assert_array_equal(C1, C2)


def test_index_relabelling():
    ext = [4, 3, 5, 6]
    A, B, _ = synth.uniform_operands("abc=ai,ibc", ext, seed=4)
    C1 = oc.contract("abc=ai,ibc", ext, A, B)
    C2 = oc.contract("xyz=xk,kyz", ext, A, B)
    np.testing.assert_array_equal(C1, C2)


def test_strided_storage_gives_the_same_values():
    # store B (i,b,c) padded and with its modes permuted in memory
    spec, ext = "abc=ai,ibc", [4, 3, 5, 6]
    a, b, c, i = ext
    A, B, _ = synth.uniform_operands(spec, ext, seed=6)
    ref = oc.contract(spec, ext, A, B)
    Bn = B.reshape(i, b, c, order="F")
    # physical layout (c, i, b) with padding: strides i:1*(c+1), b:(c+1)*(i+2), c:1
    phys = np.zeros(((c + 1) * (i + 2) * b,))
    s_c, s_i, s_b = 1, c + 1, (c + 1) * (i + 2)
    for ii in range(i):
        for bb in range(b):
            for cc in range(c):
                phys[ii * s_i + bb * s_b + cc * s_c] = Bn[ii, bb, cc]
    # C stored with padded leading dimension
    sC = [1, a + 3, (a + 3) * b]
    strides = sC + [1, a] + [s_i, s_b, s_c]
    Cbuf = np.full(1 + (a - 1) + (b - 1) * sC[1] + (c - 1) * sC[2], np.nan)
    oc.contract(spec, ext, A, phys, C=Cbuf, beta=0.0, strides=strides)
    got = np.array([Cbuf[x + y * sC[1] + z * sC[2]]
                    for z in range(c) for y in range(b) for x in range(a)])
    np.testing.assert_array_equal(got, ref)


def test_alpha_beta_and_nan_safe_beta_zero():
    spec, ext = "abc=ai,ibc", [3, 4, 2, 5]
    A, B, C0 = synth.integer_operands(spec, ext, seed=8, with_c=True)
    S = oc.contract(spec, ext, A, B)
    C = C0.copy()
    oc.contract(spec, ext, A, B, C=C, alpha=3.0, beta=-2.0)
    assert np.array_equal(C, 3.0 * S - 2.0 * C0)
    C = np.full_like(C0, np.nan)
    oc.contract(spec, ext, A, B, C=C, alpha=1.0, beta=0.0)
    assert np.array_equal(C, S)


def test_slab_and_points_agree_with_the_full_result():
    spec, ext = "abc=iaj,jbic", [5, 4, 6, 3, 2]
    A, B, _ = synth.uniform_operands(spec, ext, seed=12)
    full = oc.contract(spec, ext, A, B, threads=2)
    slab = np.zeros_like(full)
    oc.contract(spec, ext, A, B, C=slab, outer_range=(2, 4))
    a, b, c = ext[:3]
    f3 = full.reshape(a, b, c, order="F")
    s3 = slab.reshape(a, b, c, order="F")
    assert np.array_equal(s3[:, :, 2:4], f3[:, :, 2:4])
    assert np.all(s3[:, :, :2] == 0) and np.all(s3[:, :, 4:] == 0)
    rng = np.random.default_rng(0)
    pts = np.stack([rng.integers(0, e, 20) for e in (a, b, c)], axis=1)
    vals = oc.contract_points(spec, ext, A, B, pts)
    assert np.array_equal(vals, f3[pts[:, 0], pts[:, 1], pts[:, 2]])


def test_extent_one_reduces_to_matrix_product():
    # abc=ai,ibc with c = 1 is the plain product A (a x i) times B (i x b)
    a, b, i = 9, 7, 5
    A, B, _ = synth.uniform_operands("abc=ai,ibc", [a, b, 1, i], seed=13)
    C = oc.contract("abc=ai,ibc", [a, b, 1, i], A, B)
    ref = A.reshape(a, i, order="F") @ B.reshape(i, b, order="F")
    np.testing.assert_allclose(C.reshape(a, b, order="F"), ref, rtol=1e-13,
                               atol=1e-14)


def test_scalar_output():
    # C = sum_i A_i B_i is the dot product
    A = np.arange(1.0, 8.0)
    B = np.arange(2.0, 9.0)
    C = oc.contract("=i,i", [7], A, B)
    assert C.shape == (1,) and C[0] == float(np.dot(A, B))


def test_batch_index_is_a_loop_of_matrix_products():
    # C[:,:,h] = A[:,:,h] @ B[:,:,h] for every h (brute force over the
    # batch index with numpy.matmul), and the Hadamard case C[h,a,b] =
    # A[h,a] * B[h,b] with no contracted index
    a, i, b, h = 9, 7, 8, 5
    rng = np.random.default_rng(13)
    A = rng.uniform(-1, 1, a * i * h)
    B = rng.uniform(-1, 1, i * b * h)
    C = oc.contract("abh=aih,ibh", [a, b, h, i], A, B).reshape(a, b, h, order="F")
    A3, B3 = A.reshape(a, i, h, order="F"), B.reshape(i, b, h, order="F")
    for x in range(h):
        np.testing.assert_allclose(C[:, :, x], A3[:, :, x] @ B3[:, :, x], rtol=1e-13, atol=1e-13)
    Ah, Bh = rng.integers(-8, 9, h * a).astype(float), rng.integers(-8, 9, h * b).astype(float)
    Ch = oc.contract("hab=ha,hb", [h, a, b], Ah, Bh).reshape(h, a, b, order="F")
    want = Ah.reshape(h, a, order="F")[:, :, None] * Bh.reshape(h, b, order="F")[:, None, :]
    assert np.array_equal(Ch, want)
