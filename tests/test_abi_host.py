"""Host-side checks of the C ABI (no GPU): the library loads and exports
every declared entry point, the planner rejects malformed input, and its
algorithm generator agrees exactly with the oracle's (integer work)."""
import ctypes

import pytest

import __graft_entry__
from oracle import algorithms as oa
from paper_1409_8608_gb300 import tc
from tests.abi_util import declared_functions


@pytest.fixture(scope="module")
def lib():
    __graft_entry__.build_library()
    return tc.load()


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert "tc_execute" in names and "tc_plan_create" in names
    for name in names:
        assert hasattr(lib, name), name


def test_binding_covers_the_header(lib):
    for name in declared_functions():
        assert name in tc.SIGNATURES or hasattr(tc, name), name


@pytest.mark.parametrize("spec,extents", [
    ("abc=ai,ibc", [8, 9, 10, 4]),
    ("abc=iaj,jbic", [6, 5, 4, 3, 2]),
    ("abc=ija,jbic", [6, 5, 4, 3, 2]),
    ("ab=aij,jib", [7, 6, 3, 2]),
    ("a=iaj,ji", [5, 4, 3]),
    ("ab=ai,ib", [3, 4, 5]),
    ("abcd=iabj,jcid", [2, 3, 4, 5, 2, 3]),
    # batch (Hadamard) indices: in A, B and C, always sliced loops
    ("habc=hai,hibc", [3, 6, 5, 4, 2]),
    ("abh=aih,ibh", [4, 5, 3, 2]),
    ("hab=ha,hb", [3, 4, 5]),
    ("gha=giah,hig", [2, 3, 4, 5]),
])
def test_enumeration_matches_oracle(lib, spec, extents):
    plan = tc.Plan(spec, extents)
    got = plan.algorithms()
    want = oa.enumerate_algorithms(spec, extents)
    assert got[0]["name"] == "gett" and got[0]["kernel"] == "gett"
    assert len(got) == len(want) + 1
    for g, w in zip(got[1:], want):
        assert g["id"] == w["id"] + 1
        assert g["name"] == w["name"]
        assert g["kernel"] == w["kernel"]
        assert g["loops"] == w["loops"]
        assert g["kernel_indices"] == w["kernel_indices"]
        lv = {op: g["copy_level"][k] for k, op in enumerate("ABC") if g["copy_level"][k] != -2}
        assert lv == w["copies"], g["name"]
    plan.close()


def test_strided_copy_decision_matches_oracle(lib):
    strides = [1, 4, 2, 8, 1, 3]
    plan = tc.Plan("ab=ai,ib", [4, 5, 3], strides=strides)
    got = plan.algorithms()
    want = oa.enumerate_algorithms("ab=ai,ib", [4, 5, 3], strides=strides)
    assert [g["name"] for g in got[1:]] == [w["name"] for w in want]
    plan.close()


def test_phase_counts(lib):
    plan = tc.Plan("abc=iaj,jbic", [64, 64, 64, 16, 16])
    algs = {a["name"]: a for a in plan.algorithms()}
    # i'c-gemm: the copy loop i encloses the free loop c -> 16 phases
    assert algs["i'c-gemm"]["n_phases"] == 16
    # ci'-gemm: the contracted loop is innermost -> one phase
    assert algs["ci'-gemm"]["n_phases"] == 1
    assert algs["gett"]["n_phases"] == 1
    plan.close()


@pytest.mark.parametrize("spec,extents,strides,status", [
    ("abc", [1, 2, 3], None, "TC_ERROR_INVALID_SPEC"),
    ("abc=ai,ibc,x", [1, 2, 3, 4], None, "TC_ERROR_INVALID_SPEC"),
    ("ab=aik,ib", [2, 2, 2, 2], None, "TC_ERROR_INVALID_SPEC"),       # k in A only
    ("ab=aai,ib", [2, 2, 2], None, "TC_ERROR_INVALID_SPEC"),          # repeated index
    ("aB=ai,iB", [2, 2, 2], None, "TC_ERROR_INVALID_SPEC"),           # not a-z
    ("ab=ai,ib", [2, 0, 2], None, "TC_ERROR_INVALID_EXTENT"),
    ("ab=ai,ib", [2, 3, 2], [1, 1, 1, 2, 1, 2], "TC_ERROR_INVALID_STRIDE"),  # C overlaps
    ("ab=ai,ib", [2, 3, 2], [1, 2, 0, 2, 1, 2], "TC_ERROR_INVALID_STRIDE"),  # zero stride
])
def test_rejections(lib, spec, extents, strides, status):
    with pytest.raises(tc.TcError) as e:
        tc.tc_plan_create(spec, extents, strides)
    assert tc.STATUS_NAMES[e.value.status] == status


def test_status_strings_and_null_arguments(lib):
    for code in tc.STATUS_NAMES:
        assert tc.tc_status_string(code)
    assert lib.tc_plan_destroy(None) == 0
    assert lib.tc_plan_select(None, 0) == 9
    plan = tc.Plan("abc=ai,ibc", [4, 4, 4, 2])
    with pytest.raises(tc.TcError):
        plan.select(999)
    # NULL operands are rejected before any device work
    a = ctypes.c_double(1.0)
    st = lib.tc_execute(plan.handle, ctypes.addressof(a), None, None, ctypes.addressof(a), None, None)
    assert st == 9
    plan.close()


def test_flops_and_workspace(lib):
    plan = tc.Plan("abc=iaj,jbic", [8, 8, 8, 4, 4])
    assert plan.flops == 2 * 8 * 8 * 8 * 4 * 4
    algs = {a["name"]: a["id"] for a in plan.algorithms()}
    assert plan.workspace(algs["cab" + "j-dot"] if "cabj-dot" in algs else 1) == 0
    # i'c-gemm copies A[i,:,:] (a x j doubles) once per phase
    assert plan.workspace(algs["i'c-gemm"]) == ((8 * 4 * 8 + 255) // 256) * 256
    plan.close()


def test_plan_option_validation(lib):
    plan = tc.Plan("ab=aij,jib", [8, 8, 4, 4], dtype="bf16x3")
    for chunk in (-1, 0, 32, 256, 4096):
        plan.set_compensation(chunk)
    for chunk in (-2, 16, 100):
        with pytest.raises(tc.TcError) as e:
            plan.set_compensation(chunk)
        assert tc.STATUS_NAMES[e.value.status] == "TC_ERROR_INVALID_ARGUMENT"
    for width in (0, 128, 256):
        plan.set_gett_tile(width)
    with pytest.raises(tc.TcError):
        plan.set_gett_tile(64)
    with pytest.raises(tc.TcError):
        plan.set_gett_tma(2)
    for mode in (0, 1, 2, 3):
        plan.set_gett_pack(mode)
    for mode in (-1, 4):
        with pytest.raises(tc.TcError) as e:
            plan.set_gett_pack(mode)
        assert tc.STATUS_NAMES[e.value.status] == "TC_ERROR_INVALID_ARGUMENT"
    plan.close()


def test_selftest_rejects_bad_limits(lib):
    for limit in (0, -5, 20_000_000_000):
        st = tc.tc_selftest_bounded_wait(limit, 0)
        assert tc.STATUS_NAMES[st] == "TC_ERROR_INVALID_ARGUMENT"


def test_gett_pack_choice(lib):
    # automatic pre-conversion only where the inputs are contiguous along
    # different contracted indices and one is much smaller; mode 2 forces
    # it for the FP32-input tensor forms, mode 0 turns it off
    cases = [("abc=iaj,jbic", [512, 512, 512, 16, 16], True),
             ("abc=ai,ibc", [512, 512, 512, 64], False),
             ("ab=aij,jib", [256, 256, 16, 16], False),
             ("abc=iaj,jbic", [512, 512, 4, 16, 16], False)]   # A not 8x smaller
    for spec, ext, auto in cases:
        for dtype in ("bf16x3", "tf32", "bf16", "f32"):
            plan = tc.Plan(spec, ext, dtype=dtype)
            float_in = dtype in ("bf16x3", "tf32")
            assert (plan.workspace(0) > 0) == (auto and float_in), (spec, ext, dtype)
            plan.set_gett_pack(2)
            assert (plan.workspace(0) > 0) == float_in, (spec, ext, dtype)
            plan.set_gett_pack(0)
            assert plan.workspace(0) == 0
            plan.close()


def test_gett_pack_both_choice(lib):
    # both inputs pre-converted: by default for the compensated split forms
    # (K past the 256-element chunk) and wherever M and N are both at least
    # 1024; mode 3 on request.  The workspace then holds both inputs' images
    # (6 / 8 / 4 / 2 / 1 bytes per element for split-BF16 / 3xTF32 / TF32 /
    # BF16 and FP16 / E4M3, rows and K rounded up to whole tiles and stages)
    img = {"bf16x3": 6, "tf32x3": 8, "tf32": 4, "bf16": 2, "f16": 2, "e4m3": 1}

    def both(ws, M, N, K, b):  # within the documented bound, at least the exact images
        return b * (M + N) * K <= ws <= b * (M + N + 512) * (K + 31) + 256

    # the compensated form (K = 288 > 256): both inputs, whatever the sizes
    for dtype in ("bf16x3", "tf32x3"):
        plan = tc.Plan("ab=aij,jib", [300, 40, 24, 12], dtype=dtype)
        assert both(plan.workspace(0), 300, 40, 288, img[dtype]), dtype
        plan.set_compensation(0)  # no compensation: one small input at most
        assert plan.workspace(0) < img[dtype] * (300 + 40) * 288, dtype
        plan.close()
    # M and N of 1024 and more: every tensor form with FP32, 16-bit or E4M3 inputs
    for dtype in img:
        plan = tc.Plan("ab=aij,jib", [1024, 1536, 8, 8], dtype=dtype)
        assert both(plan.workspace(0), 1024, 1536, 64, img[dtype]), dtype
        plan.set_gett_pack(0)
        assert plan.workspace(0) == 0, dtype
        plan.close()
        plan = tc.Plan("ab=aij,jib", [512, 1536, 8, 8], dtype=dtype)  # M below 1024
        assert plan.workspace(0) < img[dtype] * (512 + 1536) * 64, dtype
        plan.set_gett_pack(3)  # on request
        assert both(plan.workspace(0), 512, 1536, 64, img[dtype]), dtype
        plan.close()
    # FP64 / FP32 run the SIMT GETT: nothing to pre-convert
    for dtype in ("f64", "f32"):
        plan = tc.Plan("ab=aij,jib", [1024, 1536, 8, 8], dtype=dtype)
        plan.set_gett_pack(3)
        assert plan.workspace(0) == 0
        plan.close()


def test_batch_indices_are_accepted_and_never_kernel_indices(lib):
    # an index in A, B and C is a batch index: the plan accepts it, and in
    # every algorithm it is one of the sliced loops, never a kernel index
    plan = tc.Plan("habc=hai,hibc", [3, 6, 5, 4, 2])
    algs = plan.algorithms()
    assert len(algs) == 1 + 130  # 24 dot + 72 axpy + 18 gemv + 12 ger + 4 gemm
    for a in algs[1:]:
        assert "h" in a["loops"] and "h" not in a["kernel_indices"], a["name"]
    plan.close()
