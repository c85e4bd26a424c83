"""CTA pairs (tcgen05.mma.cta_group::2) and split accumulators in the
tensor-core GETT, against the single-CTA kernel and the FP64 oracle.

A pair computes every C element from the same slice products in the same
K order as one CTA does, so pair on and off must give the same bits (with
the same accumulator setting).  Split accumulators change the rounding:
those results are checked against the oracle -- exactly on integer inputs
(every partial sum is exact in FP32), and within the bounds of the other
GETT tests on uniform inputs.  Shapes cover every way a pair tile can be
ragged: M not a multiple of 256 (the second CTA partly or wholly past M),
N not a multiple of 256, the smaller input pre-converted (A, or B), and
both inputs staged by TMA."""
import numpy as np
import pytest

from oracle import contraction as oc
from paper_1409_8608_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

U32 = 2.0 ** -24


@pytest.fixture(scope="module")
def tcmod():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build_library()
    from paper_1409_8608_gb300 import tc
    tc.load()
    return tc


def ksize(spec, ext):
    c, a, b = oc.parse_spec(spec)
    e = dict(zip(oc.index_order(spec), ext))
    k = 1
    for x in a:
        if x in b and x not in c:
            k *= e[x]
    return k


def run(tc, spec, ext, dtype, dA, dB, pair, split, pack=None, C0=None, alpha=1.0, beta=0.0):
    plan = tc.Plan(spec, ext, dtype=dtype)
    plan.set_gett_pair(pair)
    if dtype == "bf16x3":
        plan.set_split_accumulators(split)
    if pack is not None:
        plan.set_gett_pack(pack)
    plan.select(0)
    n = synth.dense_sizes(spec, ext)[0]
    dC = torch.full((n,), float("nan"), dtype=torch.float32, device="cuda:0") if C0 is None else \
        torch.from_numpy(C0).float().to("cuda:0")
    plan.execute(dA, dB, dC, alpha=alpha, beta=beta)
    torch.cuda.synchronize()
    plan.device_status()
    plan.close()
    return dC.double().cpu().numpy()


PAIR_CASES = [
    ("abc=iaj,jbic", [512, 256, 4, 16, 16], None),   # the benchmark layout: A pre-converted
    ("abc=iaj,jbic", [300, 256, 3, 16, 16], None),   # M = 300: the last pair's second CTA partly past M
    ("abc=iaj,jbic", [136, 128, 5, 16, 16], None),   # M = 136: one pair tile, second CTA 8 rows
    ("abc=ai,ibc", [512, 256, 5, 64], None),         # both inputs staged by TMA
    ("abc=ai,ibc", [384, 200, 3, 32], None),         # N = 600: ragged last tile
    ("ab=aij,jib", [256, 512, 16, 16], None),        # M-contiguous A, K-contiguous B
    ("abc=iaj,jbic", [512, 256, 4, 16, 16], 2),      # pre-conversion forced (A)
    ("abc=iaj,jbic", [520, 128, 3, 16, 16], None),   # M = 520: a pair tile with 8 + 0 rows
]


@pytest.mark.parametrize("dtype", ["bf16x3", "tf32"])
@pytest.mark.parametrize("spec,ext,pack", PAIR_CASES)
def test_pair_matches_single_cta_bitwise(tcmod, spec, ext, pack, dtype):
    A, B, _ = synth.uniform_operands(spec, ext, seed=21)
    dA = torch.from_numpy(A).float().cuda()
    dB = torch.from_numpy(B).float().cuda()
    for split in ((1, 0) if dtype == "bf16x3" else (0,)):
        one = run(tcmod, spec, ext, dtype, dA, dB, pair=0, split=split, pack=pack)
        two = run(tcmod, spec, ext, dtype, dA, dB, pair=1, split=split, pack=pack)
        assert np.isfinite(two).all()
        assert np.array_equal(one, two), (split, float(np.nanmax(np.abs(one - two))))
    # and within the bound against the oracle (the FP32 values as given)
    Ar, Br = A.astype(np.float32).astype(np.float64), B.astype(np.float32).astype(np.float64)
    want = oc.contract(spec, ext, Ar, Br)
    scale = oc.contract(spec, ext, np.abs(Ar), np.abs(Br))
    K = ksize(spec, ext)
    if dtype == "bf16x3":
        bound = (6 * K + 4) * U32
    else:  # TF32 products of inputs rounded to 10 mantissa bits, FP32 sums
        bound = 2 * 2.0 ** -11 + (K + 1) * U32
    err = float(np.max(np.abs(two - want) / scale))
    assert err <= bound, err


@pytest.mark.parametrize("split", [0, 1])
@pytest.mark.parametrize("spec,ext", [("abc=iaj,jbic", [300, 256, 3, 16, 16]), ("abc=ai,ibc", [384, 200, 3, 32])])
def test_pair_and_split_exact_on_integers(tcmod, spec, ext, split):
    A, B, C0 = synth.integer_operands(spec, ext, seed=22, with_c=True)
    dA = torch.from_numpy(A).float().cuda()
    dB = torch.from_numpy(B).float().cuda()
    got = run(tcmod, spec, ext, "bf16x3", dA, dB, pair=1, split=split, C0=C0, alpha=2.0, beta=-1.0)
    want = 2.0 * oc.contract(spec, ext, A, B) - C0
    assert np.array_equal(got, want)


@pytest.mark.parametrize("pair", [0, 1])
def test_split_accumulators_cut_the_rounding(tcmod, pair):
    # lognormal per-slice scales on the benchmark layout (a reduced c): the
    # split accumulators must meet the FP32-level target, and not be worse
    # than one accumulator
    spec, ext = "abc=iaj,jbic", [512, 512, 8, 16, 16]
    A, B, _ = synth.lognormal_slice_operands(spec, ext, seed=1)
    dA = torch.from_numpy(A).float().cuda()
    dB = torch.from_numpy(B).float().cuda()
    Ar, Br = A.astype(np.float32).astype(np.float64), B.astype(np.float32).astype(np.float64)
    want = oc.contract(spec, ext, Ar, Br, threads=4)
    scale = oc.contract(spec, ext, np.abs(Ar), np.abs(Br), threads=4)
    errs = {}
    for split in (0, 1):
        got = run(tcmod, spec, ext, "bf16x3", dA, dB, pair=pair, split=split)
        errs[split] = float(np.max(np.abs(got - want) / scale))
    assert errs[1] <= 1e-6, errs
    assert errs[1] <= errs[0], errs


def test_pair_setters_reject_bad_values(tcmod):
    plan = tcmod.Plan("abc=ai,ibc", [8, 8, 8, 8], dtype="bf16x3")
    for fn in (plan.set_gett_pair, plan.set_split_accumulators):
        with pytest.raises(tcmod.TcError):
            fn(2)
    with pytest.raises(tcmod.TcError):
        plan.set_gett_pair(-1)
    plan.set_split_accumulators(-1)  # automatic: by K
    plan.close()
