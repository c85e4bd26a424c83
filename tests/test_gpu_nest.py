"""GPU parity of every Section 2 algorithm (and the SIMT GETT) against the
FP64 oracle, through the C ABI.

Tolerances: integer-valued inputs in [-8, 8] make every product and partial
sum exact in FP64 (and in FP32 while sums stay below 2**24), so those runs
must match the oracle bit for bit whatever the summation order.  For
uniform inputs the bound is the componentwise forward-error bound of a
length-K FMA chain, |c_hat - c| <= gamma(K+1) * (|A||B|) with
gamma(n) = n*u/(1 - n*u) (u = 2**-53 for FP64, 2**-24 for FP32); the FP64
gate is additionally the 1e-12 componentwise relative error of the
specification."""
import numpy as np
import pytest

from oracle import contraction as oc
from paper_1409_8608_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def tcmod():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build_library()
    from paper_1409_8608_gb300 import tc
    tc.load()
    return tc


TORCH_DT = {"f64": torch.float64, "f32": torch.float32}
NP_DT = {"f64": np.float64, "f32": np.float32}
UNIT = {"f64": 2.0 ** -53, "f32": 2.0 ** -24}


def contracted_size(spec, ext):
    c, a, b = oc.parse_spec(spec)
    e = dict(zip(oc.index_order(spec), ext))
    k = 1
    for x in a:
        if x in b and x not in c:
            k *= e[x]
    return k


def run_all(tc, spec, ext, dtype, A, B, C0=None, alpha=1.0, beta=0.0, ids=None, strides=None,
            nC=None):
    """Execute the algorithms through the C ABI; return {name: C as float64}."""
    dev = torch.device("cuda:0")
    dA = torch.from_numpy(A.astype(NP_DT[dtype])).to(dev)
    dB = torch.from_numpy(B.astype(NP_DT[dtype])).to(dev)
    plan = tc.Plan(spec, ext, strides=strides, dtype=dtype)
    algs = plan.algorithms()
    out = {}
    n = nC if nC is not None else synth.dense_sizes(spec, ext)[0]
    for a in algs:
        if ids is not None and a["id"] not in ids:
            continue
        if C0 is None:
            dC = torch.full((n,), float("nan"), dtype=TORCH_DT[dtype], device=dev)
        else:
            dC = torch.from_numpy(C0.astype(NP_DT[dtype])).to(dev)
        plan.select(a["id"])
        plan.execute(dA, dB, dC, alpha=alpha, beta=beta)
        out[a["name"]] = dC
    torch.cuda.synchronize()
    plan.device_status()
    plan.close()
    return {k: v.double().cpu().numpy() for k, v in out.items()}


def rounded(x, dtype):
    return x.astype(NP_DT[dtype]).astype(np.float64)


CASES = [
    ("abc=ai,ibc", [64, 64, 64, 8]),          # the plain small workload, every algorithm
    ("abc=iaj,jbic", [13, 11, 9, 5, 3]),      # ragged, several tiles of nothing
    ("ab=aij,jib", [70, 67, 5, 3]),           # ragged, gemm tiles with tails
    ("a=iaj,ji", [37, 9, 11]),                # Test 2: BLAS-1/2 only
    ("abc=bi,iac", [9, 7, 5, 4]),             # C slices without a unit stride: C copies
    # batch (Hadamard) indices: always sliced, free loops with strides in A, B and C
    ("habc=hai,hibc", [3, 20, 13, 9, 8]),     # 130 algorithms
    ("abh=aih,ibh", [33, 27, 3, 7]),          # batched matrix product
    ("hab=ha,hb", [4, 30, 20]),               # Hadamard outer product, no contracted index
    ("gha=giah,hig", [3, 4, 20, 5]),          # two batch indices in different orders
]


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("spec,ext", CASES)
def test_every_algorithm_exact_on_integers(tcmod, spec, ext, dtype):
    A, B, _ = synth.integer_operands(spec, ext, seed=3)
    want = oc.contract(spec, ext, A, B)
    got = run_all(tcmod, spec, ext, dtype, A, B)
    assert len(got) == len(tcmod.Plan(spec, ext).algorithms())
    for name, c in got.items():
        assert np.array_equal(c, want), (name, float(np.nanmax(np.abs(c - want))))


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("spec,ext", CASES)
def test_every_algorithm_within_bound_on_uniform(tcmod, spec, ext, dtype):
    A, B, _ = synth.uniform_operands(spec, ext, seed=0)
    Ar, Br = rounded(A, dtype), rounded(B, dtype)
    want = oc.contract(spec, ext, Ar, Br)
    scale = oc.contract(spec, ext, np.abs(Ar), np.abs(Br))
    K = contracted_size(spec, ext)
    u = UNIT[dtype]
    gamma = (K + 1) * u / (1 - (K + 1) * u)
    got = run_all(tcmod, spec, ext, dtype, A, B)
    for name, c in got.items():
        err = np.max(np.abs(c - want) / scale)
        assert err <= gamma, (name, err, gamma)
        if dtype == "f64":
            assert err <= 1e-12


def test_same_contracted_order_is_bitwise_identical(tcmod):
    # with enough outputs per phase (here 64 x 64 x 48, above one wave of
    # threads) every nest kernel runs one FMA chain per C element over the
    # contracted indices in nest order; algorithms that share that order
    # agree bit for bit (the GETT chooses its own order and is excluded).
    # A phase with fewer outputs splits its innermost contracted index over
    # a lane group and adds the partial sums in a fixed tree: the paper fixes
    # no summation order inside a BLAS kernel, so those agree within
    # rounding (the bound tests above)
    spec, ext = "abc=iaj,jbic", [64, 64, 48, 6, 5]
    A, B, _ = synth.uniform_operands(spec, ext, seed=7)
    plan = tcmod.Plan(spec, ext)
    algs = {a["name"]: a for a in plan.algorithms()}
    plan.close()
    got = run_all(tcmod, spec, ext, "f64", A, B)

    def order(a):
        seq = [x for x in a["loops"] if x in "ij"]
        if a["kernel"] in ("dot", "gemv", "gemm"):
            seq.append(a["kernel_indices"][-1])
        return "".join(seq)

    groups = {}
    for name, a in algs.items():
        if a["kernel"] == "gett":
            continue
        groups.setdefault(order(a), []).append(name)
    assert set(groups) == {"ij", "ji"}
    for key, names in groups.items():
        ref = got[names[0]]
        for n in names[1:]:
            assert np.array_equal(got[n], ref), (key, names[0], n)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_alpha_beta(tcmod, dtype):
    spec, ext = "abc=iaj,jbic", [12, 7, 6, 4, 3]
    A, B, C0 = synth.integer_operands(spec, ext, seed=4, with_c=True)
    S = oc.contract(spec, ext, A, B)
    for alpha, beta in ((1.0, 1.0), (-2.0, 0.5), (0.5, -3.0)):
        want = alpha * S + beta * C0
        got = run_all(tcmod, spec, ext, dtype, A, B, C0=C0, alpha=alpha, beta=beta)
        for name, c in got.items():
            assert np.array_equal(c, want), (name, alpha, beta)


def test_beta_zero_never_reads_c(tcmod):
    spec, ext = "abc=ai,ibc", [20, 9, 7, 5]
    A, B, _ = synth.integer_operands(spec, ext, seed=1)
    C0 = np.full(synth.dense_sizes(spec, ext)[0], np.nan)
    got = run_all(tcmod, spec, ext, "f64", A, B, C0=C0, alpha=1.0, beta=0.0)
    want = oc.contract(spec, ext, A, B)
    for name, c in got.items():
        assert np.array_equal(c, want), name


def test_strided_operands_with_copies(tcmod):
    # B stored (c, i, b) with padding, C with a padded leading dimension:
    # the copy decisions follow the strides
    spec, ext = "abc=ai,ibc", [11, 6, 5, 4]
    a, b, c, i = ext
    A, B, _ = synth.integer_operands(spec, ext, seed=2)
    Bn = B.reshape(i, b, c, order="F")
    s_c, s_i, s_b = 1, c + 1, (c + 1) * (i + 2)
    phys = np.zeros(s_b * b)
    for ii in range(i):
        for bb in range(b):
            for cc in range(c):
                phys[ii * s_i + bb * s_b + cc * s_c] = Bn[ii, bb, cc]
    sC = [1, a + 3, (a + 3) * b]
    strides = sC + [1, a] + [s_i, s_b, s_c]
    nC = 1 + (a - 1) + (b - 1) * sC[1] + (c - 1) * sC[2]
    want_buf = np.zeros(nC)
    oc.contract(spec, ext, A, phys, C=want_buf, strides=strides)
    C0 = np.zeros(nC)
    got = run_all(tcmod, spec, ext, "f64", A, phys, C0=C0, beta=0.0, strides=strides, nC=nC)
    mask = np.zeros(nC, bool)
    for z in range(c):
        for y in range(b):
            for x in range(a):
                mask[x + y * sC[1] + z * sC[2]] = True
    copies = 0
    plan = tcmod.Plan(spec, ext, strides=strides)
    copies = sum(1 for al in plan.algorithms() if al["copy_mask"])
    plan.close()
    assert copies > 0
    for name, cbuf in got.items():
        assert np.array_equal(cbuf[mask], want_buf[mask]), name
        assert np.all(cbuf[~mask] == 0), name  # padding untouched


def test_extent_one_modes(tcmod):
    spec, ext = "abc=iaj,jbic", [1, 5, 1, 1, 4]
    A, B, _ = synth.integer_operands(spec, ext, seed=5)
    want = oc.contract(spec, ext, A, B)
    for name, c in run_all(tcmod, spec, ext, "f64", A, B).items():
        assert np.array_equal(c, want), name


def test_large_permuted_sampled(tcmod):
    # the permuted plain workload at n = 256 (i = j = 16): GETT and the gemm
    # algorithms, checked on sampled outputs computed one by one
    spec, ext = "abc=iaj,jbic", [256, 256, 256, 16, 16]
    A, B, _ = synth.uniform_operands(spec, ext, seed=1)
    plan = tcmod.Plan(spec, ext)
    ids = [a["id"] for a in plan.algorithms() if a["kernel"] in ("gett", "gemm")]
    plan.close()
    rng = np.random.default_rng(0)
    pts = np.stack([rng.integers(0, 256, 3000) for _ in range(3)], axis=1)
    want = oc.contract_points(spec, ext, A, B, pts, threads=4)
    scale = oc.contract_points(spec, ext, np.abs(A), np.abs(B), pts, threads=4)
    for dtype in ("f64", "f32"):
        Ar, Br = rounded(A, dtype), rounded(B, dtype)
        if dtype == "f32":
            want = oc.contract_points(spec, ext, Ar, Br, pts, threads=4)
        got = run_all(tcmod, spec, ext, dtype, A, B, ids=ids)
        K = 256
        gamma = (K + 1) * UNIT[dtype] / (1 - (K + 1) * UNIT[dtype])
        lin = pts[:, 0] + 256 * pts[:, 1] + 256 * 256 * pts[:, 2]
        for name, c in got.items():
            err = np.max(np.abs(c[lin] - want) / scale)
            assert err <= gamma, (dtype, name, err)
