"""GPU parity of contraction chains (two kernels in one tree) against the
chain oracle's direct sum, for every variant (pair order, sliced or not)
and dtype; and the predictor's choice of order."""
import numpy as np
import pytest

from oracle import chain as och

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

U = {"f64": 2.0 ** -53, "f32": 2.0 ** -24}


@pytest.fixture(scope="module")
def tcmod():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build_library()
    from paper_1409_8608_gb300 import tc
    tc.load()
    return tc


CHAINS = [
    ("ad=ab,bc,cd", [40, 36, 24, 32]),          # matrix chain: a, d, b, c
    ("abc=ai,ij,jbc", [24, 20, 12, 16, 8]),     # a, b, c, i, j
    ("ab=ai,ij,jbi", [30, 20, 12, 16]),         # i in all three operands
    ("ac=aij,jk,kic", [9, 7, 5, 6, 10]),        # two contracted indices per step
]


def operands(spec, ext, seed, integer):
    sizes = och.chain_sizes(spec, ext)
    rng = np.random.default_rng(seed)
    if integer:
        return [rng.integers(-4, 5, n).astype(np.float64) for n in sizes[1:]]
    return [rng.uniform(-1, 1, n) for n in sizes[1:]]


def run_variant(tc, ch, i, dev_ops, n_d, tdt, alpha=1.0, beta=0.0, D0=None):
    ch.select(i)
    D = torch.full((n_d,), float("nan"), dtype=tdt, device="cuda") if D0 is None else D0.clone()
    ch.execute(*dev_ops, D, alpha=alpha, beta=beta)
    torch.cuda.synchronize()
    ch.device_status()
    return D.double().cpu().numpy()


@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16x3"])
@pytest.mark.parametrize("spec,ext", CHAINS)
def test_every_variant_exact_on_integers(tcmod, spec, ext, dtype):
    # integers in [-4, 4]: every product and partial sum is exact in FP32
    # here (and every slice of split-BF16 past the first is zero)
    X, Y, Z = operands(spec, ext, 3, True)
    want = och.contract3(spec, ext, X, Y, Z)
    tdt = torch.float64 if dtype == "f64" else torch.float32
    dev = [torch.from_numpy(v).to(tdt).cuda() for v in (X, Y, Z)]
    ch = tcmod.Chain(spec, ext, dtype)
    vs = ch.variants()
    assert vs
    for i, v in enumerate(vs):
        got = run_variant(tcmod, ch, i, dev, want.size, tdt)
        assert np.array_equal(got, want), (spec, v)
    ch.close()


@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16x3"])
@pytest.mark.parametrize("spec,ext", CHAINS[:2])
def test_variants_within_bound_alpha_beta(tcmod, spec, ext, dtype):
    X, Y, Z = operands(spec, ext, 4, False)
    want = och.contract3(spec, ext, X, Y, Z)
    scale = och.contract3(spec, ext, np.abs(X), np.abs(Y), np.abs(Z))
    tdt = torch.float64 if dtype == "f64" else torch.float32
    if dtype != "f64":  # the FP32 inputs as given
        X, Y, Z = (v.astype(np.float32).astype(np.float64) for v in (X, Y, Z))
        want = och.contract3(spec, ext, X, Y, Z)
        scale = och.contract3(spec, ext, np.abs(X), np.abs(Y), np.abs(Z))
    dev = [torch.from_numpy(v).to(tdt).cuda() for v in (X, Y, Z)]
    D0 = torch.from_numpy(np.random.default_rng(5).uniform(-1, 1, want.size)).to(tdt).cuda()
    d0 = D0.double().cpu().numpy()
    ch = tcmod.Chain(spec, ext, dtype)
    # the summed extents of both steps bound the rounding: each step is a
    # sum of at most K products (FP32 / FP64), the intermediate rounded once
    letters = och.chain_index_order(spec)
    d = och.parse_chain(spec)[0]
    ksum = int(np.prod([e for m, e in zip(letters, ext) if m not in d]))
    for i, v in enumerate(ch.variants()):
        got = run_variant(tcmod, ch, i, dev, want.size, tdt, alpha=1.5, beta=-0.5, D0=D0)
        ref = 1.5 * want - 0.5 * d0
        err = np.max(np.abs(got - ref) / (1.5 * scale + 0.5 * np.abs(d0)))
        bound = 1e-6 if dtype == "bf16x3" else (2 * ksum + 4) * U[dtype]
        assert err <= bound, (spec, v, err, bound)
    ch.close()


def test_predictor_chooses_the_cheap_order(tcmod):
    # X: 2048 x 16, Y: 16 x 2048, Z: 2048 x 16: X (Y Z) does 128x fewer flops
    spec, ext = "ad=ab,bc,cd", [2048, 16, 16, 2048]
    ch = tcmod.Chain(spec, ext, "f32")
    ch.predict(all_algorithms=False)
    vs = ch.variants()
    assert all(v["predicted_seconds"] > 0 for v in vs)
    plain = {v["first"]: v for v in vs if v["sliced"] is None}
    assert plain[(1, 2)]["predicted_seconds"] < plain[(0, 1)]["predicted_seconds"]
    assert vs[ch.selected()]["first"] == (1, 2)
    ch.close()


def test_predict_over_every_algorithm(tcmod):
    spec, ext = "abc=ai,ij,jbc", [24, 20, 12, 16, 8]
    ch = tcmod.Chain(spec, ext, "f64")
    ch.predict(all_algorithms=True)
    vs = ch.variants()
    assert all(v["predicted_seconds"] > 0 for v in vs)
    best = min(range(len(vs)), key=lambda i: vs[i]["predicted_seconds"])
    assert ch.selected() == best
    X, Y, Z = operands(spec, ext, 6, True)
    dev = [torch.from_numpy(v).cuda() for v in (X, Y, Z)]
    got = run_variant(tcmod, ch, best, dev, och.chain_sizes(spec, ext)[0], torch.float64)
    assert np.array_equal(got, och.contract3(spec, ext, X, Y, Z))
    ch.close()
