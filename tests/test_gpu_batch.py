"""GPU parity of the batched form (many independent contractions in one
persistent launch) against the FP64 oracle, per problem."""
import numpy as np
import pytest

from oracle import contraction as oc
from paper_1409_8608_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

SPEC = "abc=ai,ibc"


@pytest.fixture(scope="module")
def tcmod():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build_library()
    from paper_1409_8608_gb300 import tc
    tc.load()
    return tc


def problems(count, lo, hi, seed):
    rng = np.random.default_rng(seed)
    a, b, c = (synth.log_uniform_int(rng, lo, hi, count) for _ in range(3))
    i = rng.choice([4, 8, 16, 32], count)
    return [[int(x) for x in r] for r in zip(a, b, c, i)]


def make(ext_rows, dtype, seed, integer=False):
    tdt = {"f32": torch.float32, "f64": torch.float64, "bf16x3": torch.float32}[dtype]
    As, Bs, Cs, host = [], [], [], []
    for q, ext in enumerate(ext_rows):
        gen = synth.integer_operands if integer else synth.uniform_operands
        A, B, _ = gen(SPEC, ext, seed=seed + q)
        host.append((A, B))
        As.append(torch.from_numpy(A).to(tdt).cuda())
        Bs.append(torch.from_numpy(B).to(tdt).cuda())
        Cs.append(torch.full((synth.dense_sizes(SPEC, ext)[0],), float("nan"), dtype=tdt, device="cuda"))
    return As, Bs, Cs, host


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_batch_exact_on_integers(tcmod, dtype):
    rows = problems(300, 8, 40, seed=1)
    As, Bs, Cs, host = make(rows, dtype, 10, integer=True)
    batch = tcmod.Batch(SPEC, rows, dtype)
    batch.set_operands(As, Bs, Cs)
    batch.execute()
    torch.cuda.synchronize()
    for ext, (A, B), C in zip(rows, host, Cs):
        assert np.array_equal(C.double().cpu().numpy(), oc.contract(SPEC, ext, A, B)), ext
    batch.close()


def test_batch_policies_launch_modes_and_graph_agree(tcmod):
    rows = problems(200, 8, 128, seed=2)
    As, Bs, Cs, host = make(rows, "f32", 20)
    batch = tcmod.Batch(SPEC, rows, "f32")
    batch.set_operands(As, Bs, Cs)
    batch.execute()
    torch.cuda.synchronize()
    ref = [c.clone() for c in Cs]
    K_max = 32
    u = 2.0 ** -24
    for (A, B), ext, C in zip(host[:40], rows[:40], ref[:40]):
        Ar, Br = A.astype(np.float32).astype(np.float64), B.astype(np.float32).astype(np.float64)
        want = oc.contract(SPEC, ext, Ar, Br)
        scale = oc.contract(SPEC, ext, np.abs(Ar), np.abs(Br))
        assert np.max(np.abs(C.double().cpu().numpy() - want) / scale) <= (K_max + 1) * u
    # fixed tiles, one launch per problem, and a captured graph: same bits
    batch.set_tiles(0)
    batch.execute()
    torch.cuda.synchronize()
    assert all(torch.equal(c, r) for c, r in zip(Cs, ref))
    batch.set_tiles(1)
    batch.execute(per_problem=True)
    torch.cuda.synchronize()
    assert all(torch.equal(c, r) for c, r in zip(Cs, ref))
    for c in Cs:
        c.fill_(float("nan"))
    batch.prepare()
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        batch.execute(stream=s)
    g.replay()
    torch.cuda.synchronize()
    assert all(torch.equal(c, r) for c, r in zip(Cs, ref))
    batch.close()


def test_batch_alpha_beta(tcmod):
    rows = problems(50, 8, 30, seed=3)
    As, Bs, Cs, host = make(rows, "f64", 30, integer=True)
    C0 = [torch.full_like(c, 3.0) for c in Cs]
    for c, c0 in zip(Cs, C0):
        c.copy_(c0)
    batch = tcmod.Batch(SPEC, rows, "f64")
    batch.set_operands(As, Bs, Cs)
    batch.execute(alpha=2.0, beta=-0.5)
    torch.cuda.synchronize()
    for ext, (A, B), C in zip(rows, host, Cs):
        want = 2.0 * oc.contract(SPEC, ext, A, B) - 1.5
        assert np.array_equal(C.cpu().numpy(), want)
    batch.close()


def test_batch_rejects_unmergeable_spec(tcmod):
    with pytest.raises(tcmod.TcError):
        tcmod.Batch("ab=aij,jib", [[4, 4, 2, 2]], "f32")


# split-BF16 batches run on the tensor-core GETT kernel (128-row tiles)
U = 2.0 ** -24


def test_batch_bf16x3_exact_on_integers(tcmod):
    rows = problems(300, 8, 40, seed=4)
    As, Bs, Cs, host = make(rows, "bf16x3", 40, integer=True)
    batch = tcmod.Batch(SPEC, rows, "bf16x3")
    batch.set_operands(As, Bs, Cs)
    batch.execute()
    torch.cuda.synchronize()
    batch.device_status()
    for ext, (A, B), C in zip(rows, host, Cs):
        assert np.array_equal(C.double().cpu().numpy(), oc.contract(SPEC, ext, A, B)), ext
    batch.close()


def test_batch_bf16x3_bound_launch_modes_and_graph(tcmod):
    rows = problems(60, 8, 128, seed=5)
    As, Bs, Cs, host = make(rows, "bf16x3", 50)
    batch = tcmod.Batch(SPEC, rows, "bf16x3")
    batch.set_operands(As, Bs, Cs)
    batch.execute()
    torch.cuda.synchronize()
    batch.device_status()
    ref = [c.clone() for c in Cs]
    for (A, B), ext, C in zip(host, rows, ref):
        Ar, Br = A.astype(np.float32).astype(np.float64), B.astype(np.float32).astype(np.float64)
        want = oc.contract(SPEC, ext, Ar, Br)
        scale = oc.contract(SPEC, ext, np.abs(Ar), np.abs(Br))
        K = ext[3]
        err = np.max(np.abs(C.double().cpu().numpy() - want) / scale)
        # the target (FP32-level, 1e-6), and the looser 6K-product sanity bound
        assert err <= 1e-6 and err <= (6 * K + 4) * U, (ext, err)
    # one launch per problem and a captured graph give the same bits
    batch.execute(per_problem=True)
    torch.cuda.synchronize()
    assert all(torch.equal(c, r) for c, r in zip(Cs, ref))
    for c in Cs:
        c.fill_(float("nan"))
    batch.prepare()
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        batch.execute(stream=s)
    g.replay()
    torch.cuda.synchronize()
    assert all(torch.equal(c, r) for c, r in zip(Cs, ref))
    # the other tile width: within the same bound
    batch.set_tiles(0)
    batch.execute()
    torch.cuda.synchronize()
    batch.device_status()
    for (A, B), ext, C in zip(host[:20], rows[:20], Cs[:20]):
        Ar, Br = A.astype(np.float32).astype(np.float64), B.astype(np.float32).astype(np.float64)
        want = oc.contract(SPEC, ext, Ar, Br)
        scale = oc.contract(SPEC, ext, np.abs(Ar), np.abs(Br))
        err = np.max(np.abs(C.double().cpu().numpy() - want) / scale)
        assert err <= 1e-6 and err <= (6 * ext[3] + 4) * U, (ext, err)
    batch.close()


def test_batch_bf16x3_alpha_beta(tcmod):
    rows = problems(50, 8, 30, seed=6)
    As, Bs, Cs, host = make(rows, "bf16x3", 60, integer=True)
    for c in Cs:
        c.fill_(3.0)
    batch = tcmod.Batch(SPEC, rows, "bf16x3")
    batch.set_operands(As, Bs, Cs)
    batch.execute(alpha=2.0, beta=-0.5)
    torch.cuda.synchronize()
    batch.device_status()
    for ext, (A, B), C in zip(rows, host, Cs):
        want = 2.0 * oc.contract(SPEC, ext, A, B) - 1.5
        assert np.array_equal(C.double().cpu().numpy(), want)
    batch.close()
