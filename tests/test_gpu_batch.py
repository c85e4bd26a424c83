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


def class_of(M, N, K):
    # the autotuner's shape class: ceil(log2 M), ceil(log2 K), N bucket
    cl = lambda x: int(np.ceil(np.log2(x))) if x > 1 else 0
    return min(cl(M), 8), min(cl(K), 7), 0 if N <= 256 else (1 if N <= 2048 else 2)


def merged(spec, ext):
    c, a, b = oc.parse_spec(spec)
    e = dict(zip(oc.index_order(spec), ext))
    M = int(np.prod([e[x] for x in a if x in c]))
    N = int(np.prod([e[x] for x in b if x in c]))
    K = int(np.prod([e[x] for x in a if x in b and x not in c]))
    return M, N, K


def chunk_useful(bk, kmax):
    return bk == 8 or kmax > bk // 2


def stage_fits(s, bk):
    pitch = 4 * (((bk + 3) >> 2) | 1)
    return bk * (8 << s) + (512 >> s) * pitch <= 6400


# every (tile shape, K chunk) the SIMT kernel runs
SHAPE_CHUNKS = [(s, bk) for s in range(5) for bk in (8, 16, 32) if stage_fits(s, bk)]

# layouts: the benchmark's (16-byte copies of B, staged C), k-contiguous A
# (element copies of A), n-contiguous B (element copies of B), C with n
# fastest (direct stores); extents with odd K, K over several chunks,
# M over 128 (several row tiles)
LAYOUT_CASES = [
    ("abc=ai,ibc", [[8, 3, 5, 4], [13, 7, 9, 12], [37, 5, 11, 5], [70, 9, 2, 40], [128, 4, 33, 32],
                    [200, 3, 6, 7], [1, 64, 2, 70], [9, 1, 1, 1]]),
    ("abc=ia,ibc", [[8, 3, 5, 4], [13, 7, 9, 12], [37, 5, 11, 5], [70, 9, 2, 40], [130, 4, 3, 33]]),
    ("abc=ai,bci", [[8, 3, 5, 4], [13, 7, 9, 12], [37, 5, 11, 5], [70, 9, 2, 40], [130, 4, 3, 33]]),
    ("bca=ai,ibc", [[8, 3, 5, 4], [13, 7, 9, 12], [37, 5, 11, 5], [70, 9, 2, 40], [130, 4, 3, 33]]),
]


def forced_cache(tmp_path, spec, dtype_code, rows, s, bk):
    # tuning-cache entries forcing (tile shape s, chunk bk) on every class of
    # the rows; keys follow the library's "batch|spec|dtype|class|device"
    name = torch.cuda.get_device_name()
    lines = []
    for ext in rows:
        M, N, K = merged(spec, ext)
        m, k, n = class_of(M, N, K)
        kb = bk if chunk_useful(bk, 1 << k) else 8
        key = f"batch|{spec}|{dtype_code}|m{m}k{k}n{n}|{name}"
        lines.append('{"key": "%s", "batch_k_chunk": %d, "batch_tile_m": %d}' % (key, kb, 8 << s))
    path = tmp_path / f"force_{s}_{bk}.jsonl"
    path.write_text("\n".join(lines) + "\n")
    return path


def operands_offset(spec, ext, dtype, seed, offset, integer=True):
    # device copies starting `offset` elements into their allocation (an
    # offset of 1 defeats every 16-byte copy and shifts the staged C)
    tdt = {"f32": torch.float32, "f64": torch.float64}[dtype]
    gen = synth.integer_operands if integer else synth.uniform_operands
    A, B, _ = gen(spec, ext, seed=seed)
    out = []
    for X in (A, B):
        buf = torch.zeros(X.size + offset, dtype=tdt, device="cuda")
        buf[offset:] = torch.from_numpy(X).to(tdt).cuda()
        out.append(buf[offset:])
    n = synth.dense_sizes(spec, ext)[0]
    cbuf = torch.full((n + offset,), float("nan"), dtype=tdt, device="cuda")
    return A, B, out[0], out[1], cbuf[offset:]


def test_batch_autotune_classes_and_bits(tcmod):
    rows = problems(400, 8, 128, seed=8)
    As, Bs, Cs, host = make(rows, "f32", 80)
    spec = SPEC
    batch = tcmod.Batch(spec, rows, "f32")
    batch.set_operands(As, Bs, Cs)
    batch.execute()  # rule tiles
    torch.cuda.synchronize()
    ref = [c.clone() for c in Cs]
    table = batch.autotune(reps=3)
    classes = {class_of(*merged(spec, e)) for e in rows}
    assert len(table) == len(classes)
    assert {(r["m_log2"], r["k_log2"], r["n_class"]) for r in table} == classes
    assert sum(r["problems"] for r in table) == len(rows)
    for r in table:
        if r["candidates"] == 0:  # answered from the cache of an earlier test
            continue
        assert r["seconds_best"] > 0 and r["seconds_best"] <= r["seconds_rule"] and \
            r["seconds_best"] <= r["seconds_fixed"], r
        assert (r["tile_m"], r["tile_n"]) in [(8 << s, 512 >> s) for s in range(5)]
        assert r["k_chunk"] in (8, 16, 32)
    cfg = batch.config()
    assert cfg["policy"] == 2 and cfg["stages"] in (2, 3)
    # the autotuner's launches left C = A.B; every tiling sums K in the same
    # order, so the tuned launch gives the rule's bits
    assert all(torch.equal(c, r) for c, r in zip(Cs, ref))
    for c in Cs:
        c.fill_(float("nan"))
    batch.execute()
    torch.cuda.synchronize()
    assert all(torch.equal(c, r) for c, r in zip(Cs, ref))
    # a second run of the tuner answers every class from the cache
    again = batch.autotune(reps=3)
    assert all(r["candidates"] == 0 for r in again)
    batch.set_tiles(1)
    with pytest.raises(tcmod.TcError):
        tcmod.Batch(spec, rows[:3], "f32").set_tiles(2)  # no tuning yet
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


# the split-BF16 stream kernel: M from 1 to 128 (MMA N 16..128), K a
# multiple of 4 in 16- and 32-wide stages, N ragged around the 128-column
# tile; rows are [a, b, c, i] of abc=ai,ibc (M = a, N = b c, K = i)
STREAM_ROWS = [[1, 1, 1, 4], [7, 127, 1, 12], [16, 128, 1, 16], [17, 129, 1, 20], [100, 3, 100, 32],
               [128, 5, 61, 8], [33, 1, 2, 28], [64, 256, 1, 24], [5, 40, 7, 4], [128, 128, 2, 32]]


def test_batch_bf16x3_stream_exact_on_integers(tcmod):
    As, Bs, Cs, host = make(STREAM_ROWS, "bf16x3", 100, integer=True)
    batch = tcmod.Batch(SPEC, STREAM_ROWS, "bf16x3")
    batch.set_operands(As, Bs, Cs)
    batch.prepare()
    assert batch.config()["kernel"] == "stream"
    batch.execute()
    torch.cuda.synchronize()
    batch.device_status()
    for ext, (A, B), C in zip(STREAM_ROWS, host, Cs):
        assert np.array_equal(C.double().cpu().numpy(), oc.contract(SPEC, ext, A, B)), ext
    # alpha, beta and one launch per problem
    C0 = [torch.from_numpy(synth.integer_operands(SPEC, e, seed=5, with_c=True)[2]).float().cuda()
          for e in STREAM_ROWS]
    for c, c0 in zip(Cs, C0):
        c.copy_(c0)
    batch.execute(alpha=2.0, beta=-3.0, per_problem=True)
    torch.cuda.synchronize()
    batch.device_status()
    for ext, (A, B), C, c0 in zip(STREAM_ROWS, host, Cs, C0):
        want = 2.0 * oc.contract(SPEC, ext, A, B) - 3.0 * c0.double().cpu().numpy()
        assert np.array_equal(C.double().cpu().numpy(), want), ext
    batch.close()


def test_batch_bf16x3_stream_bound_and_fallbacks(tcmod):
    # uniform inputs within the FP32-level target; a misaligned operand and
    # a K that is not a multiple of 4 take the GETT tiles instead
    rows = STREAM_ROWS
    As, Bs, Cs, host = make(rows, "bf16x3", 110)
    batch = tcmod.Batch(SPEC, rows, "bf16x3")
    batch.set_operands(As, Bs, Cs)
    batch.execute()
    torch.cuda.synchronize()
    batch.device_status()
    for (A, B), ext, C in zip(host, rows, Cs):
        Ar, Br = A.astype(np.float32).astype(np.float64), B.astype(np.float32).astype(np.float64)
        want = oc.contract(SPEC, ext, Ar, Br)
        scale = oc.contract(SPEC, ext, np.abs(Ar), np.abs(Br))
        err = np.max(np.abs(C.double().cpu().numpy() - want) / scale)
        assert err <= 1e-6, (ext, err)
    batch.close()
    # B of the first problem one element into its allocation
    buf = torch.zeros(Bs[0].numel() + 1, device="cuda")
    buf[1:] = Bs[0]
    batch = tcmod.Batch(SPEC, rows, "bf16x3")
    batch.set_operands(As, [buf[1:]] + Bs[1:], Cs)
    batch.prepare()
    assert batch.config()["kernel"] == "gett"
    batch.close()
    odd = [[9, 5, 3, 6], [20, 7, 2, 4]]
    As2, Bs2, Cs2, host2 = make(odd, "bf16x3", 120, integer=True)
    batch = tcmod.Batch(SPEC, odd, "bf16x3")
    batch.set_operands(As2, Bs2, Cs2)
    batch.execute()
    torch.cuda.synchronize()
    batch.device_status()
    assert batch.config()["kernel"] == "gett"
    for ext, (A, B), C in zip(odd, host2, Cs2):
        assert np.array_equal(C.double().cpu().numpy(), oc.contract(SPEC, ext, A, B)), ext
    batch.close()


def test_batch_bf16x3_autotune(tcmod):
    rows = problems(120, 8, 128, seed=9)
    As, Bs, Cs, host = make(rows, "bf16x3", 90)
    batch = tcmod.Batch(SPEC, rows, "bf16x3")
    batch.set_operands(As, Bs, Cs)
    table = batch.autotune(reps=2)
    assert len(table) == 1 and table[0]["tile_n"] in (128, 256) and table[0]["problems"] == len(rows)
    assert table[0]["candidates"] == 3 and table[0]["kernel"] in (1, 2)
    assert table[0]["seconds_best"] <= min(table[0]["seconds_rule"], table[0]["seconds_fixed"])
    cfg = batch.config()
    assert cfg["tile_n"] == table[0]["tile_n"] and cfg["kernel"] == ["simt", "gett", "stream"][table[0]["kernel"]]
    for c in Cs:
        c.fill_(float("nan"))
    batch.execute()
    torch.cuda.synchronize()
    batch.device_status()
    for (A, B), ext, C in zip(host[:30], rows[:30], Cs[:30]):
        Ar, Br = A.astype(np.float32).astype(np.float64), B.astype(np.float32).astype(np.float64)
        want = oc.contract(SPEC, ext, Ar, Br)
        scale = oc.contract(SPEC, ext, np.abs(Ar), np.abs(Br))
        err = np.max(np.abs(C.double().cpu().numpy() - want) / scale)
        assert err <= 1e-6, (ext, err)
    batch.close()


@pytest.mark.parametrize("dtype", ["f32", "f64"])
@pytest.mark.parametrize("spec,rows", LAYOUT_CASES)
def test_batch_every_tile_shape_chunk_and_layout(tcmod, tmp_path, spec, rows, dtype):
    # exact on integer inputs for every (tile shape, K chunk), copy path and
    # epilogue path, with aligned and misaligned operands
    for offset in (0, 1):
        host, As, Bs, Cs = [], [], [], []
        for q, ext in enumerate(rows):
            A, B, dA, dB, dC = operands_offset(spec, ext, dtype, 70 + q, offset)
            host.append((A, B))
            As.append(dA), Bs.append(dB), Cs.append(dC)
        want = [oc.contract(spec, ext, A, B) for ext, (A, B) in zip(rows, host)]
        batch = tcmod.Batch(spec, rows, dtype)
        batch.set_operands(As, Bs, Cs)
        for s, bk in SHAPE_CHUNKS:
            tcmod.tc_tuning_cache_load(forced_cache(tmp_path, spec, tcmod.DTYPES[dtype], rows, s, bk))
            table = batch.autotune(reps=1)
            assert all(r["candidates"] == 0 and r["tile_m"] == 8 << s for r in table), table
            for q in range(len(rows)):
                assert batch.problem_tiles(q)[:2] == (8 << s, 512 >> s)
            for c in Cs:
                c.fill_(float("nan"))
            batch.execute()
            torch.cuda.synchronize()
            for ext, C, w in zip(rows, Cs, want):
                assert np.array_equal(C.double().cpu().numpy(), w), (spec, ext, s, bk, offset)
        batch.close()
