"""GPU checks of the serving loop: every result of a mixed stream matches
the oracle, equals bit for bit the same request run alone, admission waits
for memory instead of failing, and oversize requests are refused."""
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


def mix(n, seed):
    rng = np.random.default_rng(seed)
    out = []
    for q in range(n):
        spec = ("abc=ai,ibc", "abc=iaj,jbic", "ab=aij,jib")[q % 3]
        dtype = ("f64", "f32", "bf16x3")[rng.integers(0, 3)]
        order = synth.index_order(spec)
        c, a, b = synth.spec_modes(spec)
        ext = [int(rng.integers(4, 12)) if (x in a and x in b and x not in c) else int(rng.integers(8, 70))
               for x in order]
        out.append((spec, ext, dtype))
    return out


def host_buffers(spec, ext, dtype, seed):
    A, B, _ = synth.uniform_operands(spec, ext, seed=seed)
    tdt = torch.float64 if dtype == "f64" else torch.float32
    hA = torch.from_numpy(A).to(tdt).pin_memory()
    hB = torch.from_numpy(B).to(tdt).pin_memory()
    hC = torch.full((synth.dense_sizes(spec, ext)[0],), float("nan"), dtype=tdt).pin_memory()
    return hA, hB, hC


def test_mixed_stream_matches_oracle_and_is_order_independent(tcmod):
    reqs = mix(36, seed=5)
    bufs = [host_buffers(s, e, d, seed=100 + q) for q, (s, e, d) in enumerate(reqs)]
    server = tcmod.Server(budget_bytes=1 << 30, slots=16, streams=4)
    ids = [server.submit(s, e, d, hA, hB, hC) for (s, e, d), (hA, hB, hC) in zip(reqs, bufs)]
    for rid in ids:
        server.wait(rid, 120.0)
    mixed = [hC.clone() for _, _, hC in bufs]
    st = server.stats()
    assert st["completed"] == len(reqs) and st["failed"] == 0 and st["p99_seconds"] > 0
    for q, ((spec, ext, dtype), (hA, hB, _)) in enumerate(zip(reqs, bufs)):
        Ar, Br = hA.double().numpy(), hB.double().numpy()
        want = oc.contract(spec, ext, Ar, Br)
        scale = oc.contract(spec, ext, np.abs(Ar), np.abs(Br))
        c, a, b = synth.spec_modes(spec)
        K = int(np.prod([e for x, e in zip(synth.index_order(spec), ext) if x in a and x in b and x not in c]))
        # FP32: K-term FMA chain; split-BF16: the FP32 accumulator sums 6K
        # slice products, plus at most 3u of split remainder per term
        bound = 1e-12 if dtype == "f64" else ((K + 1) * U32 if dtype == "f32" else (6 * K + 4) * U32)
        err = np.max(np.abs(mixed[q].double().numpy() - want) / scale)
        assert err <= bound, (q, spec, ext, dtype, err)
        if dtype == "bf16x3":  # the chosen form's target: FP32-level, 1e-6
            assert err <= 1e-6, (q, spec, ext, dtype, err)
    # each request alone gives the same bits
    for q, ((spec, ext, dtype), (hA, hB, hC)) in enumerate(zip(reqs, bufs)):
        hC.fill_(float("nan"))
        rid = server.submit(spec, ext, dtype, hA, hB, hC)
        server.wait(rid, 60.0)
        assert torch.equal(hC, mixed[q]), (q, spec, ext, dtype)
    server.close()


def test_admission_waits_for_memory(tcmod):
    # budget for about two requests at a time: the others wait, none fails
    spec, ext = "abc=ai,ibc", [96, 96, 96, 16]
    bufs = [host_buffers(spec, ext, "f32", seed=q) for q in range(10)]
    per = sum(synth.dense_sizes(spec, ext)) * 4
    server = tcmod.Server(budget_bytes=int(2.5 * per) + (4 << 20), slots=8, streams=4)
    ids = [server.submit(spec, ext, "f32", hA, hB, hC) for hA, hB, hC in bufs]
    for rid in ids:
        server.wait(rid, 60.0)
    st = server.stats()
    assert st["completed"] == 10 and st["failed"] == 0
    assert st["peak_inflight"] <= 3
    for hA, hB, hC in bufs:
        want = oc.contract(spec, ext, hA.double().numpy(), hB.double().numpy())
        assert np.max(np.abs(hC.double().numpy() - want)) < 1e-3
    server.close()


def test_oversize_request_is_refused(tcmod):
    server = tcmod.Server(budget_bytes=4 << 20, slots=2, streams=1)
    hA = torch.zeros(16, dtype=torch.float32).pin_memory()
    with pytest.raises(tcmod.TcError) as e:
        server.submit("abc=ai,ibc", [256, 256, 256, 16], "f32", hA, hA, None)
    assert tcmod.STATUS_NAMES[e.value.status] == "TC_ERROR_ADMISSION"
    server.close()


def test_requests_share_launches(tcmod):
    # 48 requests submitted at once on two streams: they are batched into
    # shared launches (far fewer launches than requests), every result
    # matches the oracle, and each equals the same request run alone
    rng = np.random.default_rng(11)
    reqs = []
    for q in range(48):
        spec = ("abc=ai,ibc", "abc=iaj,jbic", "ab=aij,jib")[q % 3]
        dtype = ("f64", "f32", "bf16x3")[q % 3 if q < 24 else (q // 3) % 3]
        order = synth.index_order(spec)
        c, a, b = synth.spec_modes(spec)
        ext = [int(rng.integers(4, 20)) if (x in a and x in b and x not in c) else int(rng.integers(8, 90))
               for x in order]
        reqs.append((spec, ext, dtype))
    bufs = [host_buffers(s, e, d, seed=300 + q) for q, (s, e, d) in enumerate(reqs)]
    server = tcmod.Server(budget_bytes=1 << 30, slots=64, streams=2)
    ids = [server.submit(s, e, d, hA, hB, hC) for (s, e, d), (hA, hB, hC) in zip(reqs, bufs)]
    for rid in ids:
        server.wait(rid, 120.0)
    st = server.stats()
    assert st["completed"] == 48 and st["failed"] == 0
    assert st["batches"] < 48 and st["max_batch"] > 1, st
    mixed = [hC.clone() for _, _, hC in bufs]
    for q, ((spec, ext, dtype), (hA, hB, hC)) in enumerate(zip(reqs, bufs)):
        Ar, Br = hA.double().numpy(), hB.double().numpy()
        want = oc.contract(spec, ext, Ar, Br)
        scale = oc.contract(spec, ext, np.abs(Ar), np.abs(Br))
        c, a, b = synth.spec_modes(spec)
        K = int(np.prod([e for x, e in zip(synth.index_order(spec), ext) if x in a and x in b and x not in c]))
        bound = {"f64": 1e-12, "f32": (K + 1) * U32, "bf16x3": 1e-6}[dtype]
        assert np.max(np.abs(mixed[q].double().numpy() - want) / scale) <= bound, (q, spec, ext, dtype)
    for q in range(0, 48, 5):  # alone, on the idle server
        (spec, ext, dtype), (hA, hB, hC) = reqs[q], bufs[q]
        hC.fill_(float("nan"))
        server.wait(server.submit(spec, ext, dtype, hA, hB, hC), 60.0)
        assert torch.equal(hC, mixed[q]), (q, spec, ext, dtype)
    server.close()


@pytest.mark.parametrize("spec,ext,dtype", [
    ("ab=aij,jib", [100, 120, 24, 20], "bf16x3"),   # K = 480: compensated, one launch of its own
    ("abc=iaj,jbic", [40, 36, 24, 16, 16], "bf16x3"),  # K = 256: the split-accumulator class
    ("abc=ai,ibc", [64, 48, 40, 32], "tf32"),      # another tensor dtype: one launch of its own
    ("habc=hai,hibc", [3, 60, 40, 30, 24], "bf16x3"),  # a batch index, in a batched launch
    ("habc=hai,hibc", [3, 60, 40, 30, 24], "f64"),
])
def test_solo_and_split_classes(tcmod, spec, ext, dtype):
    hA, hB, hC = host_buffers(spec, ext, dtype, seed=7)
    server = tcmod.Server(budget_bytes=1 << 28, slots=4, streams=2)
    server.wait(server.submit(spec, ext, dtype, hA, hB, hC), 60.0)
    assert server.stats()["failed"] == 0
    server.close()
    Ar, Br = hA.double().numpy(), hB.double().numpy()
    want = oc.contract(spec, ext, Ar, Br)
    scale = oc.contract(spec, ext, np.abs(Ar), np.abs(Br))
    err = float(np.max(np.abs(hC.double().numpy() - want) / scale))
    assert err <= {"bf16x3": 1e-6, "f64": 1e-12}.get(dtype, 2 * 2.0 ** -11 + 1e-5), err
