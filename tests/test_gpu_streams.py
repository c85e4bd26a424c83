"""One plan, one stream at a time (boundary rule of the C ABI): tc_execute on
a second stream while the plan's previous execute is still in flight is
refused with TC_ERROR_INVALID_ARGUMENT and enqueues nothing; executes on the
same stream queue behind one another; once the first stream has finished,
the second is accepted and the result matches the FP64 oracle."""
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


@pytest.mark.parametrize("alg", ["gett", "i'c-gemm"])
def test_second_stream_refused_while_in_flight(tcmod, alg):
    spec, ext = "abc=iaj,jbic", [40, 36, 24, 16, 16]
    dev = torch.device("cuda:0")
    A, B, _ = synth.uniform_operands(spec, ext, seed=3)
    want = oc.contract(spec, ext, A, B)
    scale = oc.contract(spec, ext, np.abs(A), np.abs(B))
    dA, dB = torch.from_numpy(A).to(dev), torch.from_numpy(B).to(dev)
    n = want.size
    plan = tcmod.Plan(spec, ext, dtype="f64")
    plan.select({a["name"]: a["id"] for a in plan.algorithms()}[alg])
    s1, s2 = torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev)
    c1 = torch.full((n,), float("nan"), dtype=torch.float64, device=dev)
    c2 = torch.full((n,), float("nan"), dtype=torch.float64, device=dev)
    torch.cuda.synchronize()
    # keep s1 busy (~tens of ms of spinning) so that its execute is still
    # pending when the second stream asks
    with torch.cuda.stream(s1):
        torch.cuda._sleep(200_000_000)
    plan.execute(dA, dB, c1, stream=s1)
    with pytest.raises(tcmod.TcError) as e:
        plan.execute(dA, dB, c2, stream=s2)
    assert tcmod.STATUS_NAMES[e.value.status] == "TC_ERROR_INVALID_ARGUMENT"
    s2.synchronize()
    assert bool(torch.isnan(c2).all())  # the refused call enqueued nothing
    # the same stream queues behind the first execute
    plan.execute(dA, dB, c1, stream=s1)
    s1.synchronize()
    # now idle: the second stream is accepted
    plan.execute(dA, dB, c2, stream=s2)
    s2.synchronize()
    plan.device_status()
    for c in (c1, c2):
        got = c.cpu().numpy()
        assert np.max(np.abs(got - want) / scale) <= 1e-12
    plan.close()
