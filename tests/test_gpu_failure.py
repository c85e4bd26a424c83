"""Failure detection on the GPU without a fault: a kernel waits on an
mbarrier that nothing arrives at, its bounded wait runs out, it returns and
the host reads TC_ERROR_TIMEOUT; the context stays usable afterwards."""
import time

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


def test_unsignalled_wait_times_out_and_context_survives(tcmod):
    t0 = time.perf_counter()
    st = tcmod.tc_selftest_bounded_wait(50_000_000, 0)  # 50 ms, nothing arrives
    dt = time.perf_counter() - t0
    assert tcmod.STATUS_NAMES[st] == "TC_ERROR_TIMEOUT"
    assert dt < 5.0
    # positive control: the same wait, signalled
    assert tcmod.tc_selftest_bounded_wait(50_000_000, 1) == 0
    # the context still runs contractions correctly
    spec, ext = "abc=ai,ibc", [40, 30, 20, 8]
    A, B, _ = synth.integer_operands(spec, ext, seed=3)
    want = oc.contract(spec, ext, A, B)
    plan = tcmod.Plan(spec, ext, dtype="f64")
    plan.select(0)
    dA = torch.from_numpy(A).cuda()
    dB = torch.from_numpy(B).cuda()
    dC = torch.empty(want.size, dtype=torch.float64, device="cuda")
    plan.execute(dA, dB, dC)
    torch.cuda.synchronize()
    plan.device_status()
    plan.close()
    assert np.array_equal(dC.cpu().numpy(), want)


def test_repeated_timeouts_stay_bounded(tcmod):
    t0 = time.perf_counter()
    for _ in range(5):
        assert tcmod.STATUS_NAMES[tcmod.tc_selftest_bounded_wait(10_000_000, 0)] == "TC_ERROR_TIMEOUT"
    assert time.perf_counter() - t0 < 10.0
