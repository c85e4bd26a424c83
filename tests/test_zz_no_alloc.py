"""tc_execute_no_alloc: the executor variant for callers that must not
allocate device memory (its copy scratch is a fixed array in the library).

It is called through the C ABI and must reproduce tc_execute: the same
algorithm runs the same chain of operations, so the results agree bit for
bit, and both stay within the FP64 bound the other parity tests use
(componentwise error <= 1e-12 relative to |A||B|).  Two calls in a row
check that the shared scratch carries nothing over from one call to the
next.  This file is collected last on purpose."""
import ctypes

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


def _no_alloc(tc, plan, alpha, dA, dB, beta, dC):
    a, b = ctypes.c_double(alpha), ctypes.c_double(beta)
    st = tc.load().tc_execute_no_alloc(plan.handle, ctypes.addressof(a), dA.data_ptr(), dB.data_ptr(),
                                       ctypes.addressof(b), dC.data_ptr(), None)
    if st != 0:
        raise tc.TcError(st, "tc_execute_no_alloc", tc.load().tc_last_error().decode())


@pytest.mark.parametrize("spec,ext,names", [
    ("abc=iaj,jbic", [40, 36, 24, 16, 16], ["i'c-gemm", "ci'-gemm", "jc'-gemm", "cbj-dot"]),
    ("abc=bi,iac", [9, 7, 5, 4], None),  # C slices copied in and out
])
def test_no_alloc_matches_tc_execute(tcmod, spec, ext, names):
    A, B, C0 = synth.uniform_operands(spec, ext, seed=2, with_c=True)
    dev = torch.device("cuda:0")
    dA, dB = torch.from_numpy(A).to(dev), torch.from_numpy(B).to(dev)
    n = C0.size
    want = oc.contract(spec, ext, A, B)
    scale = oc.contract(spec, ext, np.abs(A), np.abs(B))
    plan = tcmod.Plan(spec, ext, dtype="f64")
    algs = plan.algorithms()
    chosen = [a for a in algs if a["id"] > 0 and (names is None and a["copy_mask"] or names and a["name"] in names)]
    assert chosen and any(a["copy_mask"] for a in chosen)
    for a in chosen:
        plan.select(a["id"])
        ref = torch.full((n,), float("nan"), dtype=torch.float64, device=dev)
        plan.execute(dA, dB, ref)
        for call in range(2):  # two calls in a row share the scratch
            got = torch.full((n,), float("nan"), dtype=torch.float64, device=dev)
            _no_alloc(tcmod, plan, 1.0, dA, dB, 0.0, got)
            torch.cuda.synchronize()
            g, r = got.cpu().numpy(), ref.cpu().numpy()
            assert np.array_equal(g, r), (a["name"], call)
            assert np.max(np.abs(g - want) / scale) <= 1e-12, (a["name"], call)
        # beta != 0 reads C through the same path
        c_ref = torch.from_numpy(C0).to(dev)
        c_got = c_ref.clone()
        plan.execute(dA, dB, c_ref, alpha=2.0, beta=0.5)
        _no_alloc(tcmod, plan, 2.0, dA, dB, 0.5, c_got)
        torch.cuda.synchronize()
        assert np.array_equal(c_got.cpu().numpy(), c_ref.cpu().numpy()), a["name"]
    plan.close()


def test_no_alloc_refuses_what_it_cannot_hold(tcmod):
    # refused on the host before any device work: a copy needing more than
    # the 16 MiB array, and the GETT
    spec, ext = "abc=iaj,jbic", [256, 256, 256, 16, 16]
    plan = tcmod.Plan(spec, ext, dtype="f64")
    big = next(a for a in plan.algorithms() if a["id"] > 0 and plan.workspace(a["id"]) > (16 << 20))
    d = torch.zeros(16, dtype=torch.float64, device="cuda:0")
    plan.select(big["id"])
    with pytest.raises(tcmod.TcError) as e:
        _no_alloc(tcmod, plan, 1.0, d, d, 0.0, d)
    assert tcmod.STATUS_NAMES[e.value.status] == "TC_ERROR_INVALID_ARGUMENT"
    plan.select(0)
    with pytest.raises(tcmod.TcError) as e:
        _no_alloc(tcmod, plan, 1.0, d, d, 0.0, d)
    assert tcmod.STATUS_NAMES[e.value.status] == "TC_ERROR_INVALID_ALGORITHM"
    plan.close()
