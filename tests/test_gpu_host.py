"""tc_execute_host: operands in (pinned) host memory, copies in, the
selected algorithm, the result copied back -- one C ABI call.  Checked
against the FP64 oracle (1e-12 componentwise for FP64, the chosen form's
1e-6 for split-BF16) and bit for bit against tc_execute on device copies of
the same operands, for dense and padded-stride layouts and beta != 0."""
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


@pytest.mark.parametrize("dtype,alg", [("f64", "gett"), ("f64", "i'c-gemm"), ("f32", "gett"), ("bf16x3", "gett")])
def test_host_call_matches_device_call(tcmod, dtype, alg):
    spec, ext = "abc=iaj,jbic", [40, 36, 24, 16, 16]
    A, B, C0 = synth.uniform_operands(spec, ext, seed=8, with_c=True)
    tdt = torch.float64 if dtype == "f64" else torch.float32
    hA = torch.from_numpy(A).to(tdt).pin_memory()
    hB = torch.from_numpy(B).to(tdt).pin_memory()
    plan = tcmod.Plan(spec, ext, dtype=dtype)
    plan.select({a["name"]: a["id"] for a in plan.algorithms()}[alg])
    s = torch.cuda.Stream()
    for alpha, beta in ((1.0, 0.0), (2.0, 0.5)):
        hC = torch.from_numpy(C0).to(tdt).pin_memory()
        dC = hC.cuda()
        plan.execute_host(hA, hB, hC, alpha=alpha, beta=beta, stream=s)
        s.synchronize()
        plan.execute(hA.cuda(), hB.cuda(), dC, alpha=alpha, beta=beta, stream=s)
        s.synchronize()
        plan.device_status()
        assert torch.equal(hC, dC.cpu()), (alpha, beta)
        Ar, Br = hA.double().numpy(), hB.double().numpy()
        Cr = torch.from_numpy(C0).to(tdt).double().clone().numpy()  # C as the device saw it (the oracle writes into it)
        scale = oc.contract(spec, ext, np.abs(Ar), np.abs(Br), C=np.abs(Cr), alpha=abs(alpha), beta=abs(beta))
        want = oc.contract(spec, ext, Ar, Br, C=Cr, alpha=alpha, beta=beta)
        err = float(np.max(np.abs(hC.double().numpy() - want) / scale))
        # FP32: a (K + 2)-term FMA chain including beta * C, K = 256
        f32_bound = 258 * 2.0 ** -24 / (1 - 258 * 2.0 ** -24)
        assert err <= {"f64": 1e-12, "f32": f32_bound, "bf16x3": 1e-6}[dtype], (alpha, beta, err)
    plan.close()


def test_host_call_padded_strides(tcmod):
    # C with padded strides: the host buffer spans the padding; only the
    # elements of C are checked (with beta = 0 the padding comes back as
    # whatever the device buffer held)
    spec, ext = "abc=ai,ibc", [30, 20, 7, 12]
    a, b, c, i = ext
    sC = [1, a + 3, (a + 3) * b + 5]
    strides = sC + [1, a] + [1, i, i * b]
    span = 1 + sum((e - 1) * st for e, st in zip((a, b, c), sC))
    A, B, _ = synth.uniform_operands(spec, ext, seed=9)
    hA = torch.from_numpy(A).pin_memory()
    hB = torch.from_numpy(B).pin_memory()
    hC = torch.full((span,), 7.0, dtype=torch.float64).pin_memory()
    plan = tcmod.Plan(spec, ext, strides=strides, dtype="f64")
    plan.execute_host(hA, hB, hC, alpha=1.0, beta=0.0)
    torch.cuda.synchronize()
    want = oc.contract(spec, ext, A, B)
    got = np.empty(a * b * c)
    hc = hC.numpy()
    for z in range(c):
        for y in range(b):
            got[(z * b + y) * a:(z * b + y + 1) * a] = hc[z * sC[2] + y * sC[1]:z * sC[2] + y * sC[1] + a]
    scale = oc.contract(spec, ext, np.abs(A), np.abs(B))
    assert np.max(np.abs(got - want) / scale) <= 1e-12
    plan.close()
