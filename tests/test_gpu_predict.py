"""GPU checks of the predictor (Section 3 on the device), the ranking and
the autotuner.  Timings have no oracle: these tests check that every
prediction is a positive time, that the ranking agrees with measurement
(rank correlation), that selection picks the smallest prediction, and that
the tuner and its cache behave."""
import numpy as np
import pytest

from paper_1409_8608_gb300 import ranking

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


def test_rank_statistics_helpers():
    assert ranking.spearman([1, 2, 3, 4], [10, 20, 30, 40]) == pytest.approx(1.0)
    assert ranking.spearman([1, 2, 3, 4], [4, 3, 2, 1]) == pytest.approx(-1.0)
    assert ranking.kendall([1, 2, 3], [1, 3, 2]) == pytest.approx(1 / 3)


def test_predictions_are_positive_and_selection_uses_them(tcmod):
    plan = tcmod.Plan("abc=ai,ibc", [64, 64, 64, 8])
    pred = plan.predict()  # zero-filled scratch operands
    assert len(pred) == 37 and all(p > 0 for p in pred)
    best = plan.select_best()
    assert best == int(np.argmin(pred)) and plan.selected == best
    plan.close()


def test_small_plain_workload_ranking(tcmod):
    # the plain small workload (a=b=c=64, i=8, FP64): all 37 algorithms
    r = ranking.study("abc=ai,ibc", [64, 64, 64, 8], "f64", reps=5)
    assert len(r["algorithms"]) == 37
    assert r["spearman"] > 0.6, r
    assert r["prediction_seconds"] > 0


def test_permuted_workload_ranking(tcmod):
    r = ranking.study("abc=iaj,jbic", [96, 96, 96, 16, 16], "f64", reps=3)
    assert len(r["algorithms"]) == 177
    assert r["spearman"] > 0.6, {k: v for k, v in r.items() if k != "algorithms"}


def test_tensor_dtype_ranks_gemm_nests_and_gett(tcmod):
    # at tensor-core dtypes the gemm nests and the GETT are predicted (the
    # other kernels cannot run there), and the best prediction is one of them
    plan = tcmod.Plan("abc=iaj,jbic", [256, 256, 8, 16, 16], dtype="bf16x3")
    algs = plan.algorithms()
    gemm_ids = [a["id"] for a in algs if a["kernel"] == "gemm"]
    other = next(a["id"] for a in algs if a["kernel"] == "gemv")
    pred = plan.predict([0, other] + gemm_ids)
    assert pred[0] > 0 and pred[1] < 0 and all(t > 0 for t in pred[2:])
    best = plan.select_best()
    assert best in [0] + gemm_ids
    plan.close()


def test_autotune_and_cache(tcmod, tmp_path):
    spec, ext = "abc=iaj,jbic", [256, 512, 4, 16, 16]
    plan = tcmod.Plan(spec, ext, dtype="bf16x3")
    width, tma = plan.autotune()
    assert width in (128, 256) and tma in (0, 1)
    path = tmp_path / "tune.jsonl"
    tcmod.tc_tuning_cache_save(path)
    text = path.read_text()
    assert "gett_tile" in text and spec in text
    tcmod.tc_tuning_cache_load(path)
    plan2 = tcmod.Plan(spec, ext, dtype="bf16x3")
    assert plan2.autotune() == (width, tma)  # answered from the cache
    plan.close()
    plan2.close()
