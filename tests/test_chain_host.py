"""Contraction chains on the host (no GPU): variant enumeration, flop
counts against the chain oracle, selection under a workspace limit, and
the specs a chain rejects."""
import pytest

from oracle import chain as och


@pytest.fixture(scope="module")
def tcmod():
    import __graft_entry__
    __graft_entry__.build_library()
    from paper_1409_8608_gb300 import tc
    tc.load()
    return tc


def test_matrix_chain_variants_and_flops(tcmod):
    spec, ext = "ad=ab,bc,cd", [512, 8, 8, 512]  # a, d, b, c
    ch = tcmod.Chain(spec, ext, "f64")
    vs = ch.variants()
    # X and Z share no index: only (X Y) Z and X (Y Z), each plain and sliced
    assert {v["first"] for v in vs} == {(0, 1), (1, 2)}
    for v in vs:
        assert v["flops"] == och.chain_flops(spec, ext, v["first"])
        assert v["predicted_seconds"] < 0
    plain = [v for v in vs if v["sliced"] is None]
    assert len(plain) == 2
    # fewest flops, and unsliced before sliced
    sel = vs[ch.selected()]
    assert sel["first"] == (1, 2) and sel["sliced"] is None
    # intermediates: (X Y) is a x c, (Y Z) is b x d
    by = {(v["first"], v["sliced"]): v for v in vs}
    assert by[((0, 1), None)]["workspace_bytes"] == 512 * 512 * 8
    assert by[((1, 2), None)]["workspace_bytes"] == 8 * 8 * 8
    assert by[((0, 1), "a")]["slices"] == 512 and by[((0, 1), "a")]["workspace_bytes"] == 512 * 8
    ch.close()


def test_workspace_limit_selects_a_sliced_variant(tcmod):
    spec, ext = "abc=ai,ij,jbc", [64, 32, 16, 8, 8]  # a, b, c, i, j
    ch = tcmod.Chain(spec, ext, "f32")
    vs = ch.variants()
    plain_bytes = min(v["workspace_bytes"] for v in vs if v["sliced"] is None)
    ch.set_workspace_limit(plain_bytes - 1)
    ch.select(-1)
    sel = vs[ch.selected()]
    assert sel["sliced"] is not None and sel["workspace_bytes"] < plain_bytes
    big = next(i for i, v in enumerate(vs) if v["workspace_bytes"] >= plain_bytes)
    with pytest.raises(tcmod.TcError):
        ch.select(big)
    ch.set_workspace_limit(1)
    with pytest.raises(tcmod.TcError):
        ch.select(-1)
    ch.close()


@pytest.mark.parametrize("spec,ext,dtype", [
    ("ad=abe,bc,cd", [2, 2, 2, 2, 2], "f64"),   # e summed within one operand
    ("ad=ab,bc", [2, 2, 2, 2], "f64"),          # two operands
    ("ad=ab,bc,cd,de", [2] * 5, "f64"),         # four operands
    ("aD=ab,bc,cD", [2, 2, 2, 2], "f64"),       # not a-z
    ("ad=abb,bc,cd", [2, 2, 2, 2], "f64"),      # repeated within an operand
    ("ad=ab,bc,cd", [2, 0, 2, 2], "f64"),       # extent 0
    ("ad=ab,bc,cd", [2, 2, 2, 2], "bf16"),      # 16-bit inputs
])
def test_rejected_chains(tcmod, spec, ext, dtype):
    with pytest.raises(tcmod.TcError):
        tcmod.Chain(spec, ext, dtype)


def test_index_in_all_three_operands(tcmod):
    # i in X, Y and Z: a batch index of the first step, contracted in the second
    spec, ext = "ab=ai,ij,jbi", [6, 5, 4, 3]
    ch = tcmod.Chain(spec, ext, "f64")
    vs = ch.variants()
    assert vs and all(v["flops"] == och.chain_flops(spec, ext, v["first"]) for v in vs)
    ch.close()
