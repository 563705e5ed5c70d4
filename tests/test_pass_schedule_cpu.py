"""The pass schedule of the MT generation kernels is free of shared-memory
hazards (CPU; the schedule comes from the library, vmt_tune_pass_cut).

A block of eq. (stepnomod) is computed in passes separated by barriers.  Item
v (vector v of the block: VW lane words of row v // RV) reads the old x_k
(vector v), x_{k+1} (vector v + RV; for the last row the new x_0, vector
v + RV - NV), and x_{k+m} (old vector v + m RV for rows below n-m, else the
new vector v - (n-m) RV), and writes its new vector.  Two forms:

  * two copies (phase form): old words come from one copy, new ones go to
    the other, so only reads of new vectors matter -- each must have been
    written in an earlier pass;
  * one copy (in place): the old x_{k+1}, which another thread overwrites in
    the same pass, is loaded before the barrier that starts the pass (at the
    end of the previous pass, or of the previous block's last pass when that
    pass does not write those rows, "early"); every read must see the
    intended version and share no epoch (the span between two barriers) with
    a write of the same vector by another item.

The model replays three blocks of every compiled configuration.  A planted
mistake (the first-pass operands loaded without a barrier after them) must be
caught, so the model is not vacuous.
"""
import pytest

from paper_2309_16682_gb300 import build


@pytest.fixture(scope="module")
def vmt():
    build.build()
    import paper_2309_16682_gb300 as m
    m.lib()
    return m


def _replay(c, blocks=3, plant=False):
    """Errors of the schedule `c` over `blocks` blocks (empty: hazard-free).
    plant=True drops the barrier after the first pass's operand loads."""
    NV, S, RV, DV, MV, inplace, early = (c["vectors"], c["step"], c["row_vectors"], c["n_minus_m_vectors"],
                                         c["m_vectors"], c["in_place"], c["early"])
    passes = [(a, min(a + S, NV)) for a in range(0, NV, S)]
    hist = {}       # vector -> [(epoch, block)] of its writes
    reads = []      # (vector, epoch, block whose value is wanted, reading item)
    ep = 0

    def load_operands(pass_range, blk, e):
        for v in range(*pass_range):
            if v + RV < NV:
                reads.append((v + RV, e, blk - 1, v))

    if inplace and early:
        load_operands(passes[0], 1, ep)
    ep += 1                                    # the barrier after the call's head
    for blk in range(1, blocks + 1):
        if inplace and not early:
            load_operands(passes[0], blk, ep)
            if not plant:
                ep += 1
        for pi, (a, b) in enumerate(passes):
            assert b - a <= DV, "a pass holds a vector and the one it depends on"
            for v in range(a, b):
                if v + RV >= NV:
                    reads.append((v + RV - NV, ep, blk, v))          # new x_0
                if v >= DV:
                    reads.append((v - DV, ep, blk, v))               # new x_{k-(n-m)}
                elif inplace:
                    reads.append((v + MV, ep, blk - 1, v))           # old x_{k+m}, same copy
            if inplace:
                if pi + 1 < len(passes):
                    load_operands(passes[pi + 1], blk, ep)
                elif early:
                    load_operands(passes[0], blk + 1, ep)
            for v in range(a, b):
                hist.setdefault(v, []).append((ep, blk))
            ep += 1
    errors = []
    for pos, e, want, item in reads:
        if any(we == e for we, _ in hist.get(pos, [])):
            errors.append(("race", pos, e, item))
            continue
        got = 0
        for we, b in hist.get(pos, []):
            if we < e:
                got = b
        if got != want:
            errors.append(("stale", pos, e, item, got, want))
    return errors


def _configs(vmt):
    out = []
    for v in ("mt32", "mt64"):
        for m in (1, 2, 4, 8, 16):
            for i, k in enumerate(vmt.tune_kernels(v, m)):
                if k["form"] in ("phase", "inplace"):
                    out.append((v, m, i, vmt.tune_pass_cut(v, m, i)))
    return out


def test_every_compiled_schedule_is_free_of_hazards(vmt):
    cfgs = _configs(vmt)
    assert any(c["in_place"] for *_, c in cfgs) and any(not c["in_place"] for *_, c in cfgs)
    for v, m, i, c in cfgs:
        assert c["n_minus_m_vectors"] + c["m_vectors"] == c["vectors"]   # (n-m) + m rows of row_vectors each
        errs = _replay(c)
        assert not errs, (v, m, i, c, errs[:3])


def test_the_model_catches_a_missing_barrier(vmt):
    found = False
    for v, m, i, c in _configs(vmt):
        if c["in_place"]:
            assert _replay(dict(c, early=0), plant=True), (v, m, i)
            found = True
    assert found


def test_the_model_catches_an_early_load_of_rows_the_last_pass_writes(vmt):
    # 16-lane MT19937-64 in place is cut into two phases: the last pass writes
    # the rows the next block's first pass reads, so the library loads them
    # after the block's barrier; loading them during the last pass would race
    late = [(v, m, i, c) for v, m, i, c in _configs(vmt) if c["in_place"] and not c["early"]]
    assert late
    for v, m, i, c in late:
        assert _replay(dict(c, early=1)), (v, m, i)


def test_chain_form_and_sfmt_have_no_pass_cut(vmt):
    chain = [i for i, k in enumerate(vmt.tune_kernels("mt32", 16)) if k["form"] == "chain"]
    with pytest.raises(vmt.VMTError):
        vmt.tune_pass_cut("mt32", 16, chain[0])
    with pytest.raises(vmt.VMTError):
        vmt.tune_pass_cut("sfmt", 4, 0)
