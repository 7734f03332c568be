"""Parity of the GPU foreign-key joins (§4.2.1) with the oracle, byte for byte:
DPG-move and the direct baseline against oracle.fk_join_move, DPG-sort
against oracle.fk_join_sorted; Zipf and uniform keys, several row layouts,
bad keys, and a large sampled case."""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda", 0)


@pytest.fixture(scope="module")
def ctx():
    from paper_cs_0308004_gb300 import dpg
    c = dpg.Context(0)
    yield c
    c.close()


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def relayout(dim, fact, fk, fact_bytes, fk_off, dim_bytes, pk_off, seed=1):
    """Same keys, other row widths and key offsets."""
    n_dim, n_fact = dim.shape[0], fact.shape[0]
    d = synth.records(n_dim, dim_bytes, seed).copy()
    d[:, pk_off:pk_off + 8] = np.arange(n_dim, dtype="<i8").view(np.uint8).reshape(n_dim, 8)
    f = synth.records(n_fact, fact_bytes, seed + 1).copy()
    f[:, fk_off:fk_off + 4] = fk.astype("<i4").view(np.uint8).reshape(n_fact, 4)
    return d, f


def run_all(ctx, dim, fact, fk_off=0, pk_off=0):
    want_move = oracle.fk_join_move(fact, dim, fk_off, pk_off)
    want_sort = oracle.fk_join_sorted(fact, dim, fk_off, pk_off)
    d_dim, d_fact = to_dev(dim), to_dev(fact)
    for mode, want in (("move", want_move), ("direct", want_move), ("sort", want_sort)):
        out = torch.full(want.shape, 0xA5, dtype=torch.uint8, device=DEV)
        ctx.fk_join(d_fact, d_dim, mode, fk_off, pk_off, out=out)
        ctx.sync()
        got = out.cpu().numpy()
        if not np.array_equal(got, want):
            bad = np.nonzero(np.any(got != want, axis=1))[0]
            raise AssertionError(f"{mode}: {bad.size} rows differ, first {bad[:5]}")


@pytest.mark.parametrize("s", [0.8, 1.3, 0.0])
@pytest.mark.parametrize("n_dim,n_fact", [(1, 5), (7, 1000), (1000, 100_003), (100_000, 1_000_003), (300, 70_000)])
def test_join_matches_oracle(ctx, n_dim, n_fact, s):
    dim, fact, fk = synth.fk_tables(n_dim, n_fact, 64, 16, s, 4 + n_dim)
    run_all(ctx, dim, fact)


@pytest.mark.parametrize("run_kb", ["64", "4096"])
@pytest.mark.parametrize("variant", ["2", "3", "4"])
def test_join_retrieval_plans(ctx, monkeypatch, variant, run_kb):
    """The same join rows whatever retrieval plan is set: the L2-run plan
    (DPG-move rows through INTERNAL slots with the key check in Phase II,
    DPG-sort rows rebuilt tile by tile), the 3-pass plan, and the 2-pass
    plan, which falls back to the 3-pass plan because join rows need
    INTERNAL."""
    monkeypatch.setenv("DPG_VARIANT", variant)
    monkeypatch.setenv("DPG_L2_RUN_KB", run_kb)
    dim, fact, fk = synth.fk_tables(5000, 200_000, 64, 16, 0.8, 9)
    run_all(ctx, dim, fact)


@pytest.mark.parametrize("slot", ["0", "1"])
def test_join_sort_phase3_paths(ctx, monkeypatch, slot):
    """DPG-sort join rows on the L2-run plan, both Phase III paths: fact rows
    of up to 128 bytes rebuilt tile by tile with their dimension rows
    appended, larger ones (and all with DPG_L2_SLOT=1) gathered through
    INTERNAL slots; every layout against the oracle, a ragged last tile."""
    monkeypatch.setenv("DPG_VARIANT", "4")
    monkeypatch.setenv("DPG_L2_SLOT", slot)
    dim, fact, fk = synth.fk_tables(3000, 100_003, 64, 16, 0.8, 21)
    for fb, fo, db, po in ((16, 0, 64, 0), (24, 8, 40, 16), (12, 4, 20, 12), (128, 0, 64, 0), (132, 4, 64, 0),
                           (4, 0, 8, 0), (16, 12, 100, 3), (20, 0, 9, 1)):
        d, f = relayout(dim, fact, fk, fb, fo, db, po)
        want = oracle.fk_join_sorted(f, d, fo, po)
        out = ctx.fk_join(to_dev(f), to_dev(d), "sort", fo, po)
        ctx.sync()
        assert np.array_equal(out.cpu().numpy(), want), (fb, fo, db, po)


@pytest.mark.parametrize("variant", ["3", "4"])
def test_join_sort_four_key_bytes(ctx, monkeypatch, variant):
    """More than 2**24 dimension rows: the DPG-sort join sorts its 8-byte
    pairs on all four bytes of the foreign key (keys whose top byte is set,
    repeated keys, a ragged last tile); rows against the oracle."""
    monkeypatch.setenv("DPG_VARIANT", variant)
    n_dim, n_fact = (1 << 24) + 5, 200_003
    d = np.arange(n_dim, dtype="<i8").view(np.uint8).reshape(n_dim, 8)     # 8-byte rows: the key alone
    fk = synth.uniform_ids(n_fact, n_dim, 31).astype(np.int64)
    fk[:4] = [n_dim - 1, 0, 1 << 24, (1 << 24) + 2]
    fk[100:140] = fk[7]                                                     # a run of equal keys
    f = synth.records(n_fact, 16, 32).copy()
    f[:, :4] = fk.astype("<i4").view(np.uint8).reshape(n_fact, 4)
    want = oracle.fk_join_sorted(f, d)
    out = ctx.fk_join(to_dev(f), to_dev(d), "sort")
    ctx.sync()
    assert np.array_equal(out.cpu().numpy(), want)


@pytest.mark.parametrize("mode", ["move", "sort"])
@pytest.mark.parametrize("variant", ["3", "4"])
def test_join_bad_keys_each_plan(ctx, monkeypatch, variant, mode):
    """A referenced dimension row whose key is not its row number, one byte
    off at several places of the key: reported on either plan; DPG-move
    reports it before writing any output row."""
    from paper_cs_0308004_gb300 import dpg
    monkeypatch.setenv("DPG_VARIANT", variant)
    dim, fact, fk = synth.fk_tables(3000, 80_000, 64, 16, 0.8, 12)
    for pk_off, dim_bytes, flip in ((0, 64, 2), (3, 100, 2), (56, 64, 2), (0, 64, 7), (3, 100, 5), (8, 40, 0)):
        d, f = relayout(dim, fact, fk, 16, 0, dim_bytes, pk_off)
        d[int(fk[123]), pk_off + flip] ^= 0x40                           # one byte of one referenced key
        out = torch.full((80_000, 16 + dim_bytes), 0x33, dtype=torch.uint8, device=DEV)
        ctx.fk_join(to_dev(f), to_dev(d), mode, 0, pk_off, out=out)
        with pytest.raises(dpg.DpgRangeError):
            ctx.sync()
        if mode == "move":
            assert bool((out == 0x33).all())


@pytest.mark.parametrize("fact_bytes,fk_off,dim_bytes,pk_off", [(24, 8, 40, 16), (4, 0, 8, 0), (12, 4, 20, 12),
                                                                 (64, 60, 256, 248), (16, 12, 100, 3)])
def test_join_layouts(ctx, fact_bytes, fk_off, dim_bytes, pk_off):
    dim, fact, fk = synth.fk_tables(20_000, 300_007, 64, 16, 0.8, 5)
    d, f = relayout(dim, fact, fk, fact_bytes, fk_off, dim_bytes, pk_off)
    run_all(ctx, d, f, fk_off, pk_off)


def test_join_bad_keys(ctx):
    from paper_cs_0308004_gb300 import dpg
    dim, fact, fk = synth.fk_tables(1000, 50_000, 64, 16, 0.8, 6)
    bad = fact.copy()
    bad[777, :4] = np.array([1000], "<i4").view(np.uint8)        # fk out of range
    for mode in ("move", "sort", "direct"):
        out = torch.full((50_000, 80), 0x33, dtype=torch.uint8, device=DEV)
        ctx.fk_join(to_dev(bad), to_dev(dim), mode, out=out)
        with pytest.raises(dpg.DpgRangeError):
            ctx.sync()
        if mode != "direct":
            assert bool((out == 0x33).all()), mode
    dim2 = dim.copy()
    dim2[int(fk[10]), :8] = np.array([123456], "<i8").view(np.uint8)  # a referenced key is not its row number
    for mode in ("move", "sort", "direct"):
        out = torch.full((50_000, 80), 0x33, dtype=torch.uint8, device=DEV)
        ctx.fk_join(to_dev(fact), to_dev(dim2), mode, out=out)
        with pytest.raises(dpg.DpgRangeError):
            ctx.sync()
        if mode == "move":
            assert bool((out == 0x33).all())
    empty_dim = torch.zeros((0, 64), dtype=torch.uint8, device=DEV)
    for mode in ("move", "sort", "direct"):
        ctx.fk_join(to_dev(fact[:10]), empty_dim, mode)
        with pytest.raises(dpg.DpgRangeError):
            ctx.sync()
    ctx.sync()


def test_join_large_every_row(ctx):
    """2,000,000 dimension rows x 20,000,000 fact rows, Zipf 0.8: every row of
    the move join against oracle.fk_join_move and every row of the sort join
    against oracle.fk_join_sorted (the (fk, fact row) order of §4.2.1)."""
    n_dim, n_fact = 2_000_000, 20_000_000
    dim, fact, fk = synth.fk_tables(n_dim, n_fact, 64, 16, 0.8, 4)
    fact = fact.copy()
    fact[:, 4:8] = np.arange(n_fact, dtype="<u4").view(np.uint8).reshape(n_fact, 4)  # row ids in the payload
    d_dim, d_fact = to_dev(dim), to_dev(fact)
    move = ctx.fk_join(d_fact, d_dim, "move")
    ctx.sync()
    assert torch.equal(move, to_dev(oracle.fk_join_move(fact, dim)))
    del move
    srt = ctx.fk_join(d_fact, d_dim, "sort")
    ctx.sync()
    assert torch.equal(srt, to_dev(oracle.fk_join_sorted(fact, dim)))


@pytest.mark.parametrize("mode,dim_bytes,variant", [("move", 64, 4), ("sort", 64, 4), ("move", 256, 3)])
def test_join_default_plans(ctx, monkeypatch, mode, dim_bytes, variant):
    """Untuned joins: the L2-run plan, except DPG-move of dimension rows of
    192 bytes and more (the 3-pass plan)."""
    for name in ("DPG_VARIANT", "DPG_SEG_LOG2", "DPG_CHUNK", "DPG_L2_RUN_KB", "DPG_L2_SLOT"):
        monkeypatch.delenv(name, raising=False)
    dim, fact, fk = synth.fk_tables(4000, 90_001, dim_bytes, 16, 0.8, 13)
    want = oracle.fk_join_sorted(fact, dim) if mode == "sort" else oracle.fk_join_move(fact, dim)
    out = ctx.fk_join(to_dev(fact), to_dev(dim), mode)
    ctx.sync()
    assert ctx.last_plan()[0] == variant
    assert np.array_equal(out.cpu().numpy(), want)
