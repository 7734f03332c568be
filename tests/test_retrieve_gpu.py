"""Parity of the CUDA retrieval path with the oracle, byte for byte.

Every case compares dpg_retrieve (distribute-probe-gather: the L2-run plan and
the 3-pass and 2-pass shared-memory plans) and dpg_retrieve_direct with
oracle.retrieve on the same
seeded inputs: permutations, duplicates and skew (§2, §2.3), record sizes from
1 to 4096 bytes, ragged tails, unaligned tables, forced small segments (the
global-counter path and chunk splitting), empty and degenerate inputs, bad
rids, and the 1,000,000 x 100-byte workload in full (the larger workloads are
compared row by row in test_full_size_gpu.py).
"""
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


def rid_sequence(kind, n_src, n, seed):
    if kind == "perm":
        return synth.permutation(n_src, seed)[:n] if n <= n_src else synth.uniform_ids(n, n_src, seed)
    if kind == "dup":
        return synth.uniform_ids(n, n_src, seed)
    if kind == "skew":
        return synth.take(synth.zipf_ranks(n, n_src, 1.1, seed), synth.permutation(n_src, seed + 1))
    if kind == "same":
        return np.full(n, n_src // 2, dtype=np.int32)
    raise ValueError(kind)


def check(ctx, src, rids, variants=("dpg", "direct")):
    want = oracle.retrieve(src, rids)
    d_src, d_rids = to_dev(src), to_dev(rids)
    for v in variants:
        out = torch.full((rids.size, src.shape[1]), 0xA5, dtype=torch.uint8, device=DEV)
        fn = ctx.retrieve if v == "dpg" else ctx.retrieve_direct
        fn(d_src, d_rids, out=out)
        ctx.sync()
        got = out.cpu().numpy()
        if not np.array_equal(got, want):
            bad = np.nonzero(np.any(got != want, axis=1))[0]
            raise AssertionError(f"{v}: {bad.size} records differ, first at {bad[:5]}")


RECS = [1, 2, 3, 4, 7, 8, 12, 16, 17, 20, 24, 32, 40, 64, 100, 128, 255, 256, 1000, 4096]


@pytest.mark.parametrize("variant", ["3", "2", "4"])
@pytest.mark.parametrize("kind", ["perm", "dup", "skew"])
@pytest.mark.parametrize("rec", RECS)
def test_retrieve_matches_oracle(ctx, monkeypatch, rec, kind, variant):
    monkeypatch.setenv("DPG_VARIANT", variant)
    monkeypatch.setenv("DPG_L2_RUN_KB", "256")   # several L2 runs at these sizes
    n_src = max(37, min(60000, (3 << 20) // rec)) | 1       # several segments and a ragged tail
    n = n_src + 333 if kind != "perm" else n_src
    src = synth.records(n_src, rec, rec)
    check(ctx, src, rid_sequence(kind, n_src, n, 7 + rec))


@pytest.mark.parametrize("variant", ["3", "2"])
@pytest.mark.parametrize("seg_log2,chunk", [(0, 0), (1, 3), (3, 5), (5, 1000), (7, 64)])
def test_forced_small_segments(ctx, monkeypatch, seg_log2, chunk, variant):
    """Tiny segments give more segments than shared-memory counters (global
    counter path); small chunks split every run into many probe items."""
    monkeypatch.setenv("DPG_VARIANT", variant)
    monkeypatch.setenv("DPG_SEG_LOG2", str(seg_log2))
    monkeypatch.setenv("DPG_CHUNK", str(chunk))
    n_src, rec = 50001, 12
    src = synth.records(n_src, rec, 3)
    for kind in ("perm", "dup", "same"):
        check(ctx, src, rid_sequence(kind, n_src, 70001 if kind != "perm" else n_src, 9), variants=("dpg",))


@pytest.mark.parametrize("run_kb", ["1", "64", "100000"])
def test_l2_runs(ctx, monkeypatch, run_kb):
    """L2-run plan: one run, a few runs, and the run-count cap (1024 runs)."""
    monkeypatch.setenv("DPG_VARIANT", "4")
    monkeypatch.setenv("DPG_L2_RUN_KB", run_kb)
    for n_src, rec in ((200_003, 16), (50_001, 100), (3001, 1000)):
        src = synth.records(n_src, rec, 11)
        for kind in ("perm", "dup", "same"):
            check(ctx, src, rid_sequence(kind, n_src, 120_001 if kind != "perm" else n_src, 4), variants=("dpg",))


@pytest.mark.parametrize("slot", ["0", "1"])
@pytest.mark.parametrize("rec", [1, 8, 16, 24, 32, 64, 95, 96, 100, 128, 129, 255, 1000])
def test_l2_runs_phase3_modes(ctx, monkeypatch, rec, slot):
    """L2-run plan with either Phase III forced at every record size: the
    4-byte slot gather, or the tile rebuild (shared-memory staging up to 128-byte
    records, straight copies through the inverse tile places above)."""
    monkeypatch.setenv("DPG_VARIANT", "4")
    monkeypatch.setenv("DPG_L2_RUN_KB", "512")
    monkeypatch.setenv("DPG_L2_SLOT", slot)
    n_src = max(37, min(90_001, (4 << 20) // rec)) | 1
    src = synth.records(n_src, rec, 17 + rec)
    for kind, n in (("perm", n_src), ("dup", n_src + 4097), ("skew", 20_011)):
        check(ctx, src, rid_sequence(kind, n_src, n, 3 + rec), variants=("dpg",))


@pytest.mark.parametrize("stage_max", ["0", "16384"])
def test_l2_runs_unstaged_and_small_stage(ctx, monkeypatch, stage_max):
    """Tile rebuild without shared-memory staging (stage budget 0) and with
    smaller tiles (16 KB budget), small records."""
    monkeypatch.setenv("DPG_VARIANT", "4")
    monkeypatch.setenv("DPG_L2_RUN_KB", "256")
    monkeypatch.setenv("DPG_L2_SLOT", "0")
    monkeypatch.setenv("DPG_UNPART_STAGE_MAX", stage_max)
    for rec in (4, 16, 32, 48, 64):
        n_src = 50_001
        src = synth.records(n_src, rec, rec)
        check(ctx, src, rid_sequence("dup", n_src, 70_003, rec), variants=("dpg",))


@pytest.mark.parametrize("rid_off", [0, 1, 2, 3])
@pytest.mark.parametrize("n", [4095, 4096, 4097, 12_289, 100_003])
def test_l2_runs_rid_alignment_and_tiles(ctx, monkeypatch, rid_off, n):
    """Rid arrays at every 4-byte offset from a 16-byte boundary (vector and
    scalar histogram paths) and rid counts around the 4096-rid tile and range
    sizes (partial last tiles)."""
    monkeypatch.setenv("DPG_VARIANT", "4")
    monkeypatch.setenv("DPG_L2_RUN_KB", "128")
    n_src, rec = 33_333, 16
    src = synth.records(n_src, rec, 5)
    rids = synth.uniform_ids(n, n_src, n + rid_off)
    want = oracle.retrieve(src, rids)
    big = torch.zeros(n + 8, dtype=torch.int32, device=DEV)
    d_rids = big[rid_off:rid_off + n]
    d_rids.copy_(to_dev(rids))
    out = ctx.retrieve(to_dev(src), d_rids)
    ctx.sync()
    assert np.array_equal(out.cpu().numpy(), want)


@pytest.mark.parametrize("variant", ["3", "4"])
@pytest.mark.parametrize("n_src,n", [(1, 1), (1, 1000), (2, 1), (5, 3), (1000, 1), (70000, 2)])
def test_small_and_degenerate(ctx, monkeypatch, n_src, n, variant):
    monkeypatch.setenv("DPG_VARIANT", variant)
    for rec in (1, 4, 100):
        src = synth.records(n_src, rec, n_src)
        check(ctx, src, synth.uniform_ids(n, n_src, n))


def test_empty(ctx):
    src = to_dev(synth.records(10, 8, 1))
    out = ctx.retrieve(src, torch.zeros(0, dtype=torch.int32, device=DEV))
    ctx.retrieve_direct(src, torch.zeros(0, dtype=torch.int32, device=DEV))
    ctx.sync()
    assert out.shape == (0, 8)
    empty = torch.zeros((0, 8), dtype=torch.uint8, device=DEV)
    ctx.retrieve(empty, torch.zeros(0, dtype=torch.int32, device=DEV))
    ctx.sync()


@pytest.mark.parametrize("variant", ["3", "4"])
@pytest.mark.parametrize("src_off,dst_off", [(1, 0), (0, 3), (4, 8), (8, 4), (2, 6), (16, 1)])
def test_unaligned_tables(ctx, monkeypatch, src_off, dst_off, variant):
    monkeypatch.setenv("DPG_VARIANT", variant)
    monkeypatch.setenv("DPG_L2_RUN_KB", "64")
    n_src, n = 9001, 12000
    for rec in (16, 100, 64):
        src = synth.records(n_src, rec, 5)
        rids = synth.uniform_ids(n, n_src, 6)
        want = oracle.retrieve(src, rids)
        big = torch.zeros(n_src * rec + 64, dtype=torch.uint8, device=DEV)
        d_src = big[src_off:src_off + n_src * rec].view(n_src, rec)
        d_src.copy_(to_dev(src))
        bigd = torch.zeros(n * rec + 64, dtype=torch.uint8, device=DEV)
        d_dst = bigd[dst_off:dst_off + n * rec].view(n, rec)
        for fn in (ctx.retrieve, ctx.retrieve_direct):
            d_dst.fill_(0)
            fn(d_src, to_dev(rids), out=d_dst)
            ctx.sync()
            assert np.array_equal(d_dst.cpu().numpy(), want)
        # bytes around the destination untouched
        assert int(bigd[:dst_off].sum()) == 0 and int(bigd[dst_off + n * rec:].sum()) == 0


@pytest.mark.parametrize("variant", ["3", "2", "4"])
@pytest.mark.parametrize("bad", [-1, 5000, 2**31 - 1])
def test_bad_rid_leaves_destination_untouched(ctx, monkeypatch, bad, variant):
    from paper_cs_0308004_gb300 import dpg
    monkeypatch.setenv("DPG_VARIANT", variant)
    n_src, rec = 5000, 100
    src = to_dev(synth.records(n_src, rec, 1))
    rids = synth.uniform_ids(20000, n_src, 2)
    rids[12345] = bad
    out = torch.full((rids.size, rec), 0x5A, dtype=torch.uint8, device=DEV)
    ctx.retrieve(src, to_dev(rids), out=out)
    with pytest.raises(dpg.DpgRangeError):
        ctx.sync()
    assert bool((out == 0x5A).all())
    ctx.retrieve_direct(src, to_dev(rids), out=out)
    with pytest.raises(dpg.DpgRangeError):
        ctx.sync()
    ctx.sync()  # the error was cleared
    # the direct gather copies every record whose rid is valid
    good = np.ones(rids.size, bool)
    good[12345] = False
    want = oracle.retrieve(src.cpu().numpy(), np.where(good, rids, 0))
    assert np.array_equal(out.cpu().numpy()[good], want[good])
    # an empty source table: every rid is out of range
    empty = torch.zeros((0, rec), dtype=torch.uint8, device=DEV)
    ctx.retrieve(empty, to_dev(np.zeros(3, np.int32)))
    with pytest.raises(dpg.DpgRangeError):
        ctx.sync()


@pytest.mark.parametrize("rec", [17, 20, 24, 100, 1000])
def test_direct_bad_rids_copy_the_valid_records(ctx, rec):
    """Bad rids next to each other and at the ends: every other record is
    copied, the bad ones keep the destination's bytes (§1 baseline)."""
    from paper_cs_0308004_gb300 import dpg
    n_src, n = 3001, 4099
    src = synth.records(n_src, rec, 3)
    rids = synth.uniform_ids(n, n_src, 4)
    bad_at = [0, 1, 2, 777, 778, 2000, n - 2, n - 1]
    rids[bad_at] = [n_src, -5, n_src + 7, 2**31 - 1, n_src, -1, n_src, n_src]
    out = torch.full((n, rec), 0x3C, dtype=torch.uint8, device=DEV)
    ctx.retrieve_direct(to_dev(src), to_dev(rids), out=out)
    with pytest.raises(dpg.DpgRangeError):
        ctx.sync()
    good = np.ones(n, bool)
    good[bad_at] = False
    got = out.cpu().numpy()
    assert np.array_equal(got[good], oracle.retrieve(src, np.where(good, rids, 0))[good])
    assert bool((got[~good] == 0x3C).all())


def test_argument_errors(ctx):
    from paper_cs_0308004_gb300 import dpg
    buf = torch.zeros(1000 * 10, dtype=torch.uint8, device=DEV)
    src = buf[:5000].view(500, 10)
    rids = torch.zeros(300, dtype=torch.int32, device=DEV)
    with pytest.raises(dpg.DpgError):
        ctx.retrieve(src, rids, out=buf[4000:7000].view(300, 10))   # overlaps src
    with pytest.raises(dpg.DpgError):
        ctx.retrieve(torch.zeros((5, 0), dtype=torch.uint8, device=DEV), rids[:0].clone(),
                     out=torch.zeros((0, 0), dtype=torch.uint8, device=DEV))
    with pytest.raises(ValueError):
        ctx.retrieve(src.cpu(), rids)
    with pytest.raises(dpg.DpgError):
        ctx.retrieve(torch.zeros((2, 70000), dtype=torch.uint8, device=DEV), rids[:1].clone())


@pytest.mark.parametrize("variant", ["3", "4"])
def test_config1_full_size(ctx, monkeypatch, variant):
    """1,000,000 records of 100 bytes, a random permutation: full comparison."""
    monkeypatch.setenv("DPG_VARIANT", variant)
    src, rids = synth.plain_retrieval(1_000_000, 100, 1, 2)
    check(ctx, src, rids)
    check(ctx, src, synth.uniform_ids(1_000_000, 1_000_000, 5))


# ------------------------------------------------------------ sort copy (§3)

@pytest.mark.parametrize("variant", ["3", "4"])
@pytest.mark.parametrize("rec", [16, 32, 64, 100, 256])
def test_sort_copy_matches_oracle(ctx, monkeypatch, rec, variant):
    monkeypatch.setenv("DPG_VARIANT", variant)
    monkeypatch.setenv("DPG_L2_RUN_KB", "1024")
    n = 200_003
    src = synth.sort_file(n, rec, 3)
    pairs = oracle.sort_keyptr(src, 10)
    want = oracle.sort_copy(pairs, src)
    d_src, d_pairs = to_dev(src), to_dev(pairs)
    for fn in (ctx.sort_copy, ctx.sort_copy_direct):
        out = fn(d_pairs, d_src)
        ctx.sync()
        assert np.array_equal(out.cpu().numpy(), want)


def test_sort_copy_other_pair_layouts(ctx):
    n_src, rec = 30001, 24
    src = synth.records(n_src, rec, 4)
    rids = synth.uniform_ids(40000, n_src, 5)
    want = oracle.retrieve(src, rids)
    for stride, off in ((4, 0), (8, 4), (12, 0), (32, 20)):
        pairs = np.zeros((rids.size, stride), np.uint8)
        pairs[:, off:off + 4] = rids.astype("<i4").view(np.uint8).reshape(-1, 4)
        for fn in (ctx.sort_copy, ctx.sort_copy_direct):
            out = fn(to_dev(pairs), to_dev(src), rid_off=off)
            ctx.sync()
            assert np.array_equal(out.cpu().numpy(), want)


@pytest.mark.parametrize("rec,stride", [(16, 4), (100, 4), (100, 16), (256, 4)])
def test_tune_then_retrieve(rec, stride):
    """dpg_tune caches a plan per shape; later retrievals use it and still match the oracle."""
    from paper_cs_0308004_gb300 import dpg
    with dpg.Context(0) as c:
        n_src = 200_003
        src = synth.records(n_src, rec, 3)
        rids = synth.permutation(n_src, 4)
        d_src = to_dev(src)
        if stride == 4:
            d_rids = to_dev(rids)
            v, sl = c.tune(d_src, d_rids)
        else:
            pairs = np.zeros((n_src, 16), np.uint8)
            pairs[:, 12:16] = rids.astype("<i4").view(np.uint8).reshape(-1, 4)
            d_rids = to_dev(pairs)
            v, sl = c.tune(d_src, d_rids, rid_stride=16, rid_off=12)
        assert v in (2, 3, 4)
        out = c.retrieve(d_src, to_dev(rids)) if stride == 4 else c.sort_copy(d_rids, d_src)
        c.sync()
        assert c.last_plan() == (v, sl)
        assert np.array_equal(out.cpu().numpy(), oracle.retrieve(src, rids))


@pytest.mark.parametrize("rec,variant", [(8, 4), (16, 4), (100, 4), (191, 4), (192, 2), (256, 2), (1000, 2)])
def test_untuned_plan_by_record_size(monkeypatch, rec, variant):
    """Without a tuned plan or overrides a retrieval takes the plan its record
    size calls for (L2 runs below 192 bytes, 2-pass from 192), and still
    matches the oracle."""
    from paper_cs_0308004_gb300 import dpg
    for name in ("DPG_VARIANT", "DPG_SEG_LOG2", "DPG_CHUNK", "DPG_L2_RUN_KB", "DPG_L2_SLOT"):
        monkeypatch.delenv(name, raising=False)
    with dpg.Context(0) as c:
        n_src = 30_011
        src = synth.records(n_src, rec, 8)
        rids = synth.uniform_ids(40_009, n_src, 9)
        out = c.retrieve(to_dev(src), to_dev(rids))
        c.sync()
        assert c.last_plan()[0] == variant
        assert np.array_equal(out.cpu().numpy(), oracle.retrieve(src, rids))
