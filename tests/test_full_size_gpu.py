"""Byte-exact parity at the full sizes of the workloads, every output row
against the oracle (no sampling):

* the sort copy phase of §3 over 10,000,000 x 100-byte records (1e9 B), on the
  tuned plan, the L2-run plan, the 3-pass plan and the direct gather, and the
  whole sort (dpg_sort_records);
* the record-size sweep: 1e9 bytes of source at 16, 32, 64, 100 and 256-byte
  records, rids a permutation, on the default plan, the tuned plan and the
  direct gather;
* the foreign-key join of §4.2.1, 200,000,000 x 16-byte fact rows (Zipf 0.8
  keys) with 10,000,000 x 64-byte dimension rows (16 GB of output), in all
  three modes, compared in chunks of 10,000,000 rows with oracle.fk_join_move
  (DPG-move, direct) and with the move rows of the fact rows in
  oracle.fk_join_order's order (DPG-sort);
* the batch of 4096 requests (record counts log-uniform in [1e3, 1.6e7],
  8..256-byte records, 611 GB of output) in the benchmark's waves, every
  request against the oracle.

Comparisons run on the device (the oracle's result copied over, then
compared element by element), so the 1-16 GB outputs need not come back.
"""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

DEV = torch.device("cuda", 0)
CHUNK = 10_000_000


@pytest.fixture(scope="module")
def ctx():
    from paper_cs_0308004_gb300 import dpg
    c = dpg.Context(0)
    yield c
    c.close()


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def assert_rows_equal(got: torch.Tensor, want: np.ndarray, what: str, row0: int = 0):
    w = to_dev(want)
    if not torch.equal(got, w):
        bad = torch.nonzero((got != w).any(dim=1)).reshape(-1)
        raise AssertionError(f"{what}: {bad.numel()} of {want.shape[0]} rows differ, first at "
                             f"{(bad[:5] + row0).tolist()}")


def set_plan(monkeypatch, plan):
    for name in ("DPG_VARIANT", "DPG_SEG_LOG2", "DPG_CHUNK", "DPG_L2_RUN_KB", "DPG_L2_SLOT"):
        monkeypatch.delenv(name, raising=False)
    if plan in ("2", "3", "4"):
        monkeypatch.setenv("DPG_VARIANT", plan)


# ----------------------------------------------------- sort copy phase (§3)

@pytest.fixture(scope="module")
def sort_case():
    n, rec = 10_000_000, 100
    src = synth.sort_file(n, rec, 3)
    pairs = oracle.sort_keyptr(src, 10)
    want = oracle.sort_copy(pairs, src)
    return src, pairs, want


@pytest.mark.parametrize("plan", ["default", "tuned", "4", "3", "2", "direct"])
def test_sort_copy_full_size_every_row(ctx, monkeypatch, sort_case, plan):
    """All 10,000,000 output rows of the sort copy phase against the oracle."""
    src, pairs, want = sort_case
    set_plan(monkeypatch, plan)
    d_src, d_pairs = to_dev(src), to_dev(pairs)
    out = torch.full((src.shape[0], src.shape[1]), 0xA5, dtype=torch.uint8, device=DEV)
    if plan == "direct":
        ctx.sort_copy_direct(d_pairs, d_src, out=out)
    else:
        if plan == "tuned":
            ctx.tune(d_src, d_pairs, out, rid_stride=16, rid_off=12)
        ctx.sort_copy(d_pairs, d_src, out=out)
    ctx.sync()
    assert_rows_equal(out, want, f"sort copy, plan {plan}")


def test_sort_records_full_size_every_row(ctx, sort_case):
    """The whole GPU sort (pairs, ten radix passes, DPG copy) against the oracle's sort."""
    src, pairs, want = sort_case
    d_src = to_dev(src)
    got_pairs = ctx.sort_keyptr(d_src, 10)
    ctx.sync()
    assert_rows_equal(got_pairs, pairs, "sorted key-pointer pairs")
    del got_pairs
    out = ctx.sort_records(d_src, 10)
    ctx.sync()
    assert_rows_equal(out, want, "sorted records")


# ------------------------------------------------------- record-size sweep

@pytest.mark.parametrize("rec", [16, 32, 64, 100, 256])
def test_sweep_full_size_every_row(ctx, monkeypatch, rec):
    """1e9 bytes of source at each sweep record size, rids a permutation: the
    default plan, the tuned plan and the direct gather, every row."""
    set_plan(monkeypatch, "default")
    n = 1_000_000_000 // rec
    src = synth.records(n, rec, 3)
    rids = synth.permutation(n, 2)
    want = oracle.retrieve(src, rids)
    d_src, d_rids = to_dev(src), to_dev(rids)
    del src
    out = torch.empty((n, rec), dtype=torch.uint8, device=DEV)
    for what in ("default", "direct", "tuned"):
        out.fill_(0x5A)
        if what == "direct":
            ctx.retrieve_direct(d_src, d_rids, out=out)
        else:
            if what == "tuned":
                ctx.tune(d_src, d_rids, out)
                out.fill_(0x5A)
            ctx.retrieve(d_src, d_rids, out=out)
        ctx.sync()
        assert_rows_equal(out, want, f"{rec}-byte records, {what}")


# ------------------------------------------------- foreign-key join (§4.2.1)

@pytest.fixture(scope="module")
def join_case():
    n_dim, n_fact = 10_000_000, 200_000_000
    dim, fact, fk = synth.fk_tables(n_dim, n_fact, 64, 16, 0.8, 4)
    return dim, fact


@pytest.mark.parametrize("mode", ["move", "sort", "direct"])
def test_join_full_size_every_row(ctx, monkeypatch, join_case, mode):
    """The 2e8-row join in every mode, all 200,000,000 rows, chunk by chunk."""
    set_plan(monkeypatch, "default")
    dim, fact = join_case
    n_fact = fact.shape[0]
    d_dim, d_fact = to_dev(dim), to_dev(fact)
    out = torch.full((n_fact, 80), 0x33, dtype=torch.uint8, device=DEV)
    ctx.fk_join(d_fact, d_dim, mode, out=out)
    ctx.sync()
    del d_fact
    order = oracle.fk_join_order(fact, dim.shape[0]) if mode == "sort" else None
    for j0 in range(0, n_fact, CHUNK):
        j1 = min(n_fact, j0 + CHUNK)
        rows = fact[j0:j1] if order is None else fact[order[j0:j1]]
        assert_rows_equal(out[j0:j1], oracle.fk_join_move(rows, dim), f"join {mode}, rows {j0}..{j1}", j0)


# ---------------------------------------------------------- batched retrieval

def test_batch_full_size_every_request(ctx):
    """The 4096-request batch (seed 5: 6.9e9 records, 611 GB of output) in
    waves of at most 48 GB as the benchmark runs it, each wave one
    dpg_retrieve_batch on the persistent executor; every request's output
    against the oracle (oracle.retrieve_threads on every host core, pinned to
    oracle.retrieve by the oracle tests)."""
    import os
    n, rec, kind = synth.batch_requests(4096, 1e3, 1.6e7, 5)
    all_rids, offsets = synth.batch_rids(n, n, kind, 5)
    rows = int(n.max())
    tables = {r: synth.records(rows, r, 100 + r) for r in synth.BATCH_RECS}
    d_tab = {r: to_dev(t) for r, t in tables.items()}
    waves, cur, cur_bytes = [], [], 0
    for k in range(n.size):
        b = int(n[k]) * int(rec[k])
        if cur and cur_bytes + b > 48e9:
            waves.append(cur)
            cur, cur_bytes = [], 0
        cur.append(k)
        cur_bytes += b
    waves.append(cur)
    cores = os.cpu_count() or 1
    checked = 0
    for wave in waves:
        reqs, slices = [], []
        for r in synth.BATCH_RECS:
            ks = [k for k in wave if int(rec[k]) == r]
            if not ks:
                continue
            cat = np.concatenate([all_rids[int(offsets[k]):int(offsets[k]) + int(n[k])] for k in ks])
            d_rids = to_dev(cat)
            arena = torch.empty((cat.size, r), dtype=torch.uint8, device=DEV)
            at = 0
            for k in ks:
                m = int(n[k])
                reqs.append((d_tab[r], m, d_rids[at:at + m], arena[at:at + m]))
                slices.append((k, r, arena[at:at + m]))
                at += m
        ctx.retrieve_batch(reqs)
        ctx.sync()
        for k, r, out in slices:
            m = int(n[k])
            want = oracle.retrieve_threads(tables[r][:m], all_rids[int(offsets[k]):int(offsets[k]) + m], cores)
            assert_rows_equal(out, want, f"batch request {k} ({m} x {r} B)")
            checked += 1
        del reqs, slices, arena, d_rids
        torch.cuda.empty_cache()
    assert checked == 4096
