"""Batched retrieval (dpg_retrieve_batch, dpg_run_batch): every request's output against the
oracle, byte for byte, for requests of uneven counts and record sizes sharing
source tables; contiguous and scattered rid lists and destinations; a bad rid
in one request; replay from a captured CUDA graph."""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda", 0)
RECS = [8, 16, 32, 64, 100, 128, 256]


@pytest.fixture(scope="module")
def ctx():
    from paper_cs_0308004_gb300 import dpg
    c = dpg.Context(0)
    yield c
    c.close()


def make_batch(count, max_n, seed, table_rows=60_000):
    """Requests over one resident table per record size; request k reads the
    first n_src_k records of its table (rids a permutation or uniform draws)."""
    rng = np.random.default_rng(seed)
    tables = {rec: synth.records(table_rows, rec, 100 + rec) for rec in RECS}
    reqs = []
    for k in range(count):
        rec = RECS[int(rng.integers(len(RECS)))]
        n = int(np.exp(rng.uniform(0, np.log(max_n))))
        if rng.random() < 0.7:
            n_src = min(n, table_rows)
            rids = synth.permutation(n_src, seed * 1000 + k)
        else:
            n_src = int(rng.integers(1, table_rows + 1))
            rids = synth.uniform_ids(n, n_src, seed * 1000 + k)
        reqs.append((rec, n_src, rids))
    return tables, reqs


def test_batch_matches_oracle_scattered(ctx):
    tables, reqs = make_batch(300, 40_000, 1)
    d_tab = {rec: torch.from_numpy(t).to(DEV) for rec, t in tables.items()}
    dev_reqs, wants = [], []
    for rec, n_src, rids in reqs:
        out = torch.full((rids.size, rec), 0xA5, dtype=torch.uint8, device=DEV)
        dev_reqs.append((d_tab[rec], n_src, torch.from_numpy(rids).to(DEV), out))
        wants.append(oracle.retrieve(tables[rec][:n_src], rids))
    ctx.retrieve_batch(dev_reqs)
    ctx.sync()
    for (src, n_src, rids, out), want in zip(dev_reqs, wants):
        assert np.array_equal(out.cpu().numpy(), want)


def contiguous_layout(tables, reqs):
    """All rids of one record size back to back, destinations back to back."""
    d_tab = {rec: torch.from_numpy(t).to(DEV) for rec, t in tables.items()}
    dev_reqs = []
    for rec in RECS:
        mine = [(n_src, rids) for r, n_src, rids in reqs if r == rec]
        if not mine:
            continue
        all_rids = torch.from_numpy(np.concatenate([x[1] for x in mine])).to(DEV)
        arena = torch.full((all_rids.numel(), rec), 0xA5, dtype=torch.uint8, device=DEV)
        at = 0
        for n_src, rids in mine:
            dev_reqs.append((d_tab[rec], n_src, all_rids[at:at + rids.size], arena[at:at + rids.size]))
            at += rids.size
    return dev_reqs


def test_batch_contiguous_and_graph_replay(ctx):
    tables, reqs = make_batch(200, 30_000, 2)
    dev_reqs = contiguous_layout(tables, reqs)
    wants = [oracle.retrieve(tables[src.shape[1]][:n_src], rids.cpu().numpy()) for src, n_src, rids, out in dev_reqs]
    ctx.retrieve_batch(dev_reqs)          # eager (also sizes the work space)
    ctx.sync()
    for (src, n_src, rids, out), want in zip(dev_reqs, wants):
        assert np.array_equal(out.cpu().numpy(), want)
        out.fill_(0)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            ctx.retrieve_batch(dev_reqs, stream=s)
    for _ in range(2):
        for src, n_src, rids, out in dev_reqs:
            out.fill_(0)
        g.replay()
        torch.cuda.synchronize()
        ctx.sync()
        for (src, n_src, rids, out), want in zip(dev_reqs, wants):
            assert np.array_equal(out.cpu().numpy(), want)


def test_batch_bad_rid_in_one_request(ctx):
    from paper_cs_0308004_gb300 import dpg
    tables, reqs = make_batch(40, 5_000, 3)
    rec, n_src, rids = reqs[17]
    rids = rids.copy()
    rids[0] = n_src              # inside the table but outside this request's n_src
    reqs[17] = (rec, n_src, rids)
    dev_reqs = contiguous_layout(tables, reqs)
    ctx.retrieve_batch(dev_reqs)
    with pytest.raises(dpg.DpgRangeError):
        ctx.sync()
    ctx.sync()


def test_batch_empty_and_zero_requests(ctx):
    ctx.retrieve_batch([])
    src = torch.from_numpy(synth.records(10, 8, 1)).to(DEV)
    ctx.retrieve_batch([(src, torch.zeros(0, dtype=torch.int32, device=DEV),
                         torch.zeros((0, 8), dtype=torch.uint8, device=DEV))])
    ctx.sync()


# ------------------------------------------- the persistent batch executor

def mixed_items(seed, count=120, max_n=60_000, joins=4):
    """Retrievals over one table per record size (8..512 bytes: both plans)
    plus DPG-move joins of several layouts, as (item, expected) pairs."""
    rng = np.random.default_rng(seed)
    recs = RECS + [40, 192, 300, 512]
    tables = {rec: synth.records(70_000, rec, 200 + rec) for rec in recs}
    d_tab = {rec: torch.from_numpy(t).to(DEV) for rec, t in tables.items()}
    items, wants = [], []
    for k in range(count):
        rec = recs[int(rng.integers(len(recs)))]
        n = int(np.exp(rng.uniform(0, np.log(max_n))))
        n_src = int(rng.integers(1, 70_001))
        rids = synth.uniform_ids(n, n_src, seed * 977 + k) if rng.random() < 0.5 else \
            synth.permutation(n_src, seed * 977 + k)[:n]
        out = torch.full((rids.size, rec), 0xA5, dtype=torch.uint8, device=DEV)
        items.append(("retrieve", d_tab[rec], torch.from_numpy(rids).to(DEV), out, n_src))
        wants.append(oracle.retrieve(tables[rec][:n_src], rids))
    layouts = [(16, 0, 64, 0), (24, 8, 40, 16), (12, 4, 20, 12), (64, 60, 256, 248), (16, 12, 100, 3)]
    for k in range(joins):
        fb, fk_off, db, pk_off = layouts[k % len(layouts)]
        dim, fact, _ = synth.fk_tables(3000 + 1000 * k, 40_000 + 7 * k, db, fb, 0.8, seed + k)
        if pk_off:                                   # move the key to pk_off (the row number, int64)
            keys = np.arange(dim.shape[0], dtype="<i8").view(np.uint8).reshape(-1, 8)
            dim = dim.copy()
            dim[:, pk_off:pk_off + 8] = keys
        if fk_off:
            fact = fact.copy()
            fk = fact[:, :4].copy()
            fact[:, :4] = fact[:, fk_off:fk_off + 4]
            fact[:, fk_off:fk_off + 4] = fk
        out = torch.full((fact.shape[0], fb + db), 0x33, dtype=torch.uint8, device=DEV)
        items.append(("join", to_dev(fact), to_dev(dim), out, fk_off, pk_off))
        wants.append(oracle.fk_join_move(fact, dim, fk_off, pk_off))
    return items, wants


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def check_items(items, wants):
    for it, want in zip(items, wants):
        got = it[3].cpu().numpy()
        assert np.array_equal(got, want), f"{it[0]} item of shape {want.shape} differs"


@pytest.mark.parametrize("fused", ["1", "0"])
@pytest.mark.parametrize("plan", ["", "slot", "scatter"])
def test_exec_mixed_batch_with_joins(ctx, monkeypatch, plan, fused):
    """Retrievals of 8..512-byte records and DPG-move joins of five layouts in
    one dpg_run_batch, every item equal to the oracle: one kernel launch when
    fused; otherwise one persistent launch per DPG phase, phases C and D in
    several (slot-plan groups of 4-, 8- and 16-byte words, scatter-plan
    groups of 16-byte words, then the rest; phase D of joins is always in
    the rest)."""
    if plan:
        monkeypatch.setenv("DPG_EXEC_PLAN", plan)
    else:
        monkeypatch.delenv("DPG_EXEC_PLAN", raising=False)
    monkeypatch.setenv("DPG_EXEC_FUSED", fused)
    monkeypatch.setenv("DPG_L2_RUN_KB", "1024")      # several runs per table at these sizes
    items, wants = mixed_items(7)
    launched = ctx.kernel_launches
    ctx.run_batch(items)
    ctx.sync()
    launches = ctx.kernel_launches - launched
    if fused == "1":
        assert launches == 1
    elif plan == "slot":
        assert launches == 9        # A, B; C and D for 4-, 8-, 16-byte words; D of the joins
    elif plan == "scatter":
        assert launches == 8        # A, B; C of the joins by word size, of 16-byte-word records, of the rest; D of the joins
    else:
        assert 4 <= launches <= 11  # the plan of each record size comes from the tuned-plan cache
    check_items(items, wants)


@pytest.mark.parametrize("fused", ["1", "0"])
def test_exec_graph_capture_and_replay(ctx, monkeypatch, fused):
    monkeypatch.setenv("DPG_EXEC_FUSED", fused)
    items, wants = mixed_items(8, count=60)
    ctx.run_batch(items)                             # warm-up sizes the work space
    ctx.sync()
    check_items(items, wants)
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            ctx.run_batch(items, stream=s)
    for _ in range(2):
        for it in items:
            it[3].fill_(0)
        g.replay()
        torch.cuda.synchronize()
        ctx.sync()
        check_items(items, wants)


@pytest.mark.parametrize("fused", ["1", "0"])
def test_exec_many_tiny_requests(ctx, monkeypatch, fused):
    """Hundreds of requests of 1-5 rids: a tile and a chunk span more requests
    than fit the shared-memory list (the table is searched instead)."""
    monkeypatch.setenv("DPG_EXEC_FUSED", fused)
    rng = np.random.default_rng(3)
    for rec in (8, 200):
        table = synth.records(5000, rec, rec)
        d_table = to_dev(table)
        items, wants = [], []
        for k in range(700):
            n = int(rng.integers(1, 6))
            rids = synth.uniform_ids(n, 5000, k)
            out = torch.full((n, rec), 1, dtype=torch.uint8, device=DEV)
            items.append(("retrieve", d_table, to_dev(rids), out))
            wants.append(oracle.retrieve(table, rids))
        ctx.run_batch(items)
        ctx.sync()
        check_items(items, wants)


@pytest.mark.parametrize("fused", ["1", "0"])
def test_exec_bad_rid_or_key_leaves_every_destination_untouched(ctx, monkeypatch, fused):
    from paper_cs_0308004_gb300 import dpg
    monkeypatch.setenv("DPG_EXEC_FUSED", fused)
    items, _ = mixed_items(9, count=40, joins=2)
    bad = items[13][2].clone()
    bad[bad.numel() // 2] = items[13][4]               # inside the table, outside the request's n_src
    items[13] = items[13][:2] + (bad,) + items[13][3:]
    ctx.run_batch(items)
    with pytest.raises(dpg.DpgRangeError):
        ctx.sync()
    for it in items:
        fill = 0xA5 if it[0] == "retrieve" else 0x33
        assert bool((it[3] == fill).all())
    ctx.sync()
    # a referenced dimension row whose key is not its row number
    items, wants = mixed_items(10, count=5, joins=1)
    fact, dim = items[-1][1], items[-1][2].clone()
    fk0 = int(fact[0, :4].contiguous().view(torch.int32)[0])
    dim[fk0, 0] ^= 0x01
    items[-1] = ("join", fact, dim, items[-1][3], 0, 0)
    ctx.run_batch(items)
    with pytest.raises(dpg.DpgRangeError):
        ctx.sync()


def test_exec_argument_errors(ctx):
    from paper_cs_0308004_gb300 import dpg
    src = to_dev(synth.records(100, 8, 1))
    rids = torch.zeros(10, dtype=torch.int32, device=DEV)
    ctx.run_batch([])
    ctx.run_batch([("retrieve", src, rids[:0], torch.zeros((0, 8), dtype=torch.uint8, device=DEV))])
    ctx.sync()
    fact = to_dev(np.zeros((10, 16), np.uint8))
    dim = to_dev(np.zeros((10, 64), np.uint8))
    out = torch.zeros((10, 80), dtype=torch.uint8, device=DEV)
    with pytest.raises(dpg.DpgError):               # the fk must sit at a multiple of 4
        ctx.run_batch([("join", fact, dim, out, 2, 0)])
    with pytest.raises(dpg.DpgError):               # the destination overlaps the source
        ctx.run_batch([("retrieve", src, rids, src[:10])])


def test_grouped_batch_path_still_matches(ctx, monkeypatch):
    """The grouped multi-kernel batch (DPG_BATCH_GROUPED=1) against the oracle."""
    monkeypatch.setenv("DPG_BATCH_GROUPED", "1")
    test_batch_matches_oracle_scattered(ctx)
