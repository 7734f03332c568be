"""Batched retrieval (dpg_retrieve_batch): every request's output against the
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
