"""Serving engine (dpg_server_*): a mix of retrievals and joins submitted as a
burst and run concurrently under an HBM budget; every result against the
oracle; each result identical alone and in the mix; admission limits."""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda", 0)


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


@pytest.fixture(scope="module")
def workload():
    rng = np.random.default_rng(7)
    tables = {rec: synth.records(200_000, rec, 300 + rec) for rec in (16, 32, 64, 100, 128, 256)}
    dim, fact, fk = synth.fk_tables(50_000, 400_000, 64, 16, 0.8, 4)
    perm = synth.permutation(200_000, 11)
    jobs = []
    for k in range(40):
        if rng.random() < 0.6:
            rec = [16, 32, 64, 100, 128, 256][int(rng.integers(6))]
            n = int(np.exp(rng.uniform(np.log(1e3), np.log(2e5))))
            start = int(rng.integers(0, 200_000 - n + 1))
            jobs.append(("retrieve", rec, perm[start:start + n].copy()))
        else:
            n = int(np.exp(rng.uniform(np.log(1e3), np.log(4e5))))
            start = int(rng.integers(0, 400_000 - n + 1))
            mode = ["move", "sort", "direct"][int(rng.integers(3))]
            jobs.append(("join", mode, (start, n)))
    d_tables = {rec: to_dev(t) for rec, t in tables.items()}
    d_dim, d_fact = to_dev(dim), to_dev(fact)
    wants = []
    for kind, a, b in jobs:
        if kind == "retrieve":
            wants.append(oracle.retrieve(tables[a], b))
        else:
            start, n = b
            f = fact[start:start + n]
            wants.append(oracle.fk_join_sorted(f, dim) if a == "sort" else oracle.fk_join_move(f, dim))
    return jobs, d_tables, d_dim, d_fact, wants


def submit_all(srv, jobs, d_tables, d_dim, d_fact, keep):
    tickets = []
    for kind, a, b in jobs:
        if kind == "retrieve":
            rids = to_dev(b)
            keep.append(rids)
            tickets.append(srv.submit_retrieve(d_tables[a], rids))
        else:
            start, n = b
            tickets.append(srv.submit_join(d_fact[start:start + n], d_dim, a))
    return tickets


def test_server_mix_matches_oracle_and_alone(workload):
    from paper_cs_0308004_gb300 import dpg
    jobs, d_tables, d_dim, d_fact, wants = workload
    keep = []
    mixed = []
    with dpg.Server(0, slots=4, budget_bytes=2 << 30) as srv:    # tight budget: jobs queue for memory
        tickets = submit_all(srv, jobs, d_tables, d_dim, d_fact, keep)
        for t, want in zip(tickets, wants):
            st, out, lat = srv.result(t)
            assert st == dpg.OK
            got = out.cpu().numpy()
            assert np.array_equal(got, want)
            mixed.append(got)
            assert lat > 0
            srv.release(t)
        assert srv.held_bytes == 0
    with dpg.Server(0, slots=1, budget_bytes=8 << 30) as srv:    # each job alone
        for job, got_mixed in zip(jobs, mixed):
            t = submit_all(srv, [job], d_tables, d_dim, d_fact, keep)[0]
            st, out, _ = srv.result(t)
            assert st == dpg.OK
            assert np.array_equal(out.cpu().numpy(), got_mixed)
            srv.release(t)


def test_server_admission_and_errors(workload):
    from paper_cs_0308004_gb300 import dpg
    jobs, d_tables, d_dim, d_fact, wants = workload
    with dpg.Server(0, slots=2, budget_bytes=64 << 20) as srv:
        # 300,000 x 256-byte output records alone exceed the whole budget,
        # whichever plan the retrieval takes
        big = to_dev(synth.uniform_ids(300_000, 200_000, 3))
        with pytest.raises(dpg.DpgError):
            srv.submit_retrieve(d_tables[256], big)
        bad = to_dev(np.array([0, 5, 200_000], np.int32))
        t = srv.submit_retrieve(d_tables[16], bad)
        st, out, _ = srv.result(t)
        assert st == dpg.ERANGE
        srv.release(t)
        ok = to_dev(np.arange(1000, dtype=np.int32))
        t = srv.submit_retrieve(d_tables[16], ok)
        st, out, _ = srv.result(t)
        assert st == dpg.OK and torch.equal(out, d_tables[16][:1000])
        srv.release(t)


@pytest.mark.parametrize("bypass", ["8", "1", "0"])
def test_server_backfills_past_a_waiting_head(monkeypatch, bypass):
    """A head job that cannot fit (an earlier result still holds the budget)
    lets the small jobs behind it run, up to the bypass bound; with the bound
    at 0 the queue keeps strict arrival order.  Every result matches the
    oracle once the budget frees up."""
    import time
    from paper_cs_0308004_gb300 import dpg
    monkeypatch.setenv("DPG_SERVE_BYPASS", bypass)
    n_big, rec = 4_000_000, 256
    big = synth.records(n_big, rec, 1)
    big_rids = synth.permutation(n_big, 2)
    small = synth.records(20_000, 16, 3)
    small_rids = [synth.uniform_ids(10_000, 20_000, 4 + k) for k in range(2)]
    d_big, d_big_rids, d_small = to_dev(big), to_dev(big_rids), to_dev(small)
    d_small_rids = [to_dev(r) for r in small_rids]
    want_big = oracle.retrieve(big, big_rids)
    with dpg.Server(0, slots=4, budget_bytes=int(1.5e9)) as srv:
        t1 = srv.submit_retrieve(d_big, d_big_rids)
        st, _, _ = srv.result(t1)                 # done; its 1 GB result stays held
        assert st == dpg.OK
        t2 = srv.submit_retrieve(d_big, d_big_rids)     # cannot fit until t1 is released
        t3 = srv.submit_retrieve(d_small, d_small_rids[0])
        t4 = srv.submit_retrieve(d_small, d_small_rids[1])
        deadline = time.time() + 3.0
        done = {}
        while time.time() < deadline and len(done) < 2:
            for t in (t3, t4):
                if t not in done:
                    r = srv.result(t, wait=False)
                    if r is not None:
                        done[t] = r
            time.sleep(0.01)
        passed = {"8": {t3, t4}, "1": {t3}, "0": set()}[bypass]
        assert set(done) == passed
        assert srv.result(t2, wait=False) is None       # the head still waits for memory
        srv.release(t1)
        st, out2, _ = srv.result(t2)
        assert st == dpg.OK and np.array_equal(out2.cpu().numpy(), want_big)
        srv.release(t2)
        for t, rids in ((t3, small_rids[0]), (t4, small_rids[1])):
            st, out, _ = srv.result(t)
            assert st == dpg.OK and np.array_equal(out.cpu().numpy(), oracle.retrieve(small, rids))
            srv.release(t)
