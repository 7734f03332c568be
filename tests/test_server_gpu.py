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
