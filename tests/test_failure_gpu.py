"""Failure detection without a GPU fault.

* A bounded device wait made to run out: dpg_check_wait waits, under the
  context's wait limit, on a device word that nothing sets; the next sync
  reports DPG_ETIMEOUT, the error is cleared, and the same context then
  retrieves and sorts correctly (the sort's look-back waits run under the
  same limit).
* A host-side allocation failure: dpg_inject_alloc_failure makes the next
  device allocation of a context fail; the call that needed it returns
  DPG_ENOMEM having launched nothing, the destination is untouched, and the
  next call succeeds.
"""
import time

import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda", 0)


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def test_wait_runs_out_and_context_stays_usable():
    from paper_cs_0308004_gb300 import dpg
    with dpg.Context(0) as c:
        c.set_wait_limit(0.02)
        t0 = time.perf_counter()
        c.check_wait()
        with pytest.raises(dpg.DpgError) as e:
            c.sync()
        waited = time.perf_counter() - t0
        assert e.value.status == dpg.ETIMEOUT
        assert 0.015 < waited < 5.0
        c.sync()                                    # the timeout was reported once and cleared
        src = synth.records(50_001, 24, 3)
        rids = synth.uniform_ids(70_001, 50_001, 4)
        out = c.retrieve(to_dev(src), to_dev(rids))
        c.sync()
        assert np.array_equal(out.cpu().numpy(), oracle.retrieve(src, rids))
        c.set_wait_limit(1.0)
        keys = synth.records(100_003, 16, 5)
        pairs = c.sort_keyptr(to_dev(keys), 10)
        c.sync()
        assert np.array_equal(pairs.cpu().numpy(), oracle.sort_keyptr(keys, 10))


def test_wait_limit_arguments():
    from paper_cs_0308004_gb300 import dpg
    with dpg.Context(0) as c:
        for bad in (0.0, -1.0, 61.0, float("nan")):
            with pytest.raises(dpg.DpgError) as e:
                c.set_wait_limit(bad)
            assert e.value.status == dpg.EINVAL
        c.set_wait_limit(60.0)


@pytest.mark.parametrize("what", ["retrieve_l2", "retrieve_3pass", "sort_records", "join_sort", "retrieve_host"])
def test_injected_alloc_failure_enqueues_nothing(monkeypatch, what):
    from paper_cs_0308004_gb300 import dpg
    monkeypatch.setenv("DPG_VARIANT", "3" if what == "retrieve_3pass" else "4")
    n_src, rec = 40_009, 32
    src = synth.records(n_src, rec, 7)
    rids = synth.uniform_ids(60_013, n_src, 8)
    dim, fact, _ = synth.fk_tables(5000, 30_011, 64, 16, 0.8, 9)
    with dpg.Context(0) as c:
        def run(out):
            if what.startswith("retrieve_") and what != "retrieve_host":
                c.retrieve(to_dev(src), to_dev(rids), out=out)
                return oracle.retrieve(src, rids)
            if what == "sort_records":
                c.sort_records(to_dev(src), 10, out=out)
                return oracle.sort_records(src, 10)
            if what == "join_sort":
                c.fk_join(to_dev(fact), to_dev(dim), "sort", out=out)
                return oracle.fk_join_sorted(fact, dim)
            c.retrieve_host(torch.from_numpy(src), torch.from_numpy(rids), out)
            return oracle.retrieve(src, rids)

        shape = {"sort_records": src.shape, "join_sort": (fact.shape[0], 80)}.get(what, (rids.size, rec))
        dev = DEV if what != "retrieve_host" else torch.device("cpu")
        out = torch.full(shape, 0x5A, dtype=torch.uint8, device=dev)
        c.inject_alloc_failure(1)
        launched = c.kernel_launches
        with pytest.raises(dpg.DpgError) as e:
            run(out)
        assert e.value.status == dpg.ENOMEM
        assert c.kernel_launches == launched
        c.sync()                                    # no asynchronous error either
        assert bool((out == 0x5A).all())
        want = run(out)                             # the hook fired once: this call allocates
        c.sync()
        assert np.array_equal(out.cpu().numpy(), want)
