"""Pins for the oracle: checks against what the paper and the mathematics fix.

None of these re-types the oracle's formula.  Retrieval is pinned by an
inverse-permutation scatter (a different statement of the same result), by
decoding self-describing records, by multiset and exactly-once invariants and
by the worked example of §2.2; the three-phase statement of Figure 1 must agree
with the one-line definition of §2; the key-pointer sort of §3 is pinned by
sortedness, tie order, permutation and a brute-force selection sort; the
foreign-key joins of §4.2 by the textbook nested-loop join.
"""
import itertools
import json
import os

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def self_describing(n, rec, seed=11):
    """Records whose first min(rec, 4) bytes hold the record index (LE)."""
    src = synth.records(n, rec, seed).copy()
    k = min(rec, 4)
    idx = np.arange(n, dtype="<u4").view(np.uint8).reshape(n, 4)
    src[:, :k] = idx[:, :k]
    return src


def decode(dst, rec):
    k = min(rec, 4)
    buf = np.zeros((dst.shape[0], 4), dtype=np.uint8)
    buf[:, :k] = dst[:, :k]
    return buf.view("<u4").reshape(-1).astype(np.int64)


# ------------------------------------------------------------- retrieval (§2)

@pytest.mark.parametrize("rec", [1, 3, 4, 7, 16, 100, 255, 300])
def test_retrieve_all_permutations_small(rec):
    """Every permutation of n <= 5 rids: dst equals the inverse-permutation scatter."""
    for n in range(0, 6):
        src = synth.records(n, rec, 100 + n)
        for perm in itertools.permutations(range(n)):
            rids = np.array(perm, dtype=np.int32)
            got = oracle.retrieve(src, rids)
            inv = np.empty(n, dtype=np.int64)
            inv[rids] = np.arange(n)
            want = np.empty_like(src)
            for j in range(n):          # scatter: source record j lands at inv[j]
                want[inv[j]] = src[j]
            assert np.array_equal(got, want)


@pytest.mark.parametrize("rec", list(range(1, 301, 7)) + [256, 300])
def test_retrieve_random_permutation_by_scatter(rec):
    n = 8
    src = synth.records(n, rec, 5)
    rids = synth.permutation(n, rec)
    got = oracle.retrieve(src, rids)
    want = np.empty_like(src)
    want[np.argsort(rids, kind="stable")] = src  # dst[inv[j]] = src[j]
    assert np.array_equal(got, want)


@pytest.mark.parametrize("rec", [4, 5, 8, 100, 256])
def test_retrieve_duplicates_decode(rec):
    """Rids drawn with replacement (§2: records may be duplicated): decoding each
    destination record recovers exactly the rid sequence."""
    n_src, n = 300, 1000
    src = self_describing(n_src, rec)
    rids = synth.uniform_ids(n, n_src, 7)
    dst = oracle.retrieve(src, rids)
    assert np.array_equal(decode(dst, rec), rids.astype(np.int64))
    # numpy's fancy indexing (a library gather) agrees byte for byte
    assert np.array_equal(dst, src[rids.astype(np.int64)])


def test_retrieve_permutation_multiset_and_exactly_once():
    """A permutation rid sequence yields a permutation of the records (§2);
    every destination slot is written exactly once (no canary survives)."""
    n, rec = 2000, 100
    src = self_describing(n, rec)
    rids = synth.permutation(n, 3)
    dst = np.full((n, rec), 0xA5, dtype=np.uint8)
    oracle.retrieve(src, rids, out=dst)
    ids = decode(dst, rec)
    assert np.array_equal(np.sort(ids), np.arange(n))
    a = np.sort(dst.view(f"V{rec}").reshape(-1))
    b = np.sort(src.view(f"V{rec}").reshape(-1))
    assert np.array_equal(a, b)
    assert not np.any(np.all(dst == 0xA5, axis=1))


@pytest.mark.parametrize("bad", [-1, 50, 2**31 - 1])
def test_retrieve_out_of_range_writes_nothing(bad):
    n_src, rec = 50, 12
    # a view of the first n_src rows of a larger table: an off-by-one range
    # check would read real memory and the pin still sees it
    src = synth.records(n_src + 10, rec, 1)[:n_src]
    rids = synth.uniform_ids(40, n_src, 2)
    rids[37] = bad
    dst = np.full((40, rec), 0x5A, dtype=np.uint8)
    with pytest.raises(oracle.OracleRangeError):
        oracle.retrieve(src, rids, out=dst)
    assert np.all(dst == 0x5A)


@pytest.mark.parametrize("threads", [1, 3, 16, 200])
def test_retrieve_threads_equals_retrieve(threads):
    """The multi-core retrieval (the benchmark's CPU figure) gives the plain
    retrieval's bytes, with more threads than records too, and on a bad rid
    reports it and writes nothing."""
    for n, rec in ((0, 8), (1, 3), (150, 100), (1009, 17)):
        src = synth.records(64, rec, 5)
        rids = synth.uniform_ids(n, 64, 6)
        assert np.array_equal(oracle.retrieve_threads(src, rids, threads), oracle.retrieve(src, rids))
    src = synth.records(64, 12, 7)
    rids = synth.uniform_ids(500, 64, 8)
    rids[377] = 64
    out = np.full((500, 12), 0x5A, np.uint8)
    with pytest.raises(oracle.OracleRangeError):
        oracle.retrieve_threads(src, rids, threads, out=out)
    assert bool((out == 0x5A).all())


def test_retrieve_empty():
    src = synth.records(10, 8, 1)
    assert oracle.retrieve(src, np.zeros(0, np.int32)).shape == (0, 8)


# ------------------------------------------------ Figure 1 three phases (§2.1)

def test_worked_example_section_2_2():
    g = json.load(open(os.path.join(GOLDEN, "worked_example_dpg.json")))
    keys = g["key_of_record"]
    rec = 4
    src = np.zeros((12, rec), dtype=np.uint8)
    for r, k in enumerate(keys):
        src[r, 0] = ord(k)
        src[r, 1] = r
    rids = np.array(g["rid_sequence_in_key_order"], dtype=np.int32)
    # the paper's stated facts hold for the fixture
    gv = g["given_by_paper"]
    for k, r in gv["first_rids_in_key_order"].items():
        assert rids[ord(k) - ord("a")] == r
    assert [keys[r] for r in range(4)] == gv["first_input_run_keys_in_record_order"]
    runs, internal, dst = oracle.dpg_phases(src, rids, g["given_by_paper"]["run_length"])
    assert len(runs) == gv["runs"]
    assert runs[0].tolist() == gv["first_rid_run_after_phase_I"]
    assert [chr(c) for c in internal[0][:, 0]] == gv["first_internal_run_keys_after_phase_II"]
    assert [r.tolist() for r in runs] == g["expected"]["rid_runs"]
    assert [[chr(c) for c in x[:, 0]] for x in internal] == g["expected"]["internal_run_keys"]
    assert [chr(c) for c in dst[:, 0]] == g["expected"]["output_keys"]
    # and the three phases agree with the definition
    assert np.array_equal(dst, oracle.retrieve(src, rids))


@pytest.mark.parametrize("rec", [1, 4, 13, 100])
def test_three_phases_equal_definition(rec):
    """Figure 1 and D[i] = R[S_rid[i]] agree for every run length, with
    permutations, duplicates and skew (§2, §2.3)."""
    n_src = 37
    src = synth.records(n_src, rec, 21)
    seqs = [synth.permutation(n_src, 1), synth.uniform_ids(60, n_src, 2),
            np.full(25, 36, np.int32), np.zeros(0, np.int32),
            np.concatenate([np.full(30, 3, np.int32), synth.uniform_ids(10, n_src, 3)])]
    for rids in seqs:
        want = oracle.retrieve(src, rids)
        for L in range(1, n_src + 2):
            runs, internal, dst = oracle.dpg_phases(src, rids, L)
            assert np.array_equal(dst, want)
            assert len(runs) == -(-n_src // L)
            # Phase I keeps RID order inside each run and partitions by range
            for j, run in enumerate(runs):
                assert np.all(run // L == j)
                assert run.tolist() == [int(r) for r in rids if r // L == j]
                assert np.array_equal(internal[j], src[run.astype(np.int64)])
            assert sum(len(r) for r in runs) == rids.size


def test_three_phases_all_permutations_n6():
    rec, n = 3, 6
    src = synth.records(n, rec, 8)
    for perm in itertools.permutations(range(n)):
        rids = np.array(perm, dtype=np.int32)
        want = np.empty_like(src)
        want[np.argsort(rids)] = src
        for L in (1, 2, 4, 6):
            assert np.array_equal(oracle.dpg_phases(src, rids, L)[2], want)


# ------------------------------------------------------------- sorting (§3)

def _key_sorted_ok(pairs, key_bytes=10):
    keys = [bytes(p[:key_bytes]) for p in pairs]
    rids = oracle.pair_rids(pairs)
    for a in range(len(keys) - 1):
        assert (keys[a], rids[a]) < (keys[a + 1], rids[a + 1])


@pytest.mark.parametrize("rec", [10, 16, 100])
def test_sort_keyptr_sorted_permutation(rec):
    n = 400
    src = synth.records(n, rec, 31).copy()
    # force duplicate keys: 100 records share a few keys, ties go by rid
    src[::4, :10] = src[0, :10]
    src[1::8, :10] = src[1, :10]
    pairs = oracle.sort_keyptr(src, 10)
    _key_sorted_ok(pairs)
    rids = oracle.pair_rids(pairs)
    assert np.array_equal(np.sort(rids), np.arange(n))
    assert np.array_equal(pairs[:, :10], src[rids, :10])
    assert np.all(pairs[:, 10:12] == 0)


def test_sort_keyptr_matches_selection_sort():
    """Brute force: repeatedly take the smallest remaining (key, rid)."""
    n, rec = 40, 12
    src = synth.records(n, rec, 41).copy()
    src[5:15, :10] = src[3, :10]
    src[:, 0] &= 0x03  # many shared leading bytes
    pairs = oracle.sort_keyptr(src, 10)
    remaining = list(range(n))
    order = []
    while remaining:
        best = remaining[0]
        for r in remaining[1:]:
            if bytes(src[r, :10]) < bytes(src[best, :10]):
                best = r
        order.append(best)
        remaining.remove(best)
    assert oracle.pair_rids(pairs).tolist() == order


def test_sort_keyptr_every_key_byte_counts():
    """Keys that differ in one byte position only, placed so that rid order is the
    reverse of key order: each of the 10 key bytes must decide the order, and
    bytes past the key must not."""
    for pos in range(10):
        n, rec = 6, 16
        src = np.zeros((n, rec), np.uint8)
        src[:, pos] = np.arange(n, 0, -1)        # record 0 has the largest key
        src[:, 10] = np.arange(n)                # a non-key byte, ascending
        rids = oracle.pair_rids(oracle.sort_keyptr(src, 10))
        assert rids.tolist() == list(range(n - 1, -1, -1))
    src = np.zeros((4, 12), np.uint8)
    src[:, 11] = [3, 2, 1, 0]                    # only non-key bytes differ: rid order
    assert oracle.pair_rids(oracle.sort_keyptr(src, 10)).tolist() == [0, 1, 2, 3]


def test_sort_records_sorted_file():
    """§3: copying records by the sorted pairs yields a key-sorted file that is a
    permutation of the input."""
    n, rec = 500, 100
    src = synth.records(n, rec, 3).copy()
    src[:, 10:14] = np.arange(n, dtype="<u4").view(np.uint8).reshape(n, 4)
    src[::3, :10] = src[1, :10]       # ties
    out = oracle.sort_records(src, 10)
    ids = out[:, 10:14].copy().view("<u4").reshape(-1).astype(np.int64)
    assert np.array_equal(np.sort(ids), np.arange(n))
    keyed = [(bytes(r[:10]), int(i)) for r, i in zip(out, ids)]
    assert keyed == sorted(keyed)
    assert np.array_equal(out, src[ids])


def test_sort_copy_out_of_range():
    src = synth.records(10, 8, 1)
    pairs = np.zeros((3, 16), np.uint8)
    pairs[1, 12:16] = np.array([10], "<i4").view(np.uint8)
    with pytest.raises(oracle.OracleRangeError):
        oracle.sort_copy(pairs, src)


# ------------------------------------------------------- FK joins (§4.2)

def _fk_case(n_dim, n_fact, seed, s=0.8):
    dim, fact, fk = synth.fk_tables(n_dim, n_fact, 64, 16, s, seed)
    fact = fact.copy()
    fact[:, 4:8] = np.arange(n_fact, dtype="<u4").view(np.uint8).reshape(n_fact, 4)
    return dim, fact, fk


@pytest.mark.parametrize("n_dim,n_fact", [(1, 5), (7, 60), (50, 400)])
def test_fk_join_move_equals_nested(n_dim, n_fact):
    dim, fact, fk = _fk_case(n_dim, n_fact, n_dim)
    nested = oracle.fk_join_nested(fact, dim)
    move = oracle.fk_join_move(fact, dim)
    assert nested.shape == (n_fact, 80)
    assert np.array_equal(move, nested)
    # every row joins matching keys
    assert np.array_equal(move[:, 16:24].copy().view("<i8").reshape(-1), fk.astype(np.int64))


@pytest.mark.parametrize("n_dim,n_fact", [(7, 60), (50, 400)])
def test_fk_join_sorted_order(n_dim, n_fact):
    dim, fact, fk = _fk_case(n_dim, n_fact, 5 + n_dim)
    nested = oracle.fk_join_nested(fact, dim)
    srt = oracle.fk_join_sorted(fact, dim)
    order = sorted(range(n_fact), key=lambda i: (int(fk[i]), i))
    assert np.array_equal(srt, nested[order])


@pytest.mark.parametrize("n_dim,n_fact", [(1, 5), (7, 300), (50, 400), (1000, 20_000)])
def test_fk_join_order_is_the_sorted_join(n_dim, n_fact):
    """The linear-time join order (stable counting sort) against the
    comparison sort of oracle_fk_join_sorted and a brute-force (fk, row)
    ordering: rows of the sorted join are move-join rows of fact[order]."""
    dim, fact, fk = _fk_case(n_dim, n_fact, 11 + n_dim)
    order = oracle.fk_join_order(fact, n_dim)
    assert order.tolist() == sorted(range(n_fact), key=lambda i: (int(fk[i]), i))
    assert np.array_equal(oracle.fk_join_move(fact[order], dim), oracle.fk_join_sorted(fact, dim))
    bad = fact.copy()
    bad[n_fact // 2, :4] = np.array([n_dim], "<i4").view(np.uint8)
    with pytest.raises(oracle.OracleRangeError):
        oracle.fk_join_order(bad, n_dim)


def test_fk_join_bad_key():
    dim, fact, fk = _fk_case(10, 30, 9)
    fact[3, :4] = np.array([10], "<i4").view(np.uint8)
    with pytest.raises(oracle.OracleRangeError):
        oracle.fk_join_move(fact, dim)
    with pytest.raises(oracle.OracleRangeError):
        oracle.fk_join_sorted(fact, dim)
    dim2 = dim.copy()
    dim2[4, :8] = np.array([99], "<i8").view(np.uint8)   # pk no longer row index
    fact[3, :4] = np.array([4], "<i4").view(np.uint8)
    with pytest.raises(oracle.OracleRangeError):
        oracle.fk_join_move(fact, dim2)
