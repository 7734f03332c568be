"""Parity of the GPU three-phase sort (§3) with the oracle, byte for byte:
key-pointer pairs (dpg_sort_keyptr) and sorted records (dpg_sort_records),
over ragged tile counts, record sizes, key lengths and ties (the full-size
10,000,000 x 100-byte file is compared row by row in test_full_size_gpu.py)."""
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


def tie_heavy(n, rec, seed):
    src = synth.records(n, rec, seed).copy()
    src[::3, :10] = src[0, :10]             # a third of the keys equal
    if n > 1:
        src[1::7, :9] = src[1, :9]          # keys equal but for the last key byte
    src[2::11, 0] = 0xff                    # top byte saturated
    return src


# n spans the 8192-pair tile of the radix passes (one, several and ragged);
# key lengths put 1, 2 and 3 four-byte key groups with every tail length
@pytest.mark.parametrize("n", [1, 2, 100, 4095, 4097, 8191, 8192, 8193, 24_581, 100_003])
@pytest.mark.parametrize("rec,key_bytes", [(10, 10), (16, 10), (100, 10), (13, 3), (12, 12), (256, 1), (100, 7),
                                           (8, 4), (12, 5), (20, 8), (9, 9), (11, 11)])
def test_sort_keyptr_matches_oracle(ctx, n, rec, key_bytes):
    for src in (synth.records(n, rec, n + rec), tie_heavy(n, rec, 5)):
        want = oracle.sort_keyptr(src, key_bytes)
        got = ctx.sort_keyptr(to_dev(src), key_bytes)
        ctx.sync()
        assert np.array_equal(got.cpu().numpy(), want)


def bucket_mix(rec, seed):
    """Records whose two-byte key prefixes make buckets of chosen sizes (the
    bucket stage sorts buckets of up to 256 pairs in place and sends larger
    ones through the full LSD fallback), with whole keys repeated inside
    buckets so that ties fall back on rid order, rows shuffled."""
    rng = np.random.default_rng(seed)
    sizes = [1, 2, 3, 4, 5, 31, 32, 33, 128, 129, 255, 256, 257, 258, 511, 1000, 5000]
    prefixes = rng.choice(65536, size=len(sizes), replace=False)
    n_rand = 40_000
    n = sum(sizes) + n_rand
    src = rng.integers(0, 256, size=(n, rec), dtype=np.uint8)
    at = 0
    for size, pre in zip(sizes, prefixes):
        src[at:at + size, 0] = pre >> 8
        src[at:at + size, 1] = pre & 0xff
        if size > 3:  # a run of equal keys inside the bucket
            src[at + 1:at + 1 + size // 3, 2:10] = src[at, 2:10]
        at += size
    return src[rng.permutation(n)].copy()


@pytest.mark.parametrize("rec,key_bytes", [(16, 10), (12, 12), (16, 3), (16, 2), (16, 1), (100, 10)])
def test_sort_bucket_sizes(ctx, rec, key_bytes):
    src = bucket_mix(rec, 11 + key_bytes)
    want = oracle.sort_keyptr(src, key_bytes)
    got = ctx.sort_keyptr(to_dev(src), key_bytes)
    ctx.sync()
    assert np.array_equal(got.cpu().numpy(), want)


@pytest.mark.parametrize("what", ["keyptr", "records"])
def test_sort_graph_capture_and_replay(ctx, what):
    """The sort (its cooperative fallback launch included) captured in a CUDA
    graph after one eager call at the same size, then replayed on new input
    in the same buffers: once with keys that need the fallback, once without."""
    rec, kb = 16, 10
    a = bucket_mix(rec, 31)
    b = synth.records(a.shape[0], rec, 32)
    fn = ctx.sort_keyptr if what == "keyptr" else ctx.sort_records
    ref = oracle.sort_keyptr if what == "keyptr" else oracle.sort_records
    d_src = to_dev(a)
    out = fn(d_src, kb)  # eager: sizes the context's scratch
    ctx.sync()
    assert np.array_equal(out.cpu().numpy(), ref(a, kb))
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            fn(d_src, kb, out=out, stream=s)
    for src in (b, a):
        d_src.copy_(to_dev(src))
        out.fill_(0)
        torch.cuda.synchronize()
        g.replay()
        torch.cuda.synchronize()
        ctx.sync()
        assert np.array_equal(out.cpu().numpy(), ref(src, kb))


def test_sort_all_equal_keys(ctx):
    n, rec = 50_001, 16
    src = synth.records(n, rec, 9).copy()
    src[:, :10] = 0x42
    got = ctx.sort_keyptr(to_dev(src), 10)
    ctx.sync()
    assert np.array_equal(got.cpu().numpy(), oracle.sort_keyptr(src, 10))


@pytest.mark.parametrize("variant", ["3", "4"])
@pytest.mark.parametrize("rec", [16, 100, 256])
def test_sort_records_matches_oracle(ctx, monkeypatch, rec, variant):
    monkeypatch.setenv("DPG_VARIANT", variant)
    n = 300_007
    src = tie_heavy(n, rec, rec)
    got = ctx.sort_records(to_dev(src), 10)
    ctx.sync()
    assert np.array_equal(got.cpu().numpy(), oracle.sort_records(src, 10))


def test_sort_argument_errors(ctx):
    from paper_cs_0308004_gb300 import dpg
    src = to_dev(synth.records(100, 8, 1))
    for kb in (0, 13, 9):
        with pytest.raises(dpg.DpgError):
            ctx.sort_keyptr(src, kb)
    empty = torch.zeros((0, 8), dtype=torch.uint8, device=DEV)
    assert ctx.sort_keyptr(empty, 4).shape == (0, 16)
