"""dpg_retrieve_noalloc: the allocation-free entry point, for callers that
cannot allocate device memory when they call (a caching allocator holds all
free memory, a memory-capped region, a plug-in that must not allocate).

It is called here through the C ABI with ctypes.  On two calls in a row it
must give, byte for byte, both the oracle's result and dpg_retrieve's on the
same inputs: a ragged last segment, duplicated rids, the plain-load path of
the probe (a 7-byte record size, source and destination off their 16-byte
boundaries) and a destination at an odd address.  Its limits (too many rids,
too many source segments), an empty table and a bad rid return their errors
with the destination untouched, and a fresh process shows that calls after
the first allocate no device memory.  The file name makes pytest collect it
last; it passes alone in a fresh process too.
"""
import ctypes
import os
import subprocess
import sys

import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _lib():
    from paper_cs_0308004_gb300 import dpg
    f = dpg.lib.dpg_retrieve_noalloc
    f.argtypes = [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_size_t, ctypes.c_size_t, ctypes.c_void_p,
                  ctypes.c_void_p, ctypes.c_void_p]
    f.restype = ctypes.c_int
    return dpg, f


def _placed(arr: np.ndarray, offset: int, dev):
    """The bytes of arr on the device starting `offset` bytes past a 256-byte
    boundary, inside a zeroed buffer with 64 spare bytes on both sides."""
    flat = torch.zeros(arr.nbytes + offset + 128, dtype=torch.uint8, device=dev)
    view = flat[64 + offset:64 + offset + arr.nbytes]
    view.copy_(torch.from_numpy(np.ascontiguousarray(arr).reshape(-1).view(np.uint8)).to(dev))
    return flat, view


CASES = [
    # n_src, rec, rid kind, src offset, dst offset
    (700_001, 100, "perm", 0, 0),     # 684 segments of 1024 records, the last one holds 609
    (300_000, 16, "dup", 0, 0),       # 1,000,003 rids drawn with replacement
    (50_001, 7, "dup", 3, 1),         # plain loads in the probe, one-byte words
    (20_011, 100, "dup", 4, 1),       # source 4 bytes off its boundary, odd destination
]


@pytest.mark.parametrize("n_src,rec,kind,src_off,dst_off", CASES)
def test_noalloc_matches_oracle_and_dpg_retrieve_twice(n_src, rec, kind, src_off, dst_off):
    dpg, f = _lib()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev).cuda_stream
    src = synth.records(n_src, rec, 1)
    rids = synth.permutation(n_src, 2) if kind == "perm" else synth.uniform_ids(
        {300_000: 1_000_003}.get(n_src, n_src + 10_007), n_src, 5)
    want = oracle.retrieve(src, rids)
    _, d_src = _placed(src, src_off, dev)
    d_rids = torch.from_numpy(rids).to(dev)
    with dpg.Context(0) as ctx:
        via_dpg = ctx.retrieve(d_src.view(n_src, rec), d_rids)
        ctx.sync()
        assert np.array_equal(via_dpg.cpu().numpy(), want)
    for _ in range(2):          # two calls in a row share the static scratch
        flat, d_dst = _placed(np.full((rids.size, rec), 0xA5, np.uint8), dst_off, dev)
        st = f(d_src.data_ptr(), n_src, rec, rids.size, d_rids.data_ptr(), d_dst.data_ptr(), stream)
        assert st == 0, dpg.lib.dpg_strerror(st)
        assert np.array_equal(d_dst.view(rids.size, rec).cpu().numpy(), want)
        assert torch.equal(d_dst.view(rids.size, rec), via_dpg)
        assert int(flat[:64 + dst_off].sum()) == 0 and int(flat[64 + dst_off + d_dst.numel():].sum()) == 0


def test_noalloc_limits_empty_table_and_bad_rid():
    dpg, f = _lib()
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev).cuda_stream
    src = torch.from_numpy(synth.records(1000, 8, 1)).to(dev)
    # more rids than the array has room for
    too_many = torch.zeros((1 << 21) + 1, dtype=torch.int32, device=dev)
    out = torch.full((too_many.numel(), 8), 7, dtype=torch.uint8, device=dev)
    assert f(src.data_ptr(), 1000, 8, too_many.numel(), too_many.data_ptr(), out.data_ptr(), stream) == dpg.EINVAL
    assert bool((out == 7).all())
    # one source segment too many: 100-byte records sit 1024 to a segment
    n_big = 4096 * 1024 + 1
    big = torch.zeros((n_big, 100), dtype=torch.uint8, device=dev)
    rids = torch.zeros(10, dtype=torch.int32, device=dev)
    out = torch.full((10, 100), 7, dtype=torch.uint8, device=dev)
    assert f(big.data_ptr(), n_big, 100, 10, rids.data_ptr(), out.data_ptr(), stream) == dpg.EINVAL
    assert f(big.data_ptr(), n_big - 1, 100, 10, rids.data_ptr(), out.data_ptr(), stream) == dpg.OK
    assert torch.equal(out, big[:10])
    del big
    # an empty source table: every rid is out of range
    out = torch.full((3, 8), 7, dtype=torch.uint8, device=dev)
    assert f(src.data_ptr(), 0, 8, 3, rids.data_ptr(), out.data_ptr(), stream) == dpg.ERANGE
    assert bool((out == 7).all())
    # a bad rid
    r = np.arange(500, dtype=np.int32)
    r[77] = 1000
    d_r = torch.from_numpy(r).to(dev)
    out = torch.full((500, 8), 7, dtype=torch.uint8, device=dev)
    assert f(src.data_ptr(), 1000, 8, 500, d_r.data_ptr(), out.data_ptr(), stream) == dpg.ERANGE
    assert bool((out == 7).all())
    # and the next good call is right again (the error word starts at zero each call)
    r[77] = 999
    d_r.copy_(torch.from_numpy(r))
    assert f(src.data_ptr(), 1000, 8, 500, d_r.data_ptr(), out.data_ptr(), stream) == dpg.OK
    assert np.array_equal(out.cpu().numpy(), oracle.retrieve(src.cpu().numpy(), r))


_FRESH = r"""
import sys
sys.path.insert(0, sys.argv[1])
import ctypes, torch
import synth
from paper_cs_0308004_gb300 import dpg
f = dpg.lib.dpg_retrieve_noalloc
f.argtypes = [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_size_t, ctypes.c_size_t, ctypes.c_void_p,
              ctypes.c_void_p, ctypes.c_void_p]
f.restype = ctypes.c_int
dev = torch.device("cuda", 0)
n, rec = 200_003, 64
src = torch.from_numpy(synth.records(n, rec, 1)).to(dev)
rids = torch.from_numpy(synth.permutation(n, 2)).to(dev)
out = torch.empty((n, rec), dtype=torch.uint8, device=dev)
st = torch.cuda.current_stream(dev).cuda_stream
torch.cuda.synchronize()
free0 = torch.cuda.mem_get_info(dev)[0]
assert f(src.data_ptr(), n, rec, n, rids.data_ptr(), out.data_ptr(), st) == 0   # the set-up call
free1 = torch.cuda.mem_get_info(dev)[0]
for _ in range(3):
    assert f(src.data_ptr(), n, rec, n, rids.data_ptr(), out.data_ptr(), st) == 0
free2 = torch.cuda.mem_get_info(dev)[0]
assert torch.equal(out, src[rids.long()])
print("set-up call took", free0 - free1, "bytes; three later calls took", free1 - free2)
assert free1 == free2, (free1, free2)
"""


def test_noalloc_later_calls_allocate_nothing_fresh_process():
    """In a process where nothing of the library has run yet, the first call
    is the set-up call; the free device memory does not move on the calls
    after it."""
    res = subprocess.run([sys.executable, "-c", _FRESH, ROOT], capture_output=True, text=True, timeout=600)
    assert res.returncode == 0, res.stdout + res.stderr
