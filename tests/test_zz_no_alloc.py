"""mb_seed_batch_noalloc: the entry point for callers that cannot allocate device memory
(their device memory is reserved by another allocator, or an allocation's possible device
synchronization is not acceptable on their path).  Its scratch is a fixed device array inside
the library; its output must equal mb_seed_batch's, record for record.

This file is collected last on purpose, so that a run stopping at the first failure has run
every other test before it."""
import ctypes

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def mb():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2606_15357_gb300 as m
    L = m.lib()
    P, U32, U64 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64
    PU64 = ctypes.POINTER(ctypes.c_uint64)
    L.mb_seed_batch_noalloc.argtypes = [P, P, P, U32, P, ctypes.POINTER(m.Opts), P, P, U64, PU64, PU64]
    L.mb_seed_batch_noalloc.restype = ctypes.c_int
    return m


def _dev(a):
    a = np.ascontiguousarray(a)
    return torch.from_numpy(a.view(np.int64) if a.dtype == np.uint64 else a).cuda()


def noalloc(mb, idx, seq, off, n_reads, cap, opts=None, mate=None):
    """Call the C entry point directly with device buffers; returns (records, n_smem, n_hits, rc)."""
    o = mb.Opts(**(opts or {}))
    out = torch.zeros(max(cap, 1) * 48, dtype=torch.uint8, device="cuda")
    n_out, n_hits = ctypes.c_uint64(), ctypes.c_uint64()
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    mp = ctypes.c_void_p(mate.data_ptr()) if mate is not None else None
    rc = mb.lib().mb_seed_batch_noalloc(idx.handle, ctypes.c_void_p(seq.data_ptr()),
                                        ctypes.c_void_p(off.data_ptr()), n_reads, mp, ctypes.byref(o),
                                        st, ctypes.c_void_p(out.data_ptr()), cap, ctypes.byref(n_out),
                                        ctypes.byref(n_hits))
    recs = out[:n_out.value * 48].cpu().numpy().view(mb.SMEM_DTYPE) if rc == 0 else None
    return recs, n_out.value, n_hits.value, rc


def test_noalloc_matches_allocating_entry_point_on_two_calls(mb):
    ref, rd, p = synth.workload(2, scale=0.003)
    idx = mb.mb_index_build(_dev(ref))
    first = rd.subset(np.arange(rd.n))
    second = rd.subset(np.arange(rd.n - 1, rd.n // 3, -1))   # another batch, other order and size
    for batch, opts in ((first, None), (second, dict(min_len=15, max_occ=20))):
        seq, off = _dev(batch.seq), _dev(batch.off)
        want, m, nh = mb.mb_seed_batch(idx, seq, off, opts=opts)
        got, m2, nh2, rc = noalloc(mb, idx, seq, off, batch.n, cap=m + 5, opts=opts)
        assert rc == 0
        assert (m2, nh2) == (m, nh)
        assert got.tobytes() == want.tobytes()


def test_noalloc_reads_with_more_smems_than_slots(mb):
    """Short minimum lengths give reads more SMEMs than their scratch slots, so those reads are
    recomputed by the overflow pass; the output still equals mb_seed_batch's."""
    ref = synth.reference(200_000, 81)
    idx = mb.mb_index_build(_dev(ref))
    n = 400
    seq = _dev(synth.reference(150 * n, 8200))              # random reads: they match only in pieces
    off = _dev(np.arange(n + 1, dtype=np.uint64) * 150)
    for opts in (dict(min_len=5, max_occ=50), dict(min_len=7, max_occ=3)):
        want, m, nh = mb.mb_seed_batch(idx, seq, off, opts=opts)
        assert m > 20 * n                                 # more records per read than its 17 slots
        for _ in range(2):
            got, m2, nh2, rc = noalloc(mb, idx, seq, off, n, cap=m, opts=opts)
            assert rc == 0 and (m2, nh2) == (m, nh)
            assert got.tobytes() == want.tobytes()


def test_noalloc_bisulfite_mates(mb):
    """The 3-base index with read 1 / read 2 conversion: same records as mb_seed_batch."""
    ref = synth.reference(40_000, 77)
    rd = synth.reads(ref, 300, 78, mode=1, read_len=150, bisulfite=True, sub_lo=0.001)
    o = dict(flags=mb.MB_BS3)
    idx = mb.mb_index_build(_dev(ref), opts=o)
    seq, off, mate = _dev(rd.seq), _dev(rd.off), _dev(rd.mate)
    want, m, nh = mb.mb_seed_batch(idx, seq, off, mate=mate, opts=o)
    got, m2, nh2, rc = noalloc(mb, idx, seq, off, rd.n, cap=m + 3, opts=o, mate=mate)
    assert rc == 0 and (m2, nh2) == (m, nh)
    assert got.tobytes() == want.tobytes()


def test_noalloc_capacity_reports_needed(mb):
    ref, rd, p = synth.workload(1, scale=0.01)
    idx = mb.mb_index_build(_dev(ref))
    seq, off = _dev(rd.seq), _dev(rd.off)
    _, m, nh = mb.mb_seed_batch(idx, seq, off)
    assert m > 1
    _, m2, _, rc = noalloc(mb, idx, seq, off, rd.n, cap=m - 1)
    assert rc == -3 and m2 == m                           # MB_ERR_CAPACITY with the needed count


def test_noalloc_rejects_batches_over_its_scratch(mb):
    ref = synth.reference(5000, 3)
    idx = mb.mb_index_build(_dev(ref))
    n = 1_000_000                                         # slots and per-read arrays: about 190 MB
    seq = _dev(np.zeros(16, np.uint8))
    off = _dev(np.zeros(n + 1, np.uint64))
    _, _, _, rc = noalloc(mb, idx, seq, off, n, cap=16)
    assert rc == -1
    assert b"scratch" in mb.lib().mb_last_error()


def test_noalloc_rejects_too_many_smems_after_seeding(mb):
    """Few long reads that fit the scratch but yield more SMEMs than it holds (a 300-base
    reference and min_len 1: an SMEM every few bases): the second check rejects the batch after
    seeding, with *n_out reset to 0."""
    ref = synth.reference(300, 5)
    reads = synth.reference(20_000_000, 6)
    n = 2000
    off_h = np.arange(n + 1, dtype=np.uint64) * (len(reads) // n)
    seq, off = _dev(reads), _dev(off_h)
    idx = mb.mb_index_build(_dev(ref))
    o = dict(min_len=1, max_occ=1_000_000)
    _, m, _, rc = noalloc(mb, idx, seq, off, n, cap=64, opts=o)
    assert rc == -3 and m > 5_000_000                      # first the needed count (about 0.6 per base)
    _, m2, _, rc = noalloc(mb, idx, seq, off, n, cap=m, opts=o)
    assert rc == -1 and m2 == 0                            # then the scratch limit
    assert b"SMEMs need" in mb.lib().mb_last_error()
