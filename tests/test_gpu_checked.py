"""Checks made before any bad access is issued: device buffers against their allocations (on
the host), read offsets and records' rows (always, on the device), and with MB_CHECKED every
occurrence row a kernel reads.  Every bad input here is made on the host; none reaches memory it
should not, and the library stays usable after each."""
import ctypes

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def mb():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2606_15357_gb300 as m
    m.lib()
    return m


@pytest.fixture(scope="module")
def small(mb):
    ref, rd, p = synth.workload(2, scale=0.002)
    G = mb.mb_index_build(ref)
    sm, hits = mb.seed(G, rd.seq, rd.off)
    return ref, rd, G, sm, hits


def dev(a):
    a = np.ascontiguousarray(a)
    return torch.from_numpy(a.view(np.int64) if a.dtype == np.uint64 else a).cuda()


def test_records_with_rows_outside_the_text(mb, small):
    """A record whose rows [k, k+s) leave the text is never walked: mb_locate returns
    MB_ERR_DEVICE_CHECK, and the next call on good records is exact."""
    ref, rd, G, sm, hits = small
    bad = sm.copy()
    q = int(np.nonzero((bad["flags"] & 1) == 0)[0][0])
    bad["k"][q] = G.n - 1
    bad["s"][q] = 5
    for buf in (bad, dev(bad.view(np.uint8))):
        with pytest.raises(mb.MbError) as ei:
            mb.mb_locate(G, buf, len(bad), cap=int(hits.size) + 16)
        assert ei.value.code == -8
    h, _ = mb.mb_locate(G, sm, len(sm), cap=len(hits))
    assert np.array_equal(h, hits)


def test_decreasing_offsets(mb, small):
    """Offsets that decrease inside the batch: the read is skipped on the device and the call
    returns MB_ERR_DEVICE_CHECK (host and device buffers, with and without MB_CHECKED)."""
    ref, rd, G, sm, hits = small
    sub = rd.subset(np.arange(20))
    off = sub.off.copy()
    off[5], off[6] = off[6], off[5]          # read 5 ends before it starts
    for flags in (0, mb.MB_CHECKED):
        for s_, o_ in ((sub.seq, off), (dev(sub.seq), dev(off))):
            with pytest.raises(mb.MbError) as ei:
                mb.mb_seed_batch(G, s_, o_, opts=dict(flags=flags))
            assert ei.value.code == -8
    want, _, _ = mb.mb_seed_batch(G, sub.seq, sub.off)
    got, _, _ = mb.mb_seed_batch(G, sub.seq, sub.off)
    assert got.tobytes() == want.tobytes()


def test_offsets_past_the_device_buffer(mb, small):
    """off[n] far past the end of the device read buffer: refused on the host (MB_ERR_ARG) before
    any copy or kernel; the same for an `off` array shorter than n_reads + 1 and an output buffer
    smaller than the records.  Runs only where the driver reports allocation extents."""
    ref, rd, G, sm, hits = small
    seq = dev(rd.seq[:1000])
    b, z = ctypes.c_uint64(), ctypes.c_uint64()
    if mb.lib().mb_device_extent(ctypes.c_void_p(seq.data_ptr()), ctypes.byref(b), ctypes.byref(z)) != 0:
        pytest.skip("the driver does not report allocation extents")
    assert b.value <= seq.data_ptr() and seq.data_ptr() + 1000 <= b.value + z.value
    past = int(b.value + z.value - seq.data_ptr()) + (1 << 20)
    off = dev(np.array([0, 150, past], dtype=np.uint64))
    with pytest.raises(mb.MbError) as ei:
        mb.mb_seed_batch(G, seq, off)
    assert ei.value.code == -1 and b"allocation" in mb.lib().mb_last_error()
    short = dev(np.array([0, 150], dtype=np.uint64))
    L = mb.lib()
    n_out, n_hits = ctypes.c_uint64(), ctypes.c_uint64()
    sb, sz = ctypes.c_uint64(), ctypes.c_uint64()
    assert L.mb_device_extent(ctypes.c_void_p(short.data_ptr()), ctypes.byref(sb), ctypes.byref(sz)) == 0
    huge = int((sb.value + sz.value - short.data_ptr()) // 8) + 1024   # more offsets than its allocation holds
    rc = L.mb_seed_batch(G.handle, ctypes.c_void_p(seq.data_ptr()), ctypes.c_void_p(short.data_ptr()), huge,
                         None, ctypes.byref(mb.Opts()), None, None, 0, ctypes.byref(n_out), ctypes.byref(n_hits))
    assert rc == -1
    # an output buffer too small for the records it is declared to hold
    sub = rd.subset(np.arange(50))
    _, m, _ = mb.mb_seed_batch(G, sub.seq, sub.off)
    small_out = torch.empty(48, dtype=torch.uint8, device="cuda")
    e2 = ctypes.c_uint64()
    if L.mb_device_extent(ctypes.c_void_p(small_out.data_ptr()), ctypes.byref(b), ctypes.byref(e2)) == 0 and \
            b.value + e2.value - small_out.data_ptr() < m * 48:
        with pytest.raises(mb.MbError) as ei:
            mb.mb_seed_batch(G, dev(sub.seq), dev(sub.off), out=small_out, cap=m)
        assert ei.value.code == -1
    # the library is still usable
    got, _, _ = mb.mb_seed_batch(G, sub.seq, sub.off)
    assert len(got) == m


def test_checked_mode_same_output(mb, small):
    """MB_CHECKED changes no result on a sound index: SMEMs, hits, plan form and the no-allocation
    entry point match the unchecked calls and the oracle."""
    ref, rd, G, sm, hits = small
    o = dict(flags=mb.MB_CHECKED)
    csm, chits = mb.seed(G, rd.seq, rd.off, opts=o)
    assert csm.tobytes() == sm.tobytes() and np.array_equal(chits, hits)
    P = mb.Plan(G, rd.n, len(rd.seq), len(sm) + 8, len(hits) + 8, opts=dict(flags=mb.MB_CHECKED | mb.MB_BATCHED))
    P.run(dev(rd.seq), dev(rd.off))
    psm, phits = P.result()
    assert psm.tobytes() == sm.tobytes() and np.array_equal(phits, hits)
    X = oracle.Index(ref)
    osm, over, hoff, ohits = X.seed(rd.seq, rd.off)
    assert np.array_equal(csm["k"].astype(np.uint64), osm["k"]) and np.array_equal(chits.astype(np.uint64), ohits)
