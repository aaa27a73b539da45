"""mb_seed_locate: the whole stage in one pipelined call over chunks on two streams.

Its records and hits must be those of the oracle (Algorithm 3 SMEMs, max-occ flag, hit offsets,
Algorithm 2 positions) and, byte for byte, those of mb_seed_batch + mb_locate, whatever the chunk
size, with host or device buffers, and when a chunk outgrows its plan."""
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


def dev(a):
    a = np.ascontiguousarray(a)
    return torch.from_numpy(a.view(np.int64) if a.dtype == np.uint64 else a).cuda()


def check_oracle(sm, hits, X, seq, off):
    osm, over, hoff, ohits = X.seed(seq, off)
    assert len(sm) == len(osm)
    for f in ("read", "qbeg", "qend", "k", "kr", "s"):
        assert np.array_equal(sm[f].astype(np.uint64), osm[f]), f
    assert np.array_equal((sm["flags"] & 1).astype(bool), over)
    assert np.array_equal(sm["hit_off"].astype(np.uint64), hoff)
    assert np.array_equal(hits.astype(np.uint64), ohits)


@pytest.fixture(scope="module")
def repeat_rich(mb):
    ref, rd, p = synth.workload(2, scale=0.02)   # 2 Mbp repeat-rich, 20,000 paired reads
    G = mb.mb_index_build(ref)
    return ref, rd, G


@pytest.mark.parametrize("flags", [0, 0x100, 0x200])
@pytest.mark.parametrize("chunk", [997, 4096, 0])
def test_host_buffers_against_oracle_and_plain(mb, repeat_rich, chunk, flags):
    """mb_seed_locate on host buffers, plain walks, walks that join (MB_LOCATE_JOIN, 0x100) or
    walks to the rate-4 samples (MB_LOCATE_AUX, 0x200)."""
    ref, rd, G = repeat_rich
    o = dict(chunk_reads=chunk, prefetch_depth=4, flags=flags)
    sm, hits = mb.seed_locate(G, rd.seq, rd.off, opts=o)
    check_oracle(sm, hits, oracle.Index(ref), rd.seq, rd.off)
    psm, phits = mb.seed(G, rd.seq, rd.off)
    assert sm.tobytes() == psm.tobytes()
    assert np.array_equal(hits, phits)


def test_several_slices(mb, repeat_rich, monkeypatch):
    """Slices of at most 3,000 reads (MB_SLICE_READS lowers the 2^25 default): each slice is
    located on its own and its records' hit offsets are made batch-wide after its locate."""
    ref, rd, G = repeat_rich
    monkeypatch.setenv("MB_SLICE_READS", "3000")
    psm, phits = mb.seed(G, rd.seq, rd.off)
    for chunk in (1000, 2999, 0):
        o = dict(chunk_reads=chunk, flags=mb.MB_LOCATE_JOIN if chunk == 2999 else 0)
        sm, hits = mb.seed_locate(G, rd.seq, rd.off, opts=o)
        assert sm.tobytes() == psm.tobytes()
        assert np.array_equal(hits, phits)
    out = torch.empty(len(psm) * 48, dtype=torch.uint8, device="cuda")
    dh = torch.empty(len(phits), dtype=torch.int32, device="cuda")
    mb.seed_locate(G, dev(rd.seq), dev(rd.off), opts=dict(chunk_reads=1500), out=out, cap=len(psm), hits=dh,
                   hits_cap=len(phits))
    assert out.cpu().numpy().tobytes() == psm.tobytes()
    assert np.array_equal(dh.cpu().numpy().view(np.uint32), phits)


def test_pinned_and_device_buffers(mb, repeat_rich):
    ref, rd, G = repeat_rich
    psm, phits = mb.seed(G, rd.seq, rd.off)
    # pinned host in, device out
    seq_h = torch.from_numpy(rd.seq).pin_memory()
    off_h = torch.from_numpy(rd.off.view(np.int64)).pin_memory()
    out = torch.empty(len(psm) * 48, dtype=torch.uint8, device="cuda")
    hits = torch.empty(len(phits), dtype=torch.int32, device="cuda")
    m, nh = mb.seed_locate(G, seq_h, off_h, opts=dict(chunk_reads=3001), out=out, cap=len(psm), hits=hits,
                           hits_cap=len(phits))
    assert (m, nh) == (len(psm), len(phits))
    assert out.cpu().numpy().tobytes() == psm.tobytes()
    assert np.array_equal(hits.cpu().numpy().view(np.uint32), phits)
    # device in, pinned host out
    out_h = torch.empty(len(psm) * 48, dtype=torch.uint8).pin_memory()
    hits_h = torch.empty(len(phits), dtype=torch.int32).pin_memory()
    m, nh = mb.seed_locate(G, dev(rd.seq), dev(rd.off), opts=dict(chunk_reads=2500), out=out_h, cap=len(psm),
                           hits=hits_h, hits_cap=len(phits))
    assert out_h.numpy().tobytes() == psm.tobytes()
    assert np.array_equal(hits_h.numpy().view(np.uint32), phits)


def test_chunk_outgrows_its_plan(mb):
    """A reference of 300 near-identical copies of one 1.5 kb unit: reads have hundreds of hits,
    more than the per-chunk plan is sized for, so every chunk takes the allocating path."""
    rng = np.random.default_rng(91)
    unit = synth.reference(1500, 92)
    copies = []
    for _ in range(300):
        u = unit.copy()
        pos = rng.choice(len(u), 3, replace=False)
        u[pos] = (u[pos] + rng.integers(1, 4, 3)) % 4
        copies.append(u)
    ref = np.concatenate([synth.reference(5000, 93)] + copies + [synth.reference(5000, 94)]).astype(np.uint8)
    rd = synth.reads(ref, 600, 95, mode=0, read_len=150, sub_lo=0.002)
    G = mb.mb_index_build(ref)
    sm, hits = mb.seed_locate(G, rd.seq, rd.off, opts=dict(chunk_reads=40))
    assert len(hits) / (rd.n / 40) > 4 * (4 * 40 + 6000 // 32 + 64)   # more per chunk than its plan holds
    check_oracle(sm, hits, oracle.Index(ref), rd.seq, rd.off)


def test_records_outgrow_the_plan(mb):
    """Reads that match nowhere at length 150 but everywhere at length 5: with min_len 5 each read
    has dozens of SMEMs, more records per chunk than the chunk's plan holds, so every chunk takes
    the allocating path; the slice is still located at once."""
    ref = synth.reference(200_000, 81)
    reads = [synth.reference(150, 8200 + q) for q in range(300)]
    seq = np.concatenate(reads).astype(np.uint8)
    off = np.concatenate([[0], np.cumsum([len(r) for r in reads])]).astype(np.uint64)
    o = dict(min_len=5, max_occ=50)
    G = mb.mb_index_build(ref)
    sm, hits = mb.seed_locate(G, seq, off, opts=dict(o, chunk_reads=50))
    assert len(sm) / (300 / 50) > 4 * (4 * 50 + 7500 // 32 + 64)   # far more per chunk than its plan holds
    psm, phits = mb.seed(G, seq, off, opts=o)
    assert sm.tobytes() == psm.tobytes()
    assert np.array_equal(hits, phits)
    osm, over, hoff, ohits = oracle.Index(ref).seed(seq, off, min_len=5, max_occ=50)
    assert np.array_equal(sm["k"].astype(np.uint64), osm["k"]) and np.array_equal(hits.astype(np.uint64), ohits)


@pytest.mark.slow
def test_late_chunk_outgrows_its_plan_at_a_large_offset(mb):
    """Host buffers of 450 MB: five chunks of error-free reads (one SMEM each), then a chunk of
    random reads with min_len 5 (dozens of SMEMs each, more than its plan holds) starting 375 MB
    into the batch.  That chunk is seeded again by the allocating path on its device inputs; the
    output equals mb_seed_batch + mb_locate on the whole batch."""
    ref = synth.reference(200_000, 83)
    n_chunk = 500_000
    filler = synth.reads(ref, 5 * n_chunk, 84, mode=0, read_len=150)
    rand = synth.reference(150 * n_chunk, 85)
    seq = np.concatenate([filler.seq, rand]).astype(np.uint8)
    off = np.concatenate([filler.off, filler.off[-1] + 150 * np.arange(1, n_chunk + 1, dtype=np.uint64)])
    o = dict(min_len=5, max_occ=50)
    G = mb.mb_index_build(ref)
    sm, hits = mb.seed_locate(G, seq, off, opts=dict(o, chunk_reads=n_chunk))
    last = sm["read"] >= 5 * n_chunk
    assert int(off[5 * n_chunk]) == 375_000_000
    assert last.sum() > 4 * n_chunk + 150 * n_chunk // 32 + 64   # more than the chunk's plan holds
    psm, phits = mb.seed(G, seq, off, opts=o)
    assert sm.tobytes() == psm.tobytes()
    assert np.array_equal(hits, phits)


def test_capacity_reports_both_totals(mb, repeat_rich):
    ref, rd, G = repeat_rich
    psm, phits = mb.seed(G, rd.seq, rd.off)
    out = np.empty(len(psm), dtype=mb.SMEM_DTYPE)
    hits = np.empty(max(1, len(phits) // 2), dtype=np.uint32)
    n_out, n_hits = ctypes.c_uint64(), ctypes.c_uint64()
    o = mb.Opts(chunk_reads=5000)
    rc = mb.lib().mb_seed_locate(G.handle, mb._ptr(rd.seq), mb._ptr(rd.off), rd.n, None, ctypes.byref(o), None,
                                 mb._ptr(out), len(out), mb._ptr(hits), len(hits), ctypes.byref(n_out),
                                 ctypes.byref(n_hits))
    assert rc == -3
    assert (n_out.value, n_hits.value) == (len(psm), len(phits))


def test_bisulfite_mates(mb):
    ref = synth.reference(50_000, 71)
    rd = synth.reads(ref, 600, 72, mode=1, read_len=150, bisulfite=True, sub_lo=0.001)
    o = dict(flags=mb.MB_BS3, chunk_reads=77)
    G = mb.mb_index_build(ref, opts=o)
    sm, hits = mb.seed_locate(G, rd.seq, rd.off, mate=rd.mate, opts=o)
    psm, m, nh = mb.mb_seed_batch(G, rd.seq, rd.off, mate=rd.mate, opts=o)
    phits, _ = mb.mb_locate(G, psm, m, opts=o, cap=nh)
    assert sm.tobytes() == psm.tobytes()
    assert np.array_equal(hits, phits)
    conv = oracle.bs_convert_reads(rd.seq, rd.off, rd.mate)
    check_oracle(sm, hits, oracle.Index(ref, bs3=True), conv, rd.off)


def test_workspace_kept_between_calls(mb, repeat_rich):
    """Repeated calls reuse the kept workspace (same results), also after other options in between."""
    ref, rd, G = repeat_rich
    psm, phits = mb.seed(G, rd.seq, rd.off)
    for o in (dict(chunk_reads=3000), dict(chunk_reads=3000), dict(chunk_reads=1000, prefetch_depth=4),
              dict(chunk_reads=3000), dict(chunk_reads=2000, block_size=128), dict(chunk_reads=3000)):
        sm, hits = mb.seed_locate(G, rd.seq, rd.off, opts=o)
        assert sm.tobytes() == psm.tobytes()
        assert np.array_equal(hits, phits)


def test_edge_reads_and_empty_batch(mb):
    ref = synth.reference(20_000, 61)
    G = mb.mb_index_build(ref)
    reads = [np.zeros(0, np.uint8), ref[100:118], ref[200:219], np.zeros(0, np.uint8), ref[300:320],
             np.full(150, 4, np.uint8), np.concatenate([ref[400:450], [4], ref[451:500]]),
             ref[1000:1150], synth.reference(150, 999), np.zeros(0, np.uint8)]
    seq = np.concatenate(reads).astype(np.uint8)
    off = np.concatenate([[0], np.cumsum([len(r) for r in reads])]).astype(np.uint64)
    for chunk in (1, 2, 3, 0):
        sm, hits = mb.seed_locate(G, seq, off, opts=dict(chunk_reads=chunk))
        check_oracle(sm, hits, oracle.Index(ref), seq, off)
    sm, hits = mb.seed_locate(G, seq, off[:1])
    assert len(sm) == 0 and len(hits) == 0
