"""GPU path against the CPU oracle, through the C ABI.

Every field is integer: the bar is bit-exact equality (SA, BWT, occurrence
counts, sampled SA, k-mer table, SMEM records, max-occ flags, hit offsets,
hit positions).
"""
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
    if a.dtype == np.uint64:
        return torch.from_numpy(a.view(np.int64)).cuda()
    return torch.from_numpy(a).cuda()


def compare_index(G, X, k=10):
    e = G.export(sa=True, bwt=True, ssa=True, occ=True, kmer=True, kmer_k=k)
    assert G.n == X.n and G.primary == X.primary
    assert np.array_equal(e["sa"], X.sa())
    assert np.array_equal(e["bwt"], X.bwt())
    assert np.array_equal(e["ssa"], X.ssa())
    assert np.array_equal(e["C"], X.C)
    # block counts: #a in B[0, 64b) excluding $ (32-byte blocks: four u32 counts, two bit planes)
    B = X.bwt()
    occ = e["occ"].view(np.uint32).reshape(-1, 8)
    assert len(occ) == X.n // 64 + 1
    for a in range(4):
        cum = np.concatenate([[0], np.cumsum(B == a + 1)])
        assert np.array_equal(occ[:, a].astype(np.uint64), cum[np.arange(len(occ)) * 64].astype(np.uint64))
    # bit planes: row q of block b has code ((lo >> q) & 1) | ((hi >> q) & 1) << 1, $ as A, A after the end
    planes = e["occ"].view(np.uint64).reshape(-1, 4)[:, 2:]
    q = np.arange(64, dtype=np.uint64)
    codes = (((planes[:, :1] >> q) & 1) | (((planes[:, 1:] >> q) & 1) << 1)).reshape(-1)
    want = np.zeros(len(codes), np.uint64)
    want[:X.n] = np.where(B == 0, 0, B.astype(np.int64) - 1)
    assert np.array_equal(codes, want)
    # k-mer table against the definition
    nk = 4 ** k
    words = np.arange(nk, dtype=np.int64)
    pats = np.stack([(words >> (2 * t)) & 3 for t in range(k)], axis=1).astype(np.uint8)   # base t in bits 2t
    want = X.ds_intervals(pats).astype(np.uint32)
    got = e["kmer"].reshape(nk, 3)
    assert np.array_equal(got, want)


def compare_seed(sm, hits, X, seq, off, l=19, c=1, max_occ=500):
    osm, over, hoff, ohits = X.seed(seq, off, l, c, max_occ)
    assert len(sm) == len(osm)
    for f in ("read", "qbeg", "qend", "k", "kr", "s"):
        assert np.array_equal(sm[f].astype(np.uint64), osm[f]), f
    assert np.array_equal((sm["flags"] & 1).astype(bool), over)
    assert np.array_equal(sm["hit_off"], hoff)
    assert np.array_equal(np.asarray(hits).astype(np.uint64), ohits)


@pytest.mark.parametrize("length", [1, 2, 3, 100, 127, 128, 129, 1000, 4095])
def test_index_tiny_lengths(mb, length):
    ref = synth.reference(length, 1000 + length)
    G = mb.mb_index_build(ref, n_seed=3)
    X = oracle.Index(ref, n_seed=3)
    compare_index(G, X)


def test_index_repeat_rich_with_n(mb):
    ref = synth.repeat_rich_reference(300_000, 41, 0.45)
    assert (ref == 4).any()
    G = mb.mb_index_build(dev(ref), n_seed=77)
    X = oracle.Index(ref, n_seed=77)
    compare_index(G, X)


def test_index_periodic_text(mb):
    # one short unit repeated: common prefixes of tens of thousands of symbols force many
    # prefix-doubling rounds
    ref = np.tile(synth.reference(7, 5), 6000)
    G = mb.mb_index_build(ref)
    X = oracle.Index(ref)
    compare_index(G, X)


def test_workload1_full(mb):
    """1 Mbp uniform reference, 10,000 single-end 150 bp reads, 0.5% substitutions."""
    ref, rd, p = synth.workload(1)
    G = mb.mb_index_build(ref)
    X = oracle.Index(ref)
    compare_index(G, X)
    sm, hits = mb.seed(G, rd.seq, rd.off)
    compare_seed(sm, hits, X, rd.seq, rd.off)


@pytest.mark.parametrize("form", ["plain", "join", "aux"])
@pytest.mark.parametrize("depth", [1, 2, 4, 8, 16])
def test_locate_walks_per_lane(mb, depth, form):
    """Locate with 1, 2, 4, 8 or 16 LF-walks in flight per lane, plain, with walks that join
    (MB_LOCATE_JOIN) or with walks to the rate-4 samples (MB_LOCATE_AUX), gives the same hits."""
    ref, rd, p = synth.workload(2, scale=0.01)
    G = mb.mb_index_build(ref)
    X = oracle.Index(ref)
    sm, m, nh = mb.mb_seed_batch(G, rd.seq, rd.off)
    flags = {"plain": 0, "join": mb.MB_LOCATE_JOIN, "aux": mb.MB_LOCATE_AUX}[form]
    o = dict(prefetch_depth=depth, flags=flags)
    hits, _ = mb.mb_locate(G, sm, m, opts=o, cap=nh)
    compare_seed(sm, hits, X, rd.seq, rd.off)
    if form != "plain":   # the same through a plan
        P = mb.Plan(G, rd.n, len(rd.seq), m + 8, nh + 8, opts=o)
        P.run(torch.from_numpy(rd.seq).cuda(), torch.from_numpy(rd.off.view(np.int64)).cuda())
        psm, phits = P.result()
        assert psm.tobytes() == sm.tobytes() and np.array_equal(phits, hits)


def test_locate_aux_on_an_index_without_aux_arrays(mb):
    """MB_LOCATE_AUX on an index built with MB_NO_AUX walks to the rate-32 samples: same hits."""
    ref, rd, p = synth.workload(2, scale=0.005)
    G = mb.mb_index_build(ref, opts=dict(flags=mb.MB_NO_AUX))
    sm, m, nh = mb.mb_seed_batch(G, rd.seq, rd.off)
    want, _ = mb.mb_locate(G, sm, m, cap=nh)
    mb.profile_reset()
    got, _ = mb.mb_locate(G, sm, m, opts=dict(flags=mb.MB_LOCATE_AUX | mb.MB_COUNT), cap=nh)
    assert np.array_equal(got, want)
    keep = (sm["flags"] & 1) == 0
    rows = np.unique(np.concatenate([np.arange(int(k), int(k) + int(s_), dtype=np.uint64)
                                     for k, s_ in zip(sm["k"][keep], sm["s"][keep])]))
    wc = mb.work_counters()
    assert (wc["lf_steps"], wc["sa_reads"]) == oracle.Index(ref).count_locate(rows)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_locate_shared_rows_any_intervals(mb, seed):
    """Locate walks each distinct row once and copies the position to every hit: records with
    duplicated, nested, partially overlapping and adjacent intervals, records over max_occ and
    empty ones, in shuffled order, all get Algorithm 2's positions (the oracle's full suffix
    array) for every row."""
    ref, rd, p = synth.workload(2, scale=0.005)
    G = mb.mb_index_build(ref)
    X = oracle.Index(ref)
    S = X.sa()
    rng = np.random.default_rng(seed)
    n = X.n
    recs = []
    for _ in range(3000):
        kind = rng.integers(0, 6)
        k = int(rng.integers(0, n - 1200))          # every row stays below n
        s = int(rng.integers(1, 400))
        recs.append((k, s))
        if kind == 1:                                   # the same interval again
            recs.append((k, s))
        elif kind == 2:                                 # nested inside
            a = int(rng.integers(0, s))
            recs.append((k + a, int(rng.integers(1, s - a + 1))))
        elif kind == 3:                                 # overlapping past the end
            a = int(rng.integers(1, s + 1))
            recs.append((k + a, s + int(rng.integers(1, 100))))
        elif kind == 4:                                 # adjacent
            recs.append((k + s, int(rng.integers(1, 50))))
        elif kind == 5:                                 # a single row inside
            recs.append((k + int(rng.integers(0, s)), 1))
    order = rng.permutation(len(recs))
    sm = np.zeros(len(recs), dtype=mb.SMEM_DTYPE)
    sm["k"] = [recs[i][0] for i in order]
    sm["s"] = [recs[i][1] for i in order]
    sm["read"] = np.arange(len(recs))
    over = rng.random(len(recs)) < 0.05
    sm["flags"][over] = mb.MB_SMEM_OVER_MAX_OCC
    sm["s"][rng.random(len(recs)) < 0.02] = 0
    cnt = np.where(over, 0, sm["s"]).astype(np.uint64)
    sm["hit_off"] = np.concatenate([[0], np.cumsum(cnt)[:-1]])
    rows = np.concatenate([np.arange(int(k), int(k) + int(c), dtype=np.int64) for k, c in zip(sm["k"], cnt)])
    assert len(np.unique(rows)) < len(rows)
    for depth in (1, 16):
        for flags in (0, mb.MB_LOCATE_JOIN):
            hits, nh = mb.mb_locate(G, sm, len(sm), opts=dict(prefetch_depth=depth, flags=flags),
                                    cap=int(cnt.sum()))
            assert nh == len(rows)
            assert np.array_equal(hits.astype(np.int64), S[rows].astype(np.int64))
    dsm = torch.from_numpy(sm.view(np.uint8)).cuda()
    out = torch.empty(len(rows), dtype=torch.int32, device="cuda")
    mb.mb_locate(G, dsm, len(sm), hits=out, cap=len(rows))
    assert np.array_equal(out.cpu().numpy().view(np.uint32).astype(np.int64), S[rows].astype(np.int64))


@pytest.mark.parametrize("k", [12, 14, 16])
def test_larger_kmer_tables(mb, k):
    """k-mer tables above the paper's k = 10 (12 * 4^k bytes: 3.2 GB at k = 14, 51.5 GB at
    k = 16): sampled entries against the oracle's ds-intervals, and the same SMEMs and hits as
    without a table."""
    ref, rd, p = synth.workload(2, scale=0.005)
    G = mb.mb_index_build(ref, opts=dict(kmer_k=k))
    X = oracle.Index(ref)
    words = np.sort(np.random.default_rng(k).choice(4 ** k, 50_000, replace=False)).astype(np.int64)
    present = X.ds_intervals(np.stack([(words >> (2 * t)) & 3 for t in range(k)], axis=1).astype(np.uint8))
    # k-mers of the reference itself, so that most sampled entries are not empty
    starts = np.random.default_rng(k + 1).integers(0, len(ref) - k, 20_000)
    win = ref[starts[:, None] + np.arange(k)].astype(np.int64)
    ok = (win < 4).all(axis=1)
    rw = (win[ok] << (2 * np.arange(k))).sum(axis=1)
    allw = np.concatenate([words, rw])
    want = np.concatenate([present, X.ds_intervals(win[ok].astype(np.uint8))]).astype(np.uint32)
    assert np.array_equal(G.kmer_get(allw), want)
    assert (want[:, 2] > 0).sum() >= len(rw)
    sm, hits = mb.seed(G, rd.seq, rd.off)
    compare_seed(sm, hits, X, rd.seq, rd.off)
    nsm, nhits = mb.seed(G, rd.seq, rd.off, opts=dict(flags=mb.MB_NO_KMER))
    assert sm.tobytes() == nsm.tobytes() and np.array_equal(hits, nhits)
    with pytest.raises(mb.MbError):
        G.kmer_get([4 ** k])


def test_work_counters_match_oracle(mb):
    """The counts behind the bench's algorithmic bytes: the GPU's counting kernels (no k-mer
    table, so Algorithm 3 runs step by step as in the oracle) report the same extension steps,
    blocks read, LF steps and sampled-S reads as the oracle's own counts on the same reads.
    Locate walks each distinct row once, so its counts are Algorithm 2's over the distinct rows."""
    ref, rd, p = synth.workload(2, scale=0.005)
    G = mb.mb_index_build(ref)
    X = oracle.Index(ref)
    mb.profile_reset()
    o = dict(flags=mb.MB_COUNT | mb.MB_NO_KMER | mb.MB_STEP_ONLY)
    sm, m, nh = mb.mb_seed_batch(G, rd.seq, rd.off, opts=o)
    mb.mb_locate(G, sm, m, opts=o, cap=nh)
    wc = mb.work_counters()
    assert wc["kmer_lookups"] == 0 and wc["u_walk_steps"] == wc["u_samples"] == wc["u_text_loads"] == 0
    assert (wc["ext_steps"], wc["ext_blocks"]) == X.count_alg3(rd.seq, rd.off)
    keep = (sm["flags"] & 1) == 0
    rows = np.concatenate([np.arange(int(k), int(k) + int(s), dtype=np.uint64)
                           for k, s in zip(sm["k"][keep], sm["s"][keep])])
    assert len(np.unique(rows)) < len(rows)   # the repeat-rich reads repeat rows
    assert (wc["lf_steps"], wc["sa_reads"]) == X.count_locate(np.unique(rows))
    # walks that join in 8 passes (MB_LOCATE_JOIN): LF steps, S reads and joins as the oracle counts
    mb.profile_reset()
    mb.mb_locate(G, sm, m, opts=dict(flags=mb.MB_COUNT | mb.MB_LOCATE_JOIN), cap=nh)
    wc = mb.work_counters()
    assert (wc["lf_steps"], wc["sa_reads"], wc["joins"]) == X.count_locate_join(np.unique(rows), pass_bits=3)
    assert wc["joins"] > 0 and wc["joins_off"] == 0
    # walks to the rate-4 samples (MB_LOCATE_AUX): Algorithm 2's counts with r = 4
    mb.profile_reset()
    mb.mb_locate(G, sm, m, opts=dict(flags=mb.MB_COUNT | mb.MB_LOCATE_AUX), cap=nh)
    wc = mb.work_counters()
    assert (wc["lf_steps"], wc["sa_reads"]) == oracle.Index(ref, sa_rate=4).count_locate(np.unique(rows))
    assert wc["joins"] == 0
    # with the index's 10-mer table (Section 2.5): the same steps, blocks and lookups as the
    # oracle's Algorithm 3 with the cache
    mb.profile_reset()
    o = dict(flags=mb.MB_COUNT | mb.MB_STEP_ONLY)
    mb.mb_seed_batch(G, rd.seq, rd.off, opts=o)
    wc = mb.work_counters()
    assert (wc["ext_steps"], wc["ext_blocks"], wc["kmer_lookups"]) == X.count_alg3(rd.seq, rd.off, kmer_k=10)


def test_auxiliary_arrays_and_text_extension(mb):
    """The packed text and the rate-4 SA / ISA samples against the oracle's text and suffix array;
    SMEMs and hits are the same whether unique matches are extended by comparing text, step by
    step (MB_STEP_ONLY), or on an index without the arrays (MB_NO_AUX)."""
    ref, rd, p = synth.workload(2, scale=0.01)
    G = mb.mb_index_build(ref)
    X = oracle.Index(ref)
    t2, sx, ix = G.export_aux()
    T = X.text().astype(np.int64) - 1          # oracle coding $=0, A..T=1..4
    want = np.zeros(len(t2) * 16, np.int64)
    want[:X.n - 1] = T[:X.n - 1]
    packed = (want.reshape(-1, 16) << (2 * np.arange(16))).sum(axis=1).astype(np.uint32)
    assert np.array_equal(t2, packed)
    S = X.sa().astype(np.int64)
    assert np.array_equal(sx, S[::mb.AUX_RATE].astype(np.uint32))
    isa = np.empty(X.n, np.int64)
    isa[S] = np.arange(X.n)
    assert np.array_equal(ix, isa[::mb.AUX_RATE].astype(np.uint32))
    mb.profile_reset()
    sm, hits = mb.seed(G, rd.seq, rd.off, opts=dict(flags=mb.MB_COUNT))
    wc = mb.work_counters()
    assert wc["u_walk_steps"] > 0 and wc["u_text_loads"] > 0
    compare_seed(sm, hits, X, rd.seq, rd.off)
    sm2, hits2 = mb.seed(G, rd.seq, rd.off)
    sm3, hits3 = mb.seed(G, rd.seq, rd.off, opts=dict(flags=mb.MB_STEP_ONLY))
    N = mb.mb_index_build(ref, opts=dict(flags=mb.MB_NO_AUX))
    sm4, hits4 = mb.seed(N, rd.seq, rd.off)
    for a, b in ((sm2, hits2), (sm3, hits3), (sm4, hits4)):
        assert a.tobytes() == sm.tobytes() and np.array_equal(b, hits)
    with pytest.raises(mb.MbError):
        N.export_aux()


def test_workload2_scaled_device_pointers(mb):
    """Repeat-rich reference with N runs, paired 2x150 reads with indels; device buffers."""
    ref, rd, p = synth.workload(2, scale=0.02)
    G = mb.mb_index_build(dev(ref))
    X = oracle.Index(ref)
    seq, off = dev(rd.seq), dev(rd.off)
    out = torch.empty(rd.n * 8 * 48, dtype=torch.uint8, device="cuda")
    out, m, nh = mb.mb_seed_batch(G, seq, off, out=out, cap=rd.n * 8)
    hits = torch.empty(max(nh, 1), dtype=torch.int32, device="cuda")
    mb.mb_locate(G, out, m, hits=hits, cap=nh)
    sm = out[:m * 48].cpu().numpy().view(mb.SMEM_DTYPE)
    compare_seed(sm, hits[:nh].cpu().numpy().view(np.uint32), X, rd.seq, rd.off)


def test_workload4_mixed_lengths(mb):
    """Log-uniform 100 bp - 10 kb reads in one batch (reads that overflow their slots)."""
    ref, rd, p = synth.workload(4, scale=0.004)
    G = mb.mb_index_build(ref)
    X = oracle.Index(ref)
    sm, hits = mb.seed(G, rd.seq, rd.off)
    compare_seed(sm, hits, X, rd.seq, rd.off)


@pytest.mark.parametrize("l,c,max_occ", [(1, 1, 500), (5, 1, 3), (19, 2, 500), (12, 3, 50),
                                         (30, 1, 500)])
def test_parameters_and_overflow(mb, l, c, max_occ):
    ref = synth.repeat_rich_reference(40_000, 51, 0.3)
    rd = synth.reads(ref, 300, 52, mode=0, read_len=150, sub_lo=0.02, indel=0.002)
    G = mb.mb_index_build(ref)
    X = oracle.Index(ref)
    o = dict(min_len=l, min_occ=c, max_occ=max_occ)
    sm, hits = mb.seed(G, rd.seq, rd.off, opts=o)
    compare_seed(sm, hits, X, rd.seq, rd.off, l, c, max_occ)


def test_edge_reads(mb):
    ref = synth.reference(20_000, 61)
    G = mb.mb_index_build(ref)
    X = oracle.Index(ref)
    reads = [np.zeros(0, np.uint8), ref[100:118], ref[200:219], ref[300:320],
             np.full(150, 4, np.uint8), np.concatenate([ref[400:450], [4], ref[451:500]]),
             ref[1000:1150], synth.reference(150, 999)]
    seq = np.concatenate(reads).astype(np.uint8)
    off = np.concatenate([[0], np.cumsum([len(r) for r in reads])]).astype(np.uint64)
    sm, hits = mb.seed(G, seq, off)
    compare_seed(sm, hits, X, seq, off)
    # any code above 3 is an N: codes 5..255 in place of 4 give the same records and hits
    rng = np.random.default_rng(62)
    odd = seq.copy()
    ns = odd == 4
    odd[ns] = rng.integers(5, 256, int(ns.sum())).astype(np.uint8)
    odd[300:302] = (9, 200)   # two more inside an exact read
    same = seq.copy()
    same[300:302] = 4
    osm, ohits = mb.seed(G, odd, off)
    ssm, shits = mb.seed(G, same, off)
    assert osm.tobytes() == ssm.tobytes() and np.array_equal(ohits, shits)
    # empty batch
    e, m, nh = mb.mb_seed_batch(G, seq, off[:1])
    assert m == 0 and nh == 0


def test_capacity_error_reports_needed(mb):
    ref, rd, p = synth.workload(1, scale=0.01)
    G = mb.mb_index_build(ref)
    buf = np.empty(1, dtype=mb.SMEM_DTYPE)
    with pytest.raises(mb.MbError) as ei:
        mb.mb_seed_batch(G, rd.seq, rd.off, out=buf, cap=1)
    assert ei.value.code == -3


def test_bisulfite_index_and_seeding(mb):
    ref = synth.reference(50_000, 71)
    rd = synth.reads(ref, 400, 72, mode=1, read_len=150, bisulfite=True, sub_lo=0.001)
    o = dict(flags=mb.MB_BS3)
    G = mb.mb_index_build(ref, opts=o)
    X = oracle.Index(ref, bs3=True)
    compare_index(G, X)
    conv = oracle.bs_convert_reads(rd.seq, rd.off, rd.mate)
    sm, m, nh = mb.mb_seed_batch(G, rd.seq, rd.off, mate=rd.mate, opts=o)
    hits, _ = mb.mb_locate(G, sm, m, opts=o, cap=nh)
    compare_seed(sm, hits, X, conv, rd.off)
    keep = mb.mb_bs_filter(G, sm, m, rd.mate, hits, nh)
    osm, over, hoff, ohits = X.seed(conv, rd.off)
    cnt = np.where(over, 0, osm["s"]).astype(np.int64)
    qlen = np.repeat((osm["qend"] - osm["qbeg"]).astype(np.int64), cnt)
    rmate = np.repeat(rd.mate[osm["read"].astype(np.int64)], cnt)
    assert np.array_equal(keep.astype(bool), oracle.bs_keep(ohits, qlen, rmate, len(ref)))


def test_max_occ_boundary_planted(mb):
    """Units planted exactly 500, 501 and 3 times: the default cap keeps s = 500 (located) and
    flags s = 501 (no hits), on the GPU as in the oracle and by construction."""
    ref, units, starts = synth.planted_copies(40, [500, 501, 3], 60, 0x6D6201)
    G = mb.mb_index_build(ref)
    X = oracle.Index(ref)
    seq = units.reshape(-1)
    off = np.arange(len(units) + 1, dtype=np.uint64) * 40
    for max_occ in (500, 499, 501):
        o = dict(max_occ=max_occ)
        sm, m, nh = mb.mb_seed_batch(G, seq, off, opts=o)
        hits, _ = mb.mb_locate(G, sm, m, opts=o, cap=nh)
        compare_seed(sm, hits, X, seq, off, max_occ=max_occ)
        assert sm["s"].tolist() == [500, 501, 3]
        assert (sm["flags"] & 1).tolist() == [int(500 > max_occ), int(501 > max_occ), 0]
    sm, m, nh = mb.mb_seed_batch(G, seq, off)
    hits, _ = mb.mb_locate(G, sm, m, cap=nh)
    assert np.array_equal(np.sort(hits[:500]).astype(np.uint64), starts[0])
    assert np.array_equal(np.sort(hits[500:503]).astype(np.uint64), starts[2])


def test_bisulfite_filter_drops_hit_spanning_two_copies(mb):
    """A read-1 read planted across the C-to-T and G-to-A copies of the 3-base text: its one hit
    spans both copies and the strand filter drops it; a control read inside the C-to-T copy is
    kept (Section 2.9)."""
    m, half = 5000, 20
    ref, cross = synth.junction_read(m, half, 0x6D6202)
    seq = np.concatenate([cross, ref[1000:1000 + 2 * half]]).astype(np.uint8)
    off = np.array([0, 2 * half, 4 * half], dtype=np.uint64)
    mate = np.array([1, 1], dtype=np.uint8)
    o = dict(flags=mb.MB_BS3)
    G = mb.mb_index_build(ref, opts=o)
    sm, n_sm, nh = mb.mb_seed_batch(G, seq, off, mate=mate, opts=o)
    hits, _ = mb.mb_locate(G, sm, n_sm, opts=o, cap=nh)
    assert sm["s"].tolist() == [1, 1]
    assert hits.tolist() == [m - half, 1000]
    keep = mb.mb_bs_filter(G, sm, n_sm, mate, hits, nh)
    assert keep.tolist() == [0, 1]


def test_bisulfite_split(mb):
    """Section 2.9 T-to-C split on the GPU against the oracle: reads with 1-3% substitutions so
    that read C over reference T (read 1) and read G over reference A (read 2) occur; with the
    strand filter's keep flags and with every hit, host and device buffers."""
    ref = synth.reference(60_000, 73)
    rd = synth.reads(ref, 800, 74, mode=1, read_len=150, bisulfite=True, sub_lo=0.01, sub_hi=0.03)
    o = dict(flags=mb.MB_BS3)
    G = mb.mb_index_build(ref, opts=o)
    sm, m, nh = mb.mb_seed_batch(G, rd.seq, rd.off, mate=rd.mate, opts=o)
    hits, _ = mb.mb_locate(G, sm, m, opts=o, cap=nh)
    keep = mb.mb_bs_filter(G, sm, m, rd.mate, hits, nh)
    for kp in (keep, None):
        got = mb.mb_bs_split(G, ref, rd.seq, rd.off, rd.mate, sm, m, hits, nh, keep=kp)
        want = oracle.bs_split(ref, rd.seq, rd.off, rd.mate, sm, hits, kp)
        owner = np.repeat(np.arange(m), np.where(sm["flags"] & 1, 0, sm["s"]).astype(np.int64))
        assert len(want) > 0 and np.any(want["qbeg"] != sm["qbeg"][owner[want["hit"].astype(np.int64)]])
        assert got.tobytes() == want.astype(mb.PIECE_DTYPE).tobytes()
    dgot = mb.mb_bs_split(G, dev(ref), dev(rd.seq), dev(rd.off), dev(rd.mate), dev(sm.view(np.uint8)), m,
                          dev(hits), nh, keep=dev(keep))
    assert dgot.tobytes() == mb.mb_bs_split(G, ref, rd.seq, rd.off, rd.mate, sm, m, hits, nh, keep=keep).tobytes()
    # a plain index is refused
    P = mb.mb_index_build(ref)
    with pytest.raises(mb.MbError):
        mb.mb_bs_split(P, ref, rd.seq, rd.off, rd.mate, sm, m, hits, nh, keep=keep)


def test_save_load_roundtrip_and_corruption(mb, tmp_path):
    ref, rd, p = synth.workload(1, scale=0.02)
    G = mb.mb_index_build(ref)
    path = str(tmp_path / "i.mbi")
    G.save(path)
    H = mb.mb_index_load(path)
    a = mb.seed(G, rd.seq, rd.off)
    b = mb.seed(H, rd.seq, rd.off)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert all(np.array_equal(x, y) for x, y in zip(G.export_aux(), H.export_aux()))
    # an index without the auxiliary arrays round-trips too
    N = mb.mb_index_build(ref, opts=dict(flags=mb.MB_NO_AUX))
    N.save(str(tmp_path / "n.mbi"))
    c = mb.seed(mb.mb_index_load(str(tmp_path / "n.mbi")), rd.seq, rd.off)
    assert np.array_equal(a[0], c[0]) and np.array_equal(a[1], c[1])
    raw = bytearray(open(path, "rb").read())
    raw[200] ^= 0xFF
    bad = str(tmp_path / "bad.mbi")
    open(bad, "wb").write(bytes(raw))
    with pytest.raises(mb.MbError) as ei:
        mb.mb_index_load(bad)
    assert ei.value.code == -7
    open(bad, "wb").write(bytes(raw[:100]))
    with pytest.raises(mb.MbError) as ei:
        mb.mb_index_load(bad)
    assert ei.value.code == -7
