"""Parity at full workload sizes.

The GPU builds the whole index and seeds the whole read batch; the CPU oracle builds its own
index by sorting suffixes and checks the full suffix array, the block counts, the k-mer table,
and a seeded random sample of the reads (every SMEM record and every hit of each sampled read).

- The 1 Gbp workload runs twice: with the binding's defaults (10-mer table, fixed read ranges
  per warp, one locate walk per lane; one mb_seed_batch + one mb_locate call), and in exactly
  the launch configuration bench.py times (14-mer table, device work queue, 512 threads per
  block, locate walks that join, 2 per lane) through all three forms the bench runs: the plain calls, the
  captured CUDA graph of a plan, and mb_seed_locate on pinned host buffers.  The three must be
  identical byte for byte, and 1% of the reads must match the oracle.
- The mixed-length workload (100 Mbp, 200,000 reads of 100 bp - 10 kb) runs in the batched
  form bench.py times (autotuned plan, replayed graph) and in the work-queue shape; 5% of its
  reads are checked against the oracle.
Minutes per test: marked slow as well as gpu.
"""
import os

import numpy as np
import pytest

import oracle
import synth

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

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


def gpu_seed_all(mb, G, rd, opts=None):
    seq, off = dev(rd.seq), dev(rd.off)
    cap = 4 * rd.n
    out = torch.empty(cap * 48, dtype=torch.uint8, device="cuda")
    _, m, nh = mb.mb_seed_batch(G, seq, off, opts=opts, out=out, cap=cap)
    hits = torch.empty(max(nh, 1), dtype=torch.int32, device="cuda")
    mb.mb_locate(G, out, m, opts=opts, hits=hits, cap=nh)
    sm = out[:m * 48].cpu().numpy().view(mb.SMEM_DTYPE)
    h = hits[:nh].cpu().numpy().view(np.uint32)
    return sm, h


def check_index(G, X, k=10, sample_kmers=None):
    e = G.export(sa=True, ssa=True, occ=True, kmer=True, kmer_k=k)
    assert G.n == X.n and G.primary == X.primary
    osa = X.sa()
    assert np.array_equal(e["sa"], osa)
    del osa
    assert np.array_equal(e["ssa"], X.ssa())
    assert np.array_equal(e["C"], X.C)
    B = X.bwt()
    occ = e["occ"].view(np.uint32).reshape(-1, 8)
    for a in range(4):
        blk = np.add.reduceat((B == a + 1).view(np.uint8), np.arange(0, len(B), 64), dtype=np.uint64)
        cum = np.concatenate([[0], np.cumsum(blk)]).astype(np.uint64)[:len(occ)]
        assert np.array_equal(occ[:, a].astype(np.uint64), cum), a
    del B
    nk = 4 ** k
    words = np.arange(nk, dtype=np.int64)
    if sample_kmers:
        words = np.sort(np.random.default_rng(7).choice(nk, sample_kmers, replace=False))
    pats = np.stack([(words >> (2 * t)) & 3 for t in range(k)], axis=1).astype(np.uint8)   # base t in bits 2t
    want = X.ds_intervals(pats).astype(np.uint32)
    got = e["kmer"].reshape(nk, 3)[words]
    assert np.array_equal(got, want)


def check_sampled_reads(sm, hits, X, rd, frac, seed, params):
    rng = np.random.default_rng(seed)
    pick = np.sort(rng.choice(rd.n, max(1, int(rd.n * frac)), replace=False))
    sub = rd.subset(pick)
    osm, over, hoff, ohits = X.seed(sub.seq, sub.off, params["min_len"], params["min_occ"],
                                    params["max_occ"])
    reads = sm["read"].astype(np.int64)
    lo = np.searchsorted(reads, pick, side="left")
    hi = np.searchsorted(reads, pick, side="right")
    o_lo = np.searchsorted(osm["read"].astype(np.int64), np.arange(len(pick)), side="left")
    o_hi = np.searchsorted(osm["read"].astype(np.int64), np.arange(len(pick)), side="right")
    assert np.array_equal(hi - lo, o_hi - o_lo)
    g_idx = np.concatenate([np.arange(a, b) for a, b in zip(lo, hi)]) if len(pick) else np.zeros(0, int)
    g = sm[g_idx]
    for f in ("qbeg", "qend", "k", "kr", "s"):
        assert np.array_equal(g[f].astype(np.uint64), osm[f]), f
    assert np.array_equal(pick[osm["read"].astype(np.int64)], g["read"].astype(np.int64))
    assert np.array_equal((g["flags"] & 1).astype(bool), over)
    # hits of the sampled reads, in record order then SA-row order
    cnt = np.where(g["flags"] & 1, 0, g["s"]).astype(np.int64)
    starts = g["hit_off"].astype(np.int64)
    gh = np.concatenate([hits[s:s + c] for s, c in zip(starts, cnt)]) if len(g) else np.zeros(0)
    assert np.array_equal(gh.astype(np.uint64), ohits)
    return len(pick), len(g), len(gh)


@pytest.fixture(scope="module")
def w3(mb):
    """The 1 Gbp workload and the oracle's index of it (built once for both 1 Gbp tests)."""
    ref, rd, params = synth.workload(3)
    X = oracle.Index(ref, threads=os.cpu_count())
    yield ref, rd, params, X
    del X


def test_workload3_1gbp_full_index_and_sampled_reads(mb, w3):
    """1 Gbp repeat-rich reference, 10M pairs: full SA / blocks / k-mer sample and 1% of reads."""
    ref, rd, params, X = w3
    G = mb.mb_index_build(dev(ref))
    check_index(G, X, sample_kmers=200_000)
    G.drop_sa()
    sm, hits = gpu_seed_all(mb, G, rd)
    n, m, h = check_sampled_reads(sm, hits, X, rd, 0.01, 0x6D62, params)
    print(f"checked {n} reads, {m} SMEMs, {h} hits")
    G.free()
    torch.cuda.empty_cache()


# the launch configuration bench.py times on the 1 Gbp workload
BENCH_KMER_K = 14
BENCH_OPTS = dict(block_size=512, prefetch_depth=2)


def test_workload3_1gbp_in_the_bench_configuration(mb, w3):
    """The bench's exact configuration: 14-mer table, work queue, block 512, 2 walks per lane
    that join; plain calls == captured plan graph == mb_seed_locate on pinned host buffers, and
    1% of the reads against the oracle."""
    ref, rd, params, X = w3
    G = mb.mb_index_build(dev(ref), opts=dict(kmer_k=BENCH_KMER_K))
    words = np.sort(np.random.default_rng(0x6D67).choice(4 ** BENCH_KMER_K, 50_000, replace=False))
    pats = np.stack([(words >> (2 * t)) & 3 for t in range(BENCH_KMER_K)], axis=1).astype(np.uint8)
    assert np.array_equal(G.kmer_get(words), X.ds_intervals(pats).astype(np.uint32))
    G.drop_sa()
    opts = dict(BENCH_OPTS, flags=mb.MB_BATCHED | mb.MB_LOCATE_JOIN)
    seq, off = dev(rd.seq), dev(rd.off)
    # plain calls in the bench's launch shape
    cap = 4 * rd.n
    out = torch.empty(cap * 48, dtype=torch.uint8, device="cuda")
    _, m, nh = mb.mb_seed_batch(G, seq, off, opts=opts, out=out, cap=cap)
    hits = torch.empty(max(nh, 1), dtype=torch.int32, device="cuda")
    mb.mb_locate(G, out, m, opts=opts, hits=hits, cap=nh)
    plain_sm = out[:m * 48].cpu().numpy()
    plain_h = hits[:nh].cpu().numpy().view(np.uint32)
    del out, hits
    # the captured CUDA graph of a plan, replayed twice
    P = mb.Plan(G, rd.n, len(rd.seq), m + 1024, nh + 1024, opts=opts)
    P.capture(seq, off)
    P.replay()
    P.replay()
    gsm, gh = P.result()
    P.free()
    assert gsm.tobytes() == plain_sm.tobytes()
    assert np.array_equal(gh, plain_h)
    del plain_sm, plain_h, seq, off
    torch.cuda.empty_cache()
    # end to end through mb_seed_locate on pinned host buffers
    seq_h = torch.from_numpy(rd.seq).pin_memory()
    off_h = torch.from_numpy(rd.off.view(np.int64)).pin_memory()
    out_h = torch.empty(m * 48, dtype=torch.uint8).pin_memory()
    hits_h = torch.empty(max(nh, 1), dtype=torch.int32).pin_memory()
    m2, nh2 = mb.seed_locate(G, seq_h, off_h, opts=opts, out=out_h, cap=m, hits=hits_h, hits_cap=nh)
    assert (m2, nh2) == (m, nh)
    assert out_h.numpy().tobytes() == gsm.tobytes()
    assert np.array_equal(hits_h[:nh].numpy().view(np.uint32), gh)
    del out_h, hits_h, seq_h, off_h
    n, ms, h = check_sampled_reads(gsm, gh, X, rd, 0.01, 0x6D66, params)
    print(f"bench configuration: {m} SMEMs, {nh} hits; checked {n} reads, {ms} SMEMs, {h} hits")
    G.free()
    torch.cuda.empty_cache()


def test_workload4_full_size_batched_form_sampled_reads(mb):
    """Mixed lengths at full size (100 Mbp, 200,000 reads of 100 bp - 10 kb): the autotuned plan
    as a replayed graph and the work-queue shape give the same output, and 5% of the reads match
    the oracle."""
    ref, rd, params = synth.workload(4)
    G = mb.mb_index_build(dev(ref))
    G.drop_sa()
    seq, off = dev(rd.seq), dev(rd.off)
    sm, m, nh = mb.mb_seed_batch(G, seq, off, cap=4 * rd.n)
    best, _ = mb.autotune(G, seq, off)
    outs = []
    for o in (best, mb.Opts(flags=mb.MB_BATCHED, block_size=512, prefetch_depth=16)):
        P = mb.Plan(G, rd.n, len(rd.seq), m + 64, nh + 64, opts=o)
        P.capture(seq, off)
        P.replay()
        outs.append(P.result())
        P.free()
    (a_sm, a_h), (b_sm, b_h) = outs
    assert a_sm.tobytes() == b_sm.tobytes() and np.array_equal(a_h, b_h)
    assert a_sm.tobytes() == sm.tobytes()
    X = oracle.Index(ref, threads=os.cpu_count())
    n, ms, h = check_sampled_reads(a_sm, a_h, X, rd, 0.05, 0x6D68, params)
    print(f"mixed lengths: checked {n} reads, {ms} SMEMs, {h} hits")
    G.free()
    torch.cuda.empty_cache()


def test_workload2_100mbp_full_index_and_sampled_reads(mb):
    """100 Mbp repeat-rich reference, 1M pairs: full index and 10% of reads."""
    ref, rd, params = synth.workload(2)
    G = mb.mb_index_build(dev(ref))
    X = oracle.Index(ref, threads=os.cpu_count())
    check_index(G, X)
    G.drop_sa()
    sm, hits = gpu_seed_all(mb, G, rd)
    check_sampled_reads(sm, hits, X, rd, 0.10, 0x6D63, params)


def test_workload3_bisulfite_1gbp_three_base_index(mb):
    """Directional bisulfite set: 3-base index over CT(R).GA(R) of the 1 Gbp reference
    (n = 4e9 + 1), reads converted on the GPU (read 1 C->T, read 2 G->A), the strand filter of
    Section 2.9; full suffix array, k-mer sample and 1% of the reads against the oracle."""
    from synth import Reads
    ref, rd, params = synth.workload(3, bisulfite=True)
    o = dict(flags=mb.MB_BS3)
    G = mb.mb_index_build(dev(ref), opts=o)
    assert G.n == 4 * len(ref) + 1
    X = oracle.Index(ref, bs3=True, threads=os.cpu_count())
    check_index(G, X, sample_kmers=100_000)
    G.drop_sa()
    seq, off, mate = dev(rd.seq), dev(rd.off), dev(rd.mate)
    # three-letter reads give many SMEMs per read: let the binding size the output
    sm, m, nh = mb.mb_seed_batch(G, seq, off, mate=mate, opts=o, cap=4 * rd.n)
    h, _ = mb.mb_locate(G, sm, m, opts=o, cap=nh)
    kp = mb.mb_bs_filter(G, sm, m, rd.mate, h, nh)
    conv = Reads(oracle.bs_convert_reads(rd.seq, rd.off, rd.mate), rd.off, rd.origin, rd.mate)
    check_sampled_reads(sm, h, X, conv, 0.01, 0x6D64, params)
    # strand filter recomputed from the positions (Section 2.9)
    cnt = np.where(sm["flags"] & 1, 0, sm["s"]).astype(np.int64)
    qlen = np.repeat((sm["qend"] - sm["qbeg"]).astype(np.int64), cnt)
    rmate = np.repeat(rd.mate[sm["read"].astype(np.int64)], cnt)
    assert np.array_equal(kp.astype(bool), oracle.bs_keep(h, qlen, rmate, len(ref)))
    assert kp.sum() > 0
    # T-to-C split of every kept hit (Section 2.9), checked against the oracle on the hits of 1% of
    # the reads
    pc = mb.mb_bs_split(G, ref, rd.seq, rd.off, rd.mate, sm, m, h, nh, keep=kp)
    pick = np.random.default_rng(0x6D65).choice(rd.n, rd.n // 100, replace=False)
    msel = np.nonzero(np.isin(sm["read"].astype(np.int64), pick))[0]
    hoff = sm["hit_off"].astype(np.int64)
    hsel = np.concatenate([np.arange(hoff[q], hoff[q] + cnt[q]) for q in msel]).astype(np.int64)
    want = oracle.bs_split(ref, rd.seq, rd.off, rd.mate, sm[msel], h[hsel], kp[hsel])
    want["hit"] = hsel[want["hit"].astype(np.int64)]
    got = pc[np.isin(pc["hit"].astype(np.int64), hsel)]
    assert len(want) > 0
    assert got.tobytes() == want.astype(mb.PIECE_DTYPE).tobytes()
