"""Served form: requests of mixed sizes (short pairs and long reads) submitted together are
merged into launch groups that run concurrently; every request's records and hits must be
exactly those of the plain entry points on that request alone, and those of the CPU oracle."""
import os

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


def requests(ref, n, seed):
    rng = np.random.default_rng(seed)
    out = []
    for q in range(n):
        if rng.random() < 0.8:   # short: 1-512 pairs of 2x150
            pairs = int(np.exp(rng.uniform(0, np.log(512))))
            rd = synth.reads(ref, 2 * pairs, seed * 1000 + q, mode=1, read_len=150, sub_lo=0.001,
                             sub_hi=0.01, indel=0.0001)
        else:                     # long: 1-64 single reads of 1-10 kb
            k = int(np.exp(rng.uniform(0, np.log(64))))
            rd = synth.reads(ref, k, seed * 1000 + q, mode=2, len_lo=1000, len_hi=10000, sub_lo=0.001,
                             indel=0.0002)
        out.append(rd)
    return out


@pytest.fixture(scope="module")
def served(mb):
    ref = synth.repeat_rich_reference(2_000_000, 91, 0.3)
    G = mb.mb_index_build(ref)
    X = oracle.Index(ref)
    return ref, G, X


def same_as_oracle(X, r, sm, hits, frac=1.0, seed=0):
    """The served records and hits of request r equal the oracle's on r alone (every field of
    every record, every hit); with frac < 1 only a seeded sample of the request's reads."""
    pick = np.arange(r.n)
    if frac < 1.0:
        pick = np.sort(np.random.default_rng(seed).choice(r.n, max(1, int(r.n * frac)), replace=False))
    sub = r.subset(pick)
    osm, over, hoff, ohits = X.seed(sub.seq, sub.off)
    keep = np.isin(sm["read"].astype(np.int64), pick)
    g = sm[keep]
    assert len(g) == len(osm)
    assert np.array_equal(g["read"].astype(np.int64), pick[osm["read"].astype(np.int64)])
    for f in ("qbeg", "qend", "k", "kr", "s"):
        assert np.array_equal(g[f].astype(np.uint64), osm[f]), f
    assert np.array_equal((g["flags"] & 1).astype(bool), over)
    cnt = np.where(g["flags"] & 1, 0, g["s"]).astype(np.int64)
    gh = np.concatenate([hits[int(a):int(a) + int(c)] for a, c in zip(g["hit_off"], cnt)]) if len(g) else \
        np.zeros(0, np.uint32)
    assert np.array_equal(gh.astype(np.uint64), ohits)
    if frac >= 1.0:
        assert np.array_equal(sm["hit_off"], hoff)


def test_each_request_same_alone_and_in_the_mix(mb, served):
    ref, G, X = served
    reqs = requests(ref, 60, 5)
    srv = mb.Server(G, hbm_budget=2 << 30)
    tickets = [srv.submit(r.seq, r.off) for r in reqs]
    results = [srv.wait(t) for t in tickets]
    st = srv.stats()
    srv.close()
    assert st["slots"] >= 1 and st["groups"] >= 1
    assert st["merged"] > 0                      # requests did share launch groups
    for r, (sm, hits, lat) in zip(reqs, results):
        want_sm, want_hits = mb.seed(G, r.seq, r.off)
        assert sm.tobytes() == want_sm.tobytes()
        assert np.array_equal(hits, want_hits)
        assert lat > 0
        same_as_oracle(X, r, sm, hits)


def test_requests_arriving_while_others_run(mb, served):
    ref, G, X = served
    reqs = requests(ref, 30, 6)
    srv = mb.Server(G, hbm_budget=1 << 30)
    got = {}
    for i, r in enumerate(reqs):
        t = srv.submit(r.seq, r.off)
        got[t] = r
        if i % 3 == 2:                           # collect some results while submitting
            for tt in list(got):
                if srv.poll(tt):
                    sm, hits, _ = srv.wait(tt)
                    want_sm, want_hits = mb.seed(G, got[tt].seq, got[tt].off)
                    assert sm.tobytes() == want_sm.tobytes() and np.array_equal(hits, want_hits)
                    del got[tt]
    for tt, r in got.items():
        sm, hits, _ = srv.wait(tt)
        want_sm, want_hits = mb.seed(G, r.seq, r.off)
        assert sm.tobytes() == want_sm.tobytes() and np.array_equal(hits, want_hits)
        same_as_oracle(X, r, sm, hits)
    srv.close()


def test_oversize_request_rejected_and_timeout(mb, served):
    ref, G, X = served
    srv = mb.Server(G, hbm_budget=1 << 30)
    big_off = np.arange(0, 70000 * 10 + 1, 10, dtype=np.uint64)   # 70,000 reads > one slot
    with pytest.raises(mb.MbError) as ei:
        srv.submit(np.zeros(int(big_off[-1]), np.uint8), big_off)
    assert ei.value.code == -1
    with pytest.raises(mb.MbError):
        srv.poll(123456789)                      # unknown ticket
    r = requests(ref, 1, 7)[0]
    t = srv.submit(r.seq, r.off)
    try:
        srv.wait(t, timeout_ms=1, release=False)
    except mb.MbError as e:
        assert e.code == -5                      # MB_ERR_TIMEOUT, then it still completes
    sm, hits, _ = srv.wait(t)
    want_sm, want_hits = mb.seed(G, r.seq, r.off)
    assert sm.tobytes() == want_sm.tobytes() and np.array_equal(hits, want_hits)
    srv.close()


def config5_requests(ref, n, seed):
    """Requests shaped like the served workload: 80% short (log-uniform 1-4,096 pairs of 2x150),
    20% long (log-uniform 1-4,096 single reads of log-uniform 1-10 kb)."""
    rng = np.random.default_rng(seed)
    out = []
    for q in range(n):
        k = int(np.exp(rng.uniform(0, np.log(4096))))
        if rng.random() < 0.8:
            rd = synth.reads(ref, 2 * k, seed * 7919 + q, mode=1, read_len=150, sub_lo=0.001, sub_hi=0.01,
                             indel=0.0001)
        else:
            rd = synth.reads(ref, k, seed * 7919 + q, mode=2, len_lo=1000, len_hi=10000, sub_lo=0.001,
                             indel=0.0002)
        out.append(rd)
    return out


@pytest.mark.slow
def test_served_mix_on_100mbp_index_against_oracle(mb):
    """An index far above L2 (the 100 Mbp repeat-rich reference) serving a stream of requests of
    the served workload's shape, all submitted at once: every request equals the plain entry
    points on it alone, and a seeded 5% of each request's reads equal the oracle."""
    ref, _, _ = synth.workload(2)
    G = mb.mb_index_build(ref)
    G.drop_sa()
    reqs = config5_requests(ref, 120, 0x6D69)
    srv = mb.Server(G, hbm_budget=16 << 30)
    tickets = [srv.submit(r.seq, r.off) for r in reqs]
    results = [srv.wait(t) for t in tickets]
    st = srv.stats()
    c = srv.counters()
    srv.close()
    assert st["merged"] > 0
    # requests with reads of 1 kb or more ran in groups of their own
    n_long = sum(1 for r in reqs if (np.diff(r.off.astype(np.int64)) >= 1000).any())
    assert n_long > 0 and 0 < c["long_groups"] <= n_long < len(reqs)
    assert c["groups"] > c["long_groups"]
    X = oracle.Index(ref, threads=os.cpu_count())
    for q, (r, (sm, hits, _)) in enumerate(zip(reqs, results)):
        want_sm, want_hits = mb.seed(G, r.seq, r.off)
        assert sm.tobytes() == want_sm.tobytes(), q
        assert np.array_equal(hits, want_hits), q
        same_as_oracle(X, r, sm, hits, frac=0.05, seed=q)


def test_admission_waits_for_free_device_memory(mb, served):
    """Admission by free device memory: with the free memory admission sees held at 0 no slot can
    be made and a submitted request waits; once the real value is back it is served, with the
    same results as alone."""
    ref, G, X = served
    srv = mb.Server(G, hbm_budget=1 << 30)
    srv.inject(free_bytes=0)
    r = requests(ref, 1, 11)[0]
    t = srv.submit(r.seq, r.off)
    import time
    time.sleep(0.3)
    assert not srv.poll(t)
    c = srv.counters()
    assert c["slots"] == 0 and c["slots_created"] == 0
    srv.inject(free_bytes=-1)
    sm, hits, lat = srv.wait(t)
    assert lat >= 300
    want_sm, want_hits = mb.seed(G, r.seq, r.off)
    assert sm.tobytes() == want_sm.tobytes() and np.array_equal(hits, want_hits)
    c = srv.counters()
    assert c["slots_created"] >= 1 and c["memory_wait_ms"] >= 250
    srv.close()


def test_slot_allocation_failure_is_retried(mb, served):
    """Two slot creations fail (injected as allocation failures): admission retries, the third
    succeeds and the request is served correctly."""
    ref, G, X = served
    srv = mb.Server(G, hbm_budget=1 << 30)
    srv.inject(free_bytes=-1, fail_slots=2)
    r = requests(ref, 1, 12)[0]
    sm, hits, _ = srv.wait(srv.submit(r.seq, r.off))
    c = srv.counters()
    assert c["alloc_failures"] == 2 and c["slots_created"] >= 1
    want_sm, want_hits = mb.seed(G, r.seq, r.off)
    assert sm.tobytes() == want_sm.tobytes() and np.array_equal(hits, want_hits)
    srv.close()


def test_calls_after_destroy_are_refused(mb, served):
    """Submit, poll, stats and destroy on a destroyed server return MB_ERR_ARG (no use after free)."""
    import ctypes
    ref, G, X = served
    srv = mb.Server(G, hbm_budget=1 << 30)
    h = srv._h
    srv.close()
    L = mb.lib()
    r = requests(ref, 1, 13)[0]
    t = ctypes.c_uint64()
    seq = np.ascontiguousarray(r.seq)
    off = np.ascontiguousarray(r.off, dtype=np.uint64)
    assert L.mb_serve_submit(h, ctypes.c_void_p(seq.ctypes.data), ctypes.c_void_p(off.ctypes.data), r.n,
                             ctypes.byref(t)) == -1
    d = ctypes.c_int()
    assert L.mb_serve_poll(h, 1, ctypes.byref(d)) == -1
    assert L.mb_serve_destroy(h) == -1


def test_group_outgrowing_its_plan_goes_to_the_helper(mb):
    """Requests of 60,000 random reads seeded with min_len 5 against a 200 kbp reference: each read
    has dozens of SMEMs, so a request yields more records than a slot's 2M; its group is seeded
    again on the helper thread and every request still equals the plain entry points."""
    ref = synth.reference(200_000, 81)
    G = mb.mb_index_build(ref)
    o = dict(min_len=5, max_occ=500)
    srv = mb.Server(G, hbm_budget=2 << 30, opts=o)
    reqs = []
    for q in range(2):
        reads = synth.reference(150 * 60_000, 8300 + q)
        off = np.arange(60_001, dtype=np.uint64) * 150
        reqs.append((reads, off))
    tickets = [srv.submit(s_, o_) for s_, o_ in reqs]
    got = [srv.wait(t) for t in tickets]
    c = srv.counters()
    srv.close()
    assert c["outgrown_groups"] >= 1
    for (s_, o_), (sm, hits, _) in zip(reqs, got):
        want_sm, want_hits = mb.seed(G, s_, o_, opts=o)
        assert sm.tobytes() == want_sm.tobytes()
        assert np.array_equal(hits, want_hits)
