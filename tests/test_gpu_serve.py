"""Served form: requests of mixed sizes (short pairs and long reads) submitted together are
merged into launch groups that run concurrently; every request's records and hits must be
exactly those of the plain entry points on that request alone."""
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
    return ref, G


def test_each_request_same_alone_and_in_the_mix(mb, served):
    ref, G = served
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


def test_requests_arriving_while_others_run(mb, served):
    ref, G = served
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
    srv.close()


def test_oversize_request_rejected_and_timeout(mb, served):
    ref, G = served
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
