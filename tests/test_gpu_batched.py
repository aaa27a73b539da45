"""Batched form: mixed-length reads (100 bp - 10 kb) seeded by one persistent launch with a
device work queue, captured in a CUDA graph, in every launch shape the autotuner tries.
Every form must give the records and hits of the plain entry points, bit for bit."""
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


@pytest.fixture(scope="module")
def mixed(mb):
    ref, rd, params = synth.workload(4, scale=0.01)     # 1 Mbp repeat-rich, 2,000 reads of 100 bp-10 kb
    G = mb.mb_index_build(dev(ref))
    sm, hits = mb.seed(G, rd.seq, rd.off)
    return ref, rd, G, sm, hits


def test_plain_matches_oracle(mb, mixed):
    ref, rd, G, sm, hits = mixed
    X = oracle.Index(ref)
    osm, over, hoff, ohits = X.seed(rd.seq, rd.off)
    for f in ("read", "qbeg", "qend", "k", "kr", "s"):
        assert np.array_equal(sm[f].astype(np.uint64), osm[f])
    assert np.array_equal(hits.astype(np.uint64), ohits)


@pytest.mark.parametrize("depth", [1, 2, 4, 8, 16])
@pytest.mark.parametrize("queue", [False, True])
@pytest.mark.parametrize("block", [128, 256, 512])
def test_plan_every_launch_shape(mb, mixed, queue, block, depth):
    ref, rd, G, sm, hits = mixed
    o = dict(flags=mb.MB_BATCHED if queue else 0, block_size=block, prefetch_depth=depth)
    P = mb.Plan(G, rd.n, len(rd.seq), len(sm) + 10, len(hits) + 10, opts=o)
    P.run(dev(rd.seq), dev(rd.off))
    psm, phits = P.result()
    assert psm.tobytes() == sm.tobytes()
    assert np.array_equal(phits, hits)


@pytest.mark.parametrize("form", [dict(flags=0x80), dict(smem_burst=1, smem_wait=1), dict(smem_burst=2, smem_wait=32),
                                  dict(smem_burst=16, smem_wait=4), dict(smem_burst=64, smem_wait=16),
                                  dict(smem_reads_per_warp=1), dict(smem_reads_per_warp=5),
                                  dict(smem_reads_per_warp=16, smem_burst=4, smem_wait=2)])
@pytest.mark.parametrize("queue", [False, True])
def test_plan_every_smem_form(mb, mixed, queue, form):
    """The SMEM kernel's one-loop form and its split form at several service schedules and reads
    per warp give the same records and hits."""
    ref, rd, G, sm, hits = mixed
    o = dict(form, flags=form.get("flags", 0) | (mb.MB_BATCHED if queue else 0), block_size=512, prefetch_depth=8)
    P = mb.Plan(G, rd.n, len(rd.seq), len(sm) + 10, len(hits) + 10, opts=o)
    P.run(dev(rd.seq), dev(rd.off))
    psm, phits = P.result()
    assert psm.tobytes() == sm.tobytes()
    assert np.array_equal(phits, hits)


def test_graph_replay_on_new_batches(mb, mixed):
    ref, rd, G, sm, hits = mixed
    seq, off = dev(rd.seq), dev(rd.off)
    P = mb.Plan(G, rd.n, len(rd.seq), 4 * len(sm) + 64, 4 * len(hits) + 64, opts=dict(flags=mb.MB_BATCHED))
    P.capture(seq, off)
    for rep, seed in enumerate((0, 77, 78)):
        if seed:   # a new batch of the same shape written into the same device buffers
            other = synth.reads(ref, rd.n, seed, mode=2, len_lo=100, len_hi=10000, sub_lo=0.001,
                                indel=0.0002)
            n_keep = min(len(other.seq), len(rd.seq))
            lens = np.diff(other.off.astype(np.int64))
            cum = np.cumsum(lens)
            k = int(np.searchsorted(cum, n_keep, side="right"))
            o2 = np.concatenate([other.off[:k + 1], np.full(rd.n - k, other.off[k])]).astype(np.uint64)
            s2 = np.zeros(len(rd.seq), np.uint8)
            s2[:int(o2[-1])] = other.seq[:int(o2[-1])]
            seq.copy_(torch.from_numpy(s2).cuda())
            off.copy_(torch.from_numpy(o2.view(np.int64)).cuda())
            want_sm, want_hits = mb.seed(G, s2, o2)
        else:
            want_sm, want_hits = sm, hits
        P.replay()
        got_sm, got_hits = P.result()
        assert got_sm.tobytes() == want_sm.tobytes(), rep
        assert np.array_equal(got_hits, want_hits), rep


def test_plan_capacity_reports_needed_counts(mb, mixed):
    ref, rd, G, sm, hits = mixed
    P = mb.Plan(G, rd.n, len(rd.seq), max(1, len(sm) // 2), len(hits) + 10)
    P.run(dev(rd.seq), dev(rd.off))
    with pytest.raises(mb.MbError) as ei:
        P.result()
    assert ei.value.code == -3


def test_batched_equals_plain_per_length_bucket(mb, mixed):
    """The comparison the batched form is measured against: one plain launch per length bucket
    ([100,200), [200,400), ... 10 kb), results put back in read order."""
    ref, rd, G, sm, hits = mixed
    lens = np.diff(rd.off.astype(np.int64))
    edges = [100 * 2 ** i for i in range(8)] + [10001]
    recs, hit_lists = [], []
    for lo, hi in zip(edges[:-1], edges[1:]):
        ids = np.nonzero((lens >= lo) & (lens < hi))[0]
        if len(ids) == 0:
            continue
        sub = rd.subset(ids)
        bsm, bh = mb.seed(G, sub.seq, sub.off)
        cnt = np.where(bsm["flags"] & 1, 0, bsm["s"]).astype(np.int64)
        for x, c, h0 in zip(bsm, cnt, bsm["hit_off"].astype(np.int64)):
            recs.append((int(ids[x["read"]]), int(x["qbeg"]), int(x["qend"]), int(x["k"]), int(x["kr"]),
                         int(x["s"])))
            hit_lists.append(bh[h0:h0 + c])
    order = sorted(range(len(recs)), key=lambda i: (recs[i][0], recs[i][1]))
    want = [tuple(int(v) for v in (x["read"], x["qbeg"], x["qend"], x["k"], x["kr"], x["s"])) for x in sm]
    assert [recs[i] for i in order] == want
    got_hits = np.concatenate([hit_lists[i] for i in order]) if order else np.zeros(0, np.uint32)
    assert np.array_equal(got_hits, hits)


def test_autotune_picks_a_supported_shape(mb, mixed):
    ref, rd, G, sm, hits = mixed
    best, ms, grid = mb.autotune(G, dev(rd.seq), dev(rd.off), points=True)
    assert best.block_size in (128, 256, 512)
    assert ms > 0
    assert len(grid) in (87, 92) and min(t for _, t in grid) == ms
    shapes = {tuple(sorted(mb.shape_of(o).items())) for o, _ in grid}
    assert len(shapes) == len(grid)              # every point a distinct launch shape
    P = mb.Plan(G, rd.n, len(rd.seq), len(sm) + 1, len(hits) + 1, opts=best)
    P.run(dev(rd.seq), dev(rd.off))
    psm, phits = P.result()
    assert psm.tobytes() == sm.tobytes() and np.array_equal(phits, hits)
