"""The CPU comparator (the paper's CPU design: Algorithm 3 with one queue and prefetching, 64-byte
blocks, 10-mer table, BatchLocate) must give the oracle's SMEMs, max-occ filtering and hits."""
import numpy as np
import pytest

import cpu_batched
import oracle
import synth


def build(ref, **kw):
    X = oracle.Index(ref, **kw)
    return X, cpu_batched.Index(X.bwt(), X.primary, X.ssa())


def check(Y, X, seq, off, l=19, c=1, max_occ=500, batch=4096):
    sm, hits = Y.seed(seq, off, l, c, max_occ, batch=batch)
    osm, over, hoff, ohits = X.seed(seq, off, l, c, max_occ)
    assert len(sm) == len(osm)
    for f in ("read", "qbeg", "qend", "k", "kr", "s"):
        assert np.array_equal(sm[f], osm[f]), f
    assert np.array_equal(hits.astype(np.uint64), ohits)


def test_workload1_all_reads():
    ref, rd, p = synth.workload(1, scale=0.2)
    X, Y = build(ref)
    check(Y, X, rd.seq, rd.off)


@pytest.mark.parametrize("l,c,max_occ,batch", [(19, 1, 500, 97), (12, 2, 50, 4096), (25, 1, 3, 1), (5, 3, 500, 333)])
def test_repeat_rich_with_n_and_parameters(l, c, max_occ, batch):
    ref, rd, p = synth.workload(2, scale=0.003)
    X, Y = build(ref)
    sub = rd.subset(np.arange(min(rd.n, 1500)))
    check(Y, X, sub.seq, sub.off, l, c, max_occ, batch)


def test_edge_reads():
    ref = synth.reference(20_000, 61)
    X, Y = build(ref)
    reads = [np.zeros(0, np.uint8), ref[100:118], ref[200:219], ref[300:320], np.full(150, 4, np.uint8),
             np.concatenate([ref[400:450], [4], ref[451:500]]), ref[1000:1150], synth.reference(150, 999)]
    seq = np.concatenate(reads).astype(np.uint8)
    off = np.concatenate([[0], np.cumsum([len(x) for x in reads])]).astype(np.uint64)
    check(Y, X, seq, off)
