"""Mate-rescue prefilter (Section 2.7) on the GPU against the oracle's definition: max over
diagonals t of the number of q-mer matches (i, j) with j - i = t, per (read, window) pair."""
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


def test_mate_rescue_shaped_pairs(mb):
    ref = synth.repeat_rich_reference(300_000, 95, 0.2)
    r, ro, w, wo = synth.rescue_pairs(ref, 3000, 96)
    want = oracle.qmer_diag_max_batch(r, ro, w, wo)
    assert 0.3 < (want >= 10).mean() < 0.7
    assert np.array_equal(mb.mb_rescue_prefilter(r, ro, w, wo), want)
    got = torch.empty(len(want), dtype=torch.int32, device="cuda")
    mb.mb_rescue_prefilter(dev(r), dev(ro), dev(w), dev(wo), best=got)
    assert np.array_equal(got.cpu().numpy().view(np.uint32), want)


@pytest.mark.parametrize("q", [1, 4, 7, 11, 15])
def test_lengths_ns_and_q(mb, q):
    """Reads of 0-300 bases, windows of 0-2,000 (shorter than q included), N bases, any q."""
    rng = np.random.default_rng(q)
    reads, wins = [], []
    for t in range(600):
        W = rng.integers(0, 4, int(rng.integers(0, 2000))).astype(np.uint8)
        if t % 3 == 0 and len(W) > 300:
            s = int(rng.integers(0, len(W) - 300))
            P = W[s:s + int(rng.integers(0, 300))].copy()
        else:
            P = rng.integers(0, 4, int(rng.integers(0, 300))).astype(np.uint8)
        for x in (P, W):
            if len(x):
                k = int(rng.integers(0, 4))
                x[rng.integers(0, len(x), k)] = 4
        reads.append(P)
        wins.append(W)
    ro = np.concatenate([[0], np.cumsum([len(x) for x in reads])]).astype(np.uint64)
    wo = np.concatenate([[0], np.cumsum([len(x) for x in wins])]).astype(np.uint64)
    r, w = np.concatenate(reads).astype(np.uint8), np.concatenate(wins).astype(np.uint8)
    want = oracle.qmer_diag_max_batch(r, ro, w, wo, q)
    assert np.array_equal(mb.mb_rescue_prefilter(r, ro, w, wo, q=q), want)


def test_periodic_pairs_and_empty_batch(mb):
    P = np.tile(np.array([0, 1], np.uint8), 100)
    W = np.tile(np.array([0, 1], np.uint8), 400)
    got = mb.mb_rescue_prefilter(P, np.array([0, 200], np.uint64), W, np.array([0, 800], np.uint64))
    assert got.tolist() == [200 - 7 + 1]
    e = mb.mb_rescue_prefilter(P, np.array([0], np.uint64), W, np.array([0], np.uint64))
    assert len(e) == 0
    with pytest.raises(mb.MbError):
        mb.mb_rescue_prefilter(P, np.array([0, 200], np.uint64), W, np.array([0, 800], np.uint64), q=16)
