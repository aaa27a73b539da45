"""Second seeding round (Section 2.6): (floor(len/2), s+1)-SMEMs inside every first-round SMEM
of at least 2l bases occurring at most 10 times, against the oracle's definition."""
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


@pytest.mark.parametrize("cfg,scale", [(1, 0.2), (2, 0.01), (4, 0.003)])
def test_reseed_matches_oracle(mb, cfg, scale):
    ref, rd, params = synth.workload(cfg, scale)
    G = mb.mb_index_build(ref)
    X = oracle.Index(ref)
    sm1, m1, nh1 = mb.mb_seed_batch(G, rd.seq, rd.off)
    sm2, m2, nh2 = mb.mb_reseed(G, rd.seq, rd.off, sm1, m1)
    osm1, _, _, _ = X.seed(rd.seq, rd.off)
    osm2, over, hoff, ohits = oracle.reseed(X, rd.seq, rd.off, osm1)
    assert m2 == len(osm2) and m2 > 0
    for f in ("read", "qbeg", "qend", "k", "kr", "s"):
        assert np.array_equal(sm2[f].astype(np.uint64), osm2[f]), f
    assert np.all(sm2["flags"] & mb.MB_SMEM_ROUND2)
    assert np.array_equal((sm2["flags"] & 1).astype(bool), over)
    assert np.array_equal(sm2["hit_off"], hoff)
    hits, _ = mb.mb_locate(G, sm2, m2, cap=nh2)
    assert np.array_equal(hits.astype(np.uint64), ohits)
    # every second-round SMEM lies inside a first-round SMEM of its read and occurs more often
    assert np.all(sm2["s"] >= 2)
