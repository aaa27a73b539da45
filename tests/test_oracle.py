"""Pins of the CPU oracle against what the paper and the mathematics fix (no GPU).

Section 2.1 definitions: brute force on tiny texts, a hand-derived fixture,
the suffix array as a sorted permutation, invariants of (l,c)-SMEMs;
Algorithm 1 and 3 against the definition; Algorithm 2 against the full suffix
array; the bisulfite index layout of Section 2.9.
"""
import os

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
COMP = np.array([3, 2, 1, 0, 4], dtype=np.uint8)


def revcomp(x):
    return COMP[np.asarray(x, dtype=np.uint8)][::-1]


def parse_golden(name):
    rows = []
    for line in open(os.path.join(GOLDEN, name)):
        line = line.strip()
        if line and not line.startswith("#"):
            rows.append(line.split())
    return rows


def test_hand_derived_tiny_text():
    X = oracle.Index(np.array([0, 1, 2], np.uint8))
    assert X.n == 7
    for row in parse_golden("tiny_acg.txt"):
        tag, vals = row[0], row[1:]
        if tag == "SA":
            assert X.sa().tolist() == [int(v) for v in vals]
        elif tag == "BWT":
            assert X.bwt().tolist() == [int(v) for v in vals]
        elif tag == "PRIMARY":
            assert X.primary == int(vals[0])
        elif tag == "C":
            assert X.C.tolist() == [int(v) for v in vals]
        elif tag == "DS":
            pat = [] if vals[0] == "-" else [int(v) for v in vals[0].split(",")]
            assert X.ds_interval(np.array(pat, np.uint8)) == tuple(int(v) for v in vals[1:]), pat


def suffix_sorted_check(T, SA):
    """SA is a permutation of [0,n) and adjacent suffixes are in strictly increasing order."""
    n = len(T)
    assert np.array_equal(np.sort(SA), np.arange(n, dtype=SA.dtype))
    Tb = T.tobytes()
    for x in range(n - 1):
        assert Tb[SA[x]:] < Tb[SA[x + 1]:]


@pytest.mark.parametrize("length,seed", [(1, 1), (2, 2), (7, 3), (64, 4), (300, 5), (2500, 6)])
def test_suffix_array_sorted_permutation(length, seed):
    ref = synth.reference(length, seed)
    X = oracle.Index(ref)
    T, SA, B = X.text(), X.sa(), X.bwt()
    assert X.n == 2 * length + 1
    # T = R . revcomp(R) . $ in oracle coding
    assert np.array_equal(T[:length], ref + 1)
    assert np.array_equal(T[length:2 * length], revcomp(ref) + 1)
    assert T[-1] == 0
    suffix_sorted_check(T, SA)
    # B[i] = T[S(i) - 1], T[-1] = $
    assert np.array_equal(B, T[(SA.astype(np.int64) - 1) % X.n])
    assert SA[X.primary] == 0
    # C[a] = #{B < a}
    for a in range(5):
        assert X.C[a] == int((B < a).sum())
    # sampled SA
    assert np.array_equal(X.ssa(), SA[::32])


def test_suffix_array_repeats():
    # tandem and segmental repeats give long common prefixes
    ref = synth.repeat_rich_reference(20000, 77, 0.5)
    X = oracle.Index(ref, n_seed=3)
    suffix_sorted_check(X.text(), X.sa())


def test_ambiguous_bases_become_seeded_random_bases():
    ref = np.array([0, 4, 4, 1, 4, 2, 3] * 50, np.uint8)
    X1, X2, X3 = oracle.Index(ref, n_seed=5), oracle.Index(ref, n_seed=5), oracle.Index(ref, n_seed=6)
    T1 = X1.text()[:len(ref)]
    assert np.array_equal(T1, X2.text()[:len(ref)])
    assert T1.max() <= 4 and T1.min() >= 1          # no N left in T
    assert np.array_equal(T1[ref < 4], ref[ref < 4] + 1)
    assert not np.array_equal(T1, X3.text()[:len(ref)])
    counts = np.bincount(T1[ref == 4], minlength=5)[1:]
    assert counts.min() > 0                          # all four bases drawn


def brute_ds(T, P):
    """ds-interval straight from Section 2.1 by scanning T (oracle coding)."""
    n = len(T)
    Tb = T.tobytes()
    f = bytes((np.asarray(P, np.uint8) + 1).tolist())
    rc = bytes((revcomp(P) + 1).tolist())
    lo = sum(1 for i in range(n) if Tb[i:] < f and not Tb[i:].startswith(f))
    lor = sum(1 for i in range(n) if Tb[i:] < rc and not Tb[i:].startswith(rc))
    occ = sum(1 for i in range(n) if Tb[i:i + len(f)] == f)
    return lo, lor, occ


def test_ds_interval_by_scanning():
    rng = np.random.default_rng(1)
    ref = synth.reference(150, 11)
    X = oracle.Index(ref)
    T = X.text()
    for _ in range(300):
        m = int(rng.integers(1, 7))
        if rng.random() < 0.5:
            s = int(rng.integers(0, 2 * len(ref) - m))
            P = (T[s:s + m] - 1).astype(np.uint8)
            if (T[s:s + m] == 0).any():
                continue
        else:
            P = rng.integers(0, 4, m).astype(np.uint8)
        assert X.ds_interval(P) == brute_ds(T, P)


def test_backward_forward_ext_match_definition():
    """Algorithm 1 extends the ds-interval of P to that of aP / Pa."""
    rng = np.random.default_rng(2)
    ref = synth.repeat_rich_reference(3000, 12, 0.3)
    X = oracle.Index(ref)
    for _ in range(400):
        m = int(rng.integers(0, 12))
        P = rng.integers(0, 4, m).astype(np.uint8)
        a = int(rng.integers(0, 4))
        iv = X.ds_interval(P)
        assert X.backward_ext(iv, a) == X.ds_interval(np.concatenate([[a], P]).astype(np.uint8))
        assert X.forward_ext(iv, a) == X.ds_interval(np.concatenate([P, [a]]).astype(np.uint8))
    # N ends every match
    assert X.backward_ext((0, 0, X.n), 4) == (0, 0, 0)
    assert X.ds_interval(np.array([0, 4, 1], np.uint8)) == (0, 0, 0)


def test_pi_definition():
    ref = synth.reference(500, 13)
    X = oracle.Index(ref)
    B = X.bwt()
    for k in list(range(0, 70)) + list(range(X.n - 70, X.n + 1)):
        for a in range(5):
            assert X.pi(a, k) == int((B < a).sum() + (B[:k] == a).sum())


@pytest.mark.parametrize("seed", range(6))
def test_smem_three_ways_tiny(seed):
    """Definition (SA binary search) = Algorithm 3 = brute force over T."""
    rng = np.random.default_rng(seed)
    kind = seed % 3
    if kind == 0:
        ref = synth.reference(int(rng.integers(50, 2000)), 100 + seed)
    elif kind == 1:
        ref = synth.repeat_rich_reference(int(rng.integers(2000, 6000)), 100 + seed, 0.6)
    else:
        ref = np.tile(synth.reference(int(rng.integers(3, 40)), 100 + seed), 40)
    X = oracle.Index(ref, n_seed=seed)
    rd = synth.reads(ref, 30, 200 + seed, mode=0, read_len=int(rng.integers(20, 90)),
                     sub_lo=0.03, indel=0.01)
    # some reads with N and some from nowhere
    seq = rd.seq.copy()
    seq[rng.integers(0, len(seq), 5)] = 4
    rnd = synth.reads(synth.reference(5000, 300 + seed), 6, 400 + seed, mode=0, read_len=40)
    seq = np.concatenate([seq, rnd.seq])
    off = np.concatenate([rd.off, rd.off[-1] + rnd.off[1:]])
    T = X.text()
    for c in (1, 2, 3):
        for l in (1, 4, 9, 19, 25):
            a = oracle.smem_brute(T, seq, off, l, c)
            b = X.smem(seq, off, l, c, "def")
            d = X.smem(seq, off, l, c, "alg3")
            assert np.array_equal(a, b), (c, l)
            assert np.array_equal(b, d), (c, l)


def check_smem_invariants(X, seq, off, sm, l, c):
    by_read = {}
    for rec in sm:
        by_read.setdefault(int(rec["read"]), []).append(rec)
    for r, recs in by_read.items():
        P = seq[off[r]:off[r + 1]]
        qb = [int(x["qbeg"]) for x in recs]
        qe = [int(x["qend"]) for x in recs]
        # no SMEM contains another: both ends strictly ascending
        assert all(a < b for a, b in zip(qb, qb[1:])) and all(a < b for a, b in zip(qe, qe[1:]))
        for x in recs:
            i, j = int(x["qbeg"]), int(x["qend"])
            assert j - i >= l and int(x["s"]) >= c
            assert (int(x["k"]), int(x["kr"]), int(x["s"])) == X.ds_interval(P[i:j])
            # maximal on both sides
            if i > 0:
                assert X.ds_interval(P[i - 1:j])[2] < c
            if j < len(P):
                assert X.ds_interval(P[i:j + 1])[2] < c


def test_smem_invariants_workload1_sample():
    ref, rd, p = synth.workload(1, scale=0.05)
    X = oracle.Index(ref)
    sub = rd.subset(range(0, 200))
    sm = X.smem(sub.seq, sub.off, 19, 1)
    check_smem_invariants(X, sub.seq, sub.off, sm, 19, 1)
    # strand mirror: SMEMs of revcomp(P) are [|P|-j, |P|-i) with (k', k, s)
    rc_seq = np.concatenate([revcomp(sub.read(i)) for i in range(sub.n)])
    sm_rc = X.smem(rc_seq, sub.off, 19, 1)
    for r in range(sub.n):
        L = int(sub.off[r + 1] - sub.off[r])
        a = sorted((L - int(x["qend"]), L - int(x["qbeg"]), int(x["kr"]), int(x["k"]), int(x["s"]))
                   for x in sm[sm["read"] == r])
        b = sorted((int(x["qbeg"]), int(x["qend"]), int(x["k"]), int(x["kr"]), int(x["s"]))
                   for x in sm_rc[sm_rc["read"] == r])
        assert a == b


def test_error_free_read_single_smem_and_origin():
    ref = synth.reference(200_000, 21)
    X = oracle.Index(ref)
    rd = synth.reads(ref, 50, 22, mode=0, read_len=150)
    sm, over, hoff, hits = X.seed(rd.seq, rd.off)
    assert len(sm) == rd.n
    assert np.all(sm["qbeg"] == 0) and np.all(sm["qend"] == 150)
    for r in range(rd.n):
        st, s = int(rd.origin[r]) >> 63, int(rd.origin[r]) & ((1 << 63) - 1)
        h = hits[int(hoff[r]):int(hoff[r]) + int(sm["s"][r])]
        # forward reads start at s; reverse reads are revcomp(ref[s+16 .. s+166)) -> T position
        want = s if st == 0 else 2 * len(ref) - (s + 166)
        assert want in h.tolist()


def test_locate_three_ways_and_spelling():
    ref, rd, p = synth.workload(2, scale=0.002)
    X = oracle.Index(ref, n_seed=9)
    T = X.text()
    sub = rd.subset(range(0, 300))
    sm, over, hoff, hits = X.seed(sub.seq, sub.off, max_occ=20)
    assert len(hits) == int(np.where(over, 0, sm["s"]).sum())
    rows = np.concatenate([np.arange(int(x["k"]), int(x["k"] + x["s"]), dtype=np.uint64)
                           for x, o in zip(sm, over) if not o])
    assert np.array_equal(X.locate_slow(rows), hits)
    assert np.array_equal(X.batch_locate(rows), hits)
    for x, o, h0 in zip(sm, over, hoff):
        if o:
            continue
        P = sub.seq[sub.off[x["read"]] + x["qbeg"]:sub.off[x["read"]] + x["qend"]] + 1
        for t in hits[int(h0):int(h0) + int(x["s"])]:
            assert np.array_equal(T[int(t):int(t) + len(P)], P)
    # every SA row, and the walk through the $ row
    allrows = np.arange(X.n, dtype=np.uint64)
    assert np.array_equal(X.locate_slow(allrows), X.sa().astype(np.uint64))


def test_max_occ_flag_and_hit_offsets():
    ref = np.tile(synth.reference(37, 5), 700)   # every 19-mer occurs hundreds of times
    X = oracle.Index(ref)
    rd = synth.reads(ref, 20, 6, mode=0, read_len=60)
    sm, over, hoff, hits = X.seed(rd.seq, rd.off, max_occ=500)
    assert np.array_equal(over, sm["s"] > 500)
    assert over.any()
    kept = np.where(over, 0, sm["s"])
    assert np.array_equal(hoff, np.concatenate([[0], np.cumsum(kept)[:-1]]).astype(np.uint64))


def test_max_occ_boundary_on_planted_copies():
    """The workload's cap (not in the paper): an SMEM occurring exactly max_occ times is kept and
    located, one occurring max_occ + 1 times is flagged and gets no hits.  Each read is a unit
    planted a known number of times in a random reference, so s and the hit positions come from
    the construction, not from the oracle's own arithmetic."""
    ref, units, starts = synth.planted_copies(40, [500, 501, 3], 60, 0x6D6201)
    X = oracle.Index(ref)
    seq = units.reshape(-1)
    off = np.arange(len(units) + 1, dtype=np.uint64) * 40
    for max_occ, flagged in ((500, [False, True, False]), (499, [True, True, False]),
                             (501, [False, False, False])):
        sm, over, hoff, hits = X.seed(seq, off, max_occ=max_occ)
        assert sm["read"].tolist() == [0, 1, 2]
        assert sm["qbeg"].tolist() == [0, 0, 0] and sm["qend"].tolist() == [40, 40, 40]
        assert sm["s"].tolist() == [500, 501, 3]
        assert over.tolist() == flagged
        kept = [c for c, f in zip((500, 501, 3), flagged) if not f]
        assert len(hits) == sum(kept)
        assert hoff.tolist() == [0, 0 if flagged[0] else 500, (0 if flagged[0] else 500) + (0 if flagged[1] else 501)]
        for u in range(3):
            if not flagged[u]:
                h0 = int(hoff[u])
                assert np.array_equal(np.sort(hits[h0:h0 + [500, 501, 3][u]]), starts[u])


def test_bisulfite_filter_drops_hit_spanning_two_copies():
    """Section 2.9's strand rule keeps a hit only inside one copy of the 3-base text.  A read-1
    read planted across the end of the C-to-T copy and the start of the G-to-A copy has one
    occurrence, at a known place, spanning both copies: it is dropped; a control read inside the
    C-to-T copy is kept."""
    m, half = 5000, 20
    ref, cross = synth.junction_read(m, half, 0x6D6202)
    X = oracle.Index(ref, bs3=True)
    ctl = ref[1000:1000 + 2 * half]
    seq = np.concatenate([cross, ctl]).astype(np.uint8)
    off = np.array([0, 2 * half, 4 * half], dtype=np.uint64)
    mate = np.array([1, 1], dtype=np.uint8)
    conv = oracle.bs_convert_reads(seq, off, mate)
    T = X.text()
    assert np.array_equal(T[m - half:m + half], conv[:2 * half] + 1)   # the planted span
    sm, over, hoff, hits = X.seed(conv, off)
    assert sm["read"].tolist() == [0, 1]
    assert sm["qbeg"].tolist() == [0, 0] and sm["qend"].tolist() == [2 * half, 2 * half]
    assert sm["s"].tolist() == [1, 1]
    assert hits.tolist() == [m - half, 1000]
    keep = oracle.bs_keep(hits, np.array([2 * half, 2 * half]), mate, m)
    assert keep.tolist() == [False, True]


def test_bisulfite_index_and_filter():
    ref = synth.reference(3000, 31)
    X = oracle.Index(ref, bs3=True)
    m = len(ref)
    T = X.text()
    assert X.n == 4 * m + 1 and X.rlen == 2 * m
    ct = np.where(ref == 1, 3, ref)
    ga = np.where(ref == 2, 0, ref)
    assert np.array_equal(T[:m], ct + 1)
    assert np.array_equal(T[m:2 * m], ga + 1)
    assert np.array_equal(T[2 * m:3 * m], revcomp(ga) + 1)
    assert np.array_equal(T[3 * m:4 * m], revcomp(ct) + 1)
    suffix_sorted_check(T, X.sa())
    # bisulfite pairs: the read's true segment is among the kept hits
    rd = synth.reads(ref, 40, 32, mode=1, read_len=100, bisulfite=True)
    seq = oracle.bs_convert_reads(rd.seq, rd.off, rd.mate)
    sm, over, hoff, hits = X.seed(seq, rd.off)
    qlen = np.repeat((sm["qend"] - sm["qbeg"]).astype(np.int64), np.where(over, 0, sm["s"]).astype(np.int64))
    rmate = np.repeat(rd.mate[sm["read"].astype(np.int64)], np.where(over, 0, sm["s"]).astype(np.int64))
    keep = oracle.bs_keep(hits, qlen, rmate, m)
    segs = (hits // m)[keep]
    assert set(segs[rmate[keep] == 1].tolist()) <= {0, 2}
    assert set(segs[rmate[keep] == 2].tolist()) <= {1, 3}
    assert keep.sum() > 0


def test_second_round_windows_by_brute_force():
    """Section 2.6: the second round's SMEMs of each window equal brute force on that window."""
    ref = synth.repeat_rich_reference(6000, 41, 0.5)
    X = oracle.Index(ref)
    T = X.text()
    rd = synth.reads(ref, 40, 42, mode=0, read_len=120, sub_lo=0.01)
    sm1 = X.smem(rd.seq, rd.off, 19, 1)
    sm2, over, hoff, hits = oracle.reseed(X, rd.seq, rd.off, sm1)
    wins = [x for x in sm1 if int(x["qend"]) - int(x["qbeg"]) >= 38 and int(x["s"]) <= 10]
    assert wins
    want = []
    for x in wins:
        r, b, e, s = int(x["read"]), int(x["qbeg"]), int(x["qend"]), int(x["s"])
        w = rd.seq[int(rd.off[r]) + b:int(rd.off[r]) + e]
        got = oracle.smem_brute(T, w, np.array([0, len(w)], np.uint64), (e - b) // 2, s + 1)
        want += [(r, int(y["qbeg"]) + b, int(y["qend"]) + b, int(y["k"]), int(y["kr"]), int(y["s"])) for y in got]
    have = [tuple(int(y[f]) for f in ("read", "qbeg", "qend", "k", "kr", "s")) for y in sm2]
    assert have == want
    assert all(int(y["s"]) >= 2 for y in sm2)


def test_locate_work_counts_by_suffix_array():
    """LF steps and sampled-S reads of Algorithm 2 (the $ row taken as sampled with S = 0), pinned
    by the suffix array alone: the walk from row x visits rows ISA[S(x) - j] for j = 0, 1, ...
    and stops at the first row that is a multiple of r, or at text position 0 (the $ row)."""
    ref = synth.repeat_rich_reference(30_000, 31, 0.3)
    X = oracle.Index(ref, sa_rate=8)
    S = X.sa().astype(np.int64)
    isa = np.empty_like(S)
    isa[S] = np.arange(X.n)
    rows = np.random.default_rng(3).choice(X.n, 3000, replace=False).astype(np.uint64)
    want_steps = want_sa = 0
    for x in rows.tolist():
        t, j = int(S[x]), 0
        while isa[t - j] % 8 != 0 and t - j != 0:
            j += 1
        want_steps += j
        want_sa += int(isa[t - j] % 8 == 0)
    assert X.count_locate(rows) == (want_steps, want_sa)


def test_alg3_work_counts_exact_unique_read():
    """An error-free read that occurs in T takes exactly |P| extension steps in Algorithm 3
    (l backward steps of stage 1, then |P| - l forward steps to the end, no stage 3); the blocks
    each step reads follow from the intervals of the definition: backward step j extends
    P[j+1, l) (rows k and k+s), forward step j extends P[0, j) (rows k' and k'+s)."""
    ref = synth.reference(100_000, 41)
    X = oracle.Index(ref)
    l, L = 19, 120
    for start in (1000, 55_555, 99_000):
        P = ref[start:start + L].astype(np.uint8)
        off = np.array([0, L], np.uint64)
        br = 64
        blocks = 0
        for j in range(l - 1, -1, -1):
            k, kr, s = X.ds_interval(P[j + 1:l]) if j + 1 < l else (0, 0, X.n)
            blocks += 1 if k // br == (k + s) // br else 2
        for j in range(l, L):
            k, kr, s = X.ds_interval(P[0:j])
            blocks += 1 if kr // br == (kr + s) // br else 2
        assert X.count_alg3(P, off, l, 1, br) == (L, blocks)
        # the same with 128-row blocks
        assert X.count_alg3(P, off, l, 1, 128)[0] == L


@pytest.mark.parametrize("l,c", [(19, 1), (19, 2), (12, 3), (10, 1), (25, 1)])
def test_alg3_with_kmer_cache_gives_the_definition(l, c):
    """Section 2.5's 10-mer cache changes only the work: Algorithm 3 with it gives exactly the
    SMEMs of the definition (repeat-rich reads with N)."""
    ref, rd, p = synth.workload(2, scale=0.003)
    X = oracle.Index(ref)
    sub = rd.subset(np.arange(min(rd.n, 1500)))
    d = X.smem(sub.seq, sub.off, l, c, "def")
    a = X.smem(sub.seq, sub.off, l, c, "alg3_cache")
    assert len(d) > 0 and d.tobytes() == a.tobytes()


def test_alg3_kmer_cache_work_counts_exact_unique_read():
    """An error-free read that occurs in T, with the 10-mer cache: one lookup covers the last 10
    bases of the first window, then l - 10 backward steps and |P| - l forward steps, |P| - 10 in
    all; the blocks follow from the definition's intervals as without the cache."""
    ref = synth.reference(100_000, 41)
    X = oracle.Index(ref)
    l, L, K = 19, 120, 10
    for start in (1000, 55_555, 99_000):
        P = ref[start:start + L].astype(np.uint8)
        off = np.array([0, L], np.uint64)
        for br in (64, 128):
            blocks = 0
            for j in range(l - K - 1, -1, -1):
                k, kr, s = X.ds_interval(P[j + 1:l])
                blocks += 1 if k // br == (k + s) // br else 2
            for j in range(l, L):
                k, kr, s = X.ds_interval(P[0:j])
                blocks += 1 if kr // br == (kr + s) // br else 2
            assert X.count_alg3(P, off, l, 1, br, kmer_k=K) == (L - K, blocks, 1)


def test_locate_join_work_counts_by_suffix_array():
    """Walks that join, from the suffix array alone: the walk from the row of text position p
    visits the rows of p-1, p-2, ...; it stops at the first position q <= p whose row is sampled
    or is the $ row (q = 0), or, for q < p, whose row is another of the walked rows and lies in
    an earlier pass (pass of row y: the top bits of the 32-bit product y * 2654435761).  Its LF
    steps are p - q; the oracle's counts (steps, S reads, joins) must match this scan."""
    ref, rd, p = synth.workload(2, scale=0.002)
    X = oracle.Index(ref)
    sm, over, hoff, hits = X.seed(rd.seq, rd.off)
    rows = np.unique(np.concatenate([np.arange(int(k), int(k) + int(s_), dtype=np.uint64)
                                     for k, s_, o in zip(sm["k"], sm["s"], over) if not o]))
    SA = X.sa().astype(np.int64)
    n = len(SA)
    ISA = np.empty(n, np.int64)
    ISA[SA] = np.arange(n)
    walked = np.zeros(n, bool)
    walked[rows.astype(np.int64)] = True
    plain = X.count_locate(rows)

    def scan(bits):
        def pass_of(y):
            return ((int(y) * 2654435761) & 0xFFFFFFFF) >> (32 - bits) if bits else 0
        steps = sa = links = 0
        for row in rows.astype(np.int64):
            pos, t, own = int(SA[row]), 0, pass_of(row)
            while True:
                rr = ISA[pos - t]
                if rr % 32 == 0:
                    sa += 1
                    break
                if pos - t == 0:          # the row of position 0 is the $ row
                    break
                if t > 0 and walked[rr] and pass_of(rr) < own:
                    links += 1
                    break
                t += 1
            steps += t
        return steps, sa, links

    for bits in (0, 1, 3):
        got = X.count_locate_join(rows, pass_bits=bits)
        assert got == scan(bits), bits
    assert X.count_locate_join(rows, pass_bits=0) == plain + (0,)   # one pass: the plain walks
    steps, sa, links = X.count_locate_join(rows, pass_bits=3)
    assert links > len(rows) // 4          # repeat-rich reads: many walks join
    assert steps < plain[0] // 2


def _bs_seed_and_split(ref, seq, off, mate):
    X = oracle.Index(ref, bs3=True)
    conv = oracle.bs_convert_reads(seq, off, mate)
    sm, over, hoff, hits = X.seed(conv, off)
    cnt = np.where(over, 0, sm["s"]).astype(np.int64)
    qlen = np.repeat((sm["qend"] - sm["qbeg"]).astype(np.int64), cnt)
    rmate = np.repeat(np.asarray(mate)[sm["read"].astype(np.int64)], cnt)
    keep = oracle.bs_keep(hits, qlen, rmate, len(ref))
    return sm, over, hits, keep, oracle.bs_split(ref, seq, off, mate, sm, hits, keep, over=over)


def test_bs_split_planted_mismatches():
    """Section 2.9 split, hand-derived: read-1 C over reference T cuts a forward seed and a
    reverse seed; read-2 G over reference A cuts a forward G-to-A seed; pieces under 19 go."""
    ref = synth.reference(50_000, 77)
    M = len(ref)
    r1 = ref[100:160].copy()                       # read 1, forward strand
    t_pos = [t for t in range(25, 40) if r1[t] == 3][0]
    r1[t_pos] = 1                                  # C over reference T
    rc = revcomp(ref[200:260]).copy()              # read 1, reverse strand
    t_rc = [t for t in range(5, 15) if rc[t] == 3][0]
    rc[t_rc] = 1
    r2 = ref[300:360].copy()                       # read 2, forward strand (G->A copy)
    a_pos = [t for t in range(30, 45) if r2[t] == 0][0]
    r2[a_pos] = 2                                  # G over reference A
    seq = np.concatenate([r1, rc, r2]).astype(np.uint8)
    off = np.array([0, 60, 120, 180], np.uint64)
    mate = np.array([1, 1, 2], np.uint8)
    sm, over, hits, keep, pc = _bs_seed_and_split(ref, seq, off, mate)
    got = sorted((int(p["read"]), int(p["qbeg"]), int(p["qend"]), int(p["pos"])) for p in pc)
    want = [(0, 0, t_pos, 100), (0, t_pos + 1, 60, 100 + t_pos + 1)]
    q_rc = M - 260                                 # offset in copy 2 = rc(GA(R)) = CT(rc(R))
    if t_rc >= 19:
        want.append((1, 0, t_rc, 2 * M + q_rc))
    want.append((1, t_rc + 1, 60, 2 * M + q_rc + t_rc + 1))
    want += [(2, 0, a_pos, M + 300), (2, a_pos + 1, 60, M + 300 + a_pos + 1)]
    assert got == sorted(want)


def test_bs_split_invariants():
    """Pieces lie inside their seed, do not overlap, are at least 19 long, hold no cutting pair,
    and are maximal: each end is a seed end or next to a cutting position."""
    ref = synth.reference(40_000, 79)
    rd = synth.reads(ref, 300, 80, mode=1, read_len=150, bisulfite=True, sub_lo=0.01, sub_hi=0.03)
    sm, over, hits, keep, pc = _bs_seed_and_split(ref, rd.seq, rd.off, rd.mate)
    assert len(pc) > 0
    M = len(ref)
    comp = np.array([3, 2, 1, 0, 4], np.uint8)
    owner = np.repeat(np.arange(len(sm)), np.where(over, 0, sm["s"]).astype(np.int64))
    ncut = 0
    for p in pc:
        m = owner[int(p["hit"])]
        qb, qe = int(sm["qbeg"][m]), int(sm["qend"][m])
        assert keep[int(p["hit"])] and qb <= p["qbeg"] < p["qend"] <= qe and p["qend"] - p["qbeg"] >= 19
        hp = int(hits[int(p["hit"])])
        assert int(p["pos"]) == hp + int(p["qbeg"]) - qb
        rd_i, mt = int(p["read"]), int(rd.mate[int(p["read"])])

        def cuts(t):   # is read position t (absolute in the read) a cutting position?
            g, q = hp // M, hp - (hp // M) * M
            u = q + t - qb
            R = ref[u] if g < 2 else comp[ref[M - 1 - u]]
            x = rd.seq[int(rd.off[rd_i]) + t]
            return (mt == 1 and x == 1 and R == 3) or (mt == 2 and x == 2 and R == 0)
        assert not any(cuts(t) for t in range(int(p["qbeg"]), int(p["qend"])))
        assert p["qbeg"] == qb or cuts(int(p["qbeg"]) - 1)
        assert p["qend"] == qe or cuts(int(p["qend"]))
        ncut += int(p["qbeg"] != qb)
    assert ncut > 0


def test_qmer_prefilter_closed_forms():
    """Section 2.7 prefilter: a read copied from the window has every q-mer on one diagonal
    (max M_t = |P| - q + 1); each substitution at least q bases from the others and from the ends
    removes exactly q of them; an N removes the q-mers that cover it; a periodic pair keeps the
    full count on its best diagonal."""
    q = 7
    R = synth.reference(400, 91)
    P = R[120:270].copy()
    assert oracle.qmer_diag_max(P, R, q) == 150 - q + 1
    P2 = P.copy()
    for x in (20, 60, 100):
        P2[x] = (P2[x] + 1) % 4
    assert oracle.qmer_diag_max(P2, R, q) == 150 - q + 1 - 3 * q
    P3 = P.copy()
    P3[75] = 4
    assert oracle.qmer_diag_max(P3, R, q) == 150 - q + 1 - q
    per = np.tile(np.array([0, 1], np.uint8), 75)
    assert oracle.qmer_diag_max(per, np.tile(np.array([0, 1], np.uint8), 150), q) == 150 - q + 1
    assert oracle.qmer_diag_max(P[:q - 1], R, q) == 0


def test_qmer_prefilter_batch_equals_pairwise_definition():
    rng = np.random.default_rng(5)
    reads, wins = [], []
    for t in range(40):
        R = rng.integers(0, 4, int(rng.integers(5, 500))).astype(np.uint8)
        if t % 2 and len(R) > 200:
            s = int(rng.integers(0, len(R) - 150))
            P = R[s:s + 150].copy()
        else:
            P = rng.integers(0, 4, int(rng.integers(3, 160))).astype(np.uint8)
        k = min(len(P), 4)
        P[rng.integers(0, len(P), k)] = rng.integers(0, 5, k)
        reads.append(P)
        wins.append(R)
    ro = np.concatenate([[0], np.cumsum([len(x) for x in reads])])
    wo = np.concatenate([[0], np.cumsum([len(x) for x in wins])])
    got = oracle.qmer_diag_max_batch(np.concatenate(reads), ro, np.concatenate(wins), wo)
    want = [oracle.qmer_diag_max(P, R) for P, R in zip(reads, wins)]
    assert got.tolist() == want
