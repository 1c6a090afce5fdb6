"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

Every test here checks the oracle against something other than itself:
hand-worked vectors (tests/golden), closed forms, a textbook formula written
as a different sum, a library routine, brute force, or a proven bound.
"""
import itertools
import json
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2411_02268_gb300 import gen

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def load(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


def two_triangles():
    t = load("two_triangles.json")
    e = np.array(t["edges"])
    return gen.from_edges(t["n"], e[:, 0], e[:, 1], np.ones(len(e))), t


# ---- Algorithm 1 --------------------------------------------------------------

@pytest.mark.parametrize("case", load("sketch_vectors.json")["cases"], ids=lambda c: c["name"])
def test_sketch_hand_vectors(case):
    keys, vals = oracle.new_sketch(case["k"])
    for (c, w), exp in zip(case["stream"], case["after"]):
        oracle.sketch_update(keys, vals, c, w, case["uncond"])
        assert keys.tolist() == exp["keys"]
        assert vals.tolist() == exp["vals"]


def _random_stream(rng, ncomm, length, wmax):
    return [(int(rng.integers(ncomm)), int(rng.integers(1, wmax + 1))) for _ in range(length)]


@pytest.mark.parametrize("seed", range(20))
def test_sketch_unit_weights_misra_gries_bound(seed):
    """With unit weights the conditional rule is textbook Misra-Gries: each
    estimate lies in [f - n/(k+1), f], so every item with f > n/(k+1)
    survives (Section 3.6)."""
    rng = np.random.default_rng(seed)
    k = int(rng.choice([1, 2, 4, 8]))
    # skewed stream: a few heavy communities
    ncomm = int(rng.integers(2, 40))
    p = rng.pareto(1.0, ncomm) + 1e-3
    p /= p.sum()
    n = int(rng.integers(1, 400))
    stream = [(int(c), 1) for c in rng.choice(ncomm, size=n, p=p)]
    keys, vals = oracle.sketch_stream(stream, k)
    f = np.bincount([c for c, _ in stream], minlength=ncomm)
    est = {int(kk): int(v) for kk, v in zip(keys, vals) if v > 0}
    for c in range(ncomm):
        e = est.get(c, 0)
        assert e <= f[c]
        assert e >= f[c] - n / (k + 1) - 1e-9
        if f[c] > n / (k + 1):
            assert c in est


@pytest.mark.parametrize("seed", range(20))
def test_sketch_exact_when_few_communities(seed):
    """Conditional rule: with at most k distinct keys nothing is ever
    subtracted, so the sketch holds the exact per-community sums."""
    rng = np.random.default_rng(100 + seed)
    k = int(rng.choice([1, 2, 4, 8, 16]))
    ncomm = int(rng.integers(1, k + 1))
    stream = _random_stream(rng, ncomm, int(rng.integers(0, 200)), 16)
    keys, vals = oracle.sketch_stream(stream, k)
    exact = {}
    for c, w in stream:
        exact[c] = exact.get(c, 0) + w
    got = {int(kk): int(v) for kk, v in zip(keys, vals) if v > 0}
    assert got == exact


@pytest.mark.parametrize("seed", range(20))
def test_textbook_weighted_mg_bound(seed):
    """subtract = 2 is the weighted Misra-Gries summary of the literature:
    every decrement removes (k + 1) d of weight (d from each slot and d of the
    incoming item), so each estimate lies in [f - W/(k+1), f] for weighted
    streams of total W, and every key heavier than W/(k+1) survives.  The
    paper's clamped rule has no such guarantee (vector V3)."""
    rng = np.random.default_rng(300 + seed)
    k = int(rng.choice([1, 2, 4, 8]))
    ncomm = int(rng.integers(2, 40))
    p = rng.pareto(1.0, ncomm) + 1e-3
    p /= p.sum()
    n = int(rng.integers(1, 300))
    stream = [(int(c), int(rng.integers(1, 17))) for c in rng.choice(ncomm, size=n, p=p)]
    W = sum(w for _, w in stream)
    keys, vals = oracle.sketch_stream(stream, k, uncond=2)
    f = np.zeros(ncomm, dtype=np.int64)
    for c, w in stream:
        f[c] += w
    est = {int(kk): int(v) for kk, v in zip(keys, vals) if v > 0}
    for c in range(ncomm):
        e = est.get(c, 0)
        assert e <= f[c]
        assert e >= f[c] - W / (k + 1) - 1e-9
        if f[c] > W / (k + 1):
            assert c in est


def test_textbook_weighted_mg_keeps_v3_majority():
    """Vector V3 under the textbook rule: (b,1) then (a,3) with k = 1 keeps a
    with 3 - 1 = 2 (the paper's clamped rule loses a)."""
    keys, vals = oracle.sketch_stream([(11, 1), (10, 3)], 1, uncond=2)
    assert keys.tolist() == [10] and vals.tolist() == [2]
    keys, vals = oracle.sketch_stream([(11, 1), (10, 3)], 1)
    assert vals.tolist() == [0]


def test_sketch_weighted_bm_k1_majority():
    """k=1 weighted Boyer-Moore keeps a key whose weight exceeds the rest of
    the stream when it comes first in a run (sanity of the k=1 case)."""
    keys, vals = oracle.sketch_stream([(3, 5), (4, 1), (4, 1), (3, 2)], 1)
    assert keys.tolist() == [3] and vals.tolist() == [5]


@pytest.mark.parametrize("seed", range(10))
def test_merge_exact_when_union_small(seed):
    """merge of partial sketches whose key union has <= k keys = exact sums."""
    rng = np.random.default_rng(200 + seed)
    k = 8
    ncomm = int(rng.integers(1, k + 1))
    a = _random_stream(rng, ncomm, 30, 9)
    b = _random_stream(rng, ncomm, 30, 9)
    ak, av = oracle.sketch_stream(a, k)
    bk, bv = oracle.sketch_stream(b, k)
    oracle.sketch_merge(ak, av, bk, bv)
    exact = {}
    for c, w in a + b:
        exact[c] = exact.get(c, 0) + w
    assert {int(x): int(y) for x, y in zip(ak, av) if y > 0} == exact


def test_row_sketch_stream_partition_by_hand():
    """Stream partition: entry e goes to stream (e // V) % L, streams merged
    by the tree S[s] = merge(S[s], S[s+o]), o = L/2..1.  Rebuilt here from
    explicit per-stream sketches."""
    g = gen.random_graph(40, 600, 7, seed=3)
    labels = (np.arange(g.n) % 11).astype(np.uint32)
    k, L, V = 4, 4, 2
    sched = oracle.Schedule([10**9], [L], V)
    i = int(np.argmax(g.degrees()))
    keys, vals = oracle.row_sketch(g, i, labels, k, sched)
    streams = [[] for _ in range(L)]
    for e in range(g.offsets[i], g.offsets[i + 1]):
        j = int(g.cols[e])
        if j != i:
            streams[(e // V) % L].append((int(labels[j]), int(g.w[e])))
    S = [oracle.sketch_stream(s, k) for s in streams]
    o = L // 2
    while o >= 1:
        for s in range(o):
            oracle.sketch_merge(S[s][0], S[s][1], S[s + o][0], S[s + o][1])
        o //= 2
    assert keys.tolist() == S[0][0].tolist() and vals.tolist() == S[0][1].tolist()


# ---- Eq. 1 ---------------------------------------------------------------------

def q_textbook(g, labels):
    """Q = (1/2m) sum_ij [A_ij - K_i K_j / 2m] delta(c_i, c_j), double sum over
    vertex pairs (Newman-Girvan form), exact rationals."""
    n = g.n
    A = np.zeros((n, n), dtype=object)
    for i in range(n):
        for e in range(g.offsets[i], g.offsets[i + 1]):
            A[i, int(g.cols[e])] += int(g.w[e])
    K = [sum(A[i, j] for j in range(n)) for i in range(n)]
    two_m = sum(K)
    tot = Fraction(0)
    for i in range(n):
        for j in range(n):
            if labels[i] == labels[j]:
                tot += Fraction(A[i, j]) - Fraction(K[i] * K[j], two_m)
    return tot / two_m


@pytest.mark.parametrize("seed", range(12))
def test_modularity_textbook_double_sum(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(2, 14))
    g = gen.random_graph(n, int(rng.integers(1, 40)), 9, seed=seed, self_loops=bool(seed % 2))
    if g.nnz == 0:
        return
    labels = rng.integers(0, n, size=n).astype(np.uint32)
    assert oracle.modularity_fraction(g, labels) == q_textbook(g, labels)


def test_modularity_closed_forms():
    g, t = two_triangles()
    assert oracle.modularity_fraction(g, np.arange(6)) == Fraction(*t["q_singletons"])
    assert oracle.modularity_fraction(g, np.array(t["optimum_labels"])) == Fraction(*t["q_optimum"])
    # one community, no self-loops: sigma = 2m and Sigma = 2m, Q = 0
    assert oracle.modularity_fraction(g, np.zeros(6)) == 0
    # singletons on a ring of 5: -5 * (2/10)^2
    ring = gen.from_edges(5, [0, 1, 2, 3, 4], [1, 2, 3, 4, 0], [1] * 5)
    assert oracle.modularity_fraction(ring, np.arange(5)) == Fraction(-5, 25)


def test_modularity_networkx():
    nx = pytest.importorskip("networkx")
    g = gen.sbm(300, 6, 0.3, 0.02, wmax=5, seed=4)
    labels = (np.arange(300) * 6 // 300).astype(np.uint32)
    G = nx.Graph()
    G.add_nodes_from(range(g.n))
    for i in range(g.n):
        for e in range(g.offsets[i], g.offsets[i + 1]):
            j = int(g.cols[e])
            if i < j:
                G.add_edge(i, j, weight=int(g.w[e]))
    comms = [set(np.nonzero(labels == c)[0].tolist()) for c in range(6)]
    qn = nx.community.modularity(G, comms, weight="weight")
    assert abs(oracle.modularity(g, labels) - qn) < 1e-12


@pytest.mark.parametrize("seed", range(8))
def test_modularity_range(seed):
    g = gen.random_graph(30, 80, 5, seed=50 + seed)
    rng = np.random.default_rng(seed)
    for _ in range(20):
        lab = rng.integers(0, rng.integers(1, 30), size=30).astype(np.uint32)
        q = oracle.modularity_fraction(g, lab)
        assert Fraction(-1, 2) <= q <= 1
    # bipartite two-cluster extreme approaches -1/2
    kb = gen.from_edges(4, [0, 0, 1, 1], [2, 3, 2, 3], [1] * 4)
    assert oracle.modularity_fraction(kb, np.array([0, 0, 1, 1])) == Fraction(-1, 2)


# ---- Eq. 2 and the sweep decision -------------------------------------------------

def brute_sweep(g, labels, mode):
    """Synchronous sweep by brute force: for every vertex, evaluate every
    neighbouring community by exact recomputation of Q (Louvain) or by
    direct sums (LPA), with the same move rules as the oracle."""
    n = g.n
    labels = np.asarray(labels, dtype=np.uint32)
    size = np.bincount(labels, minlength=n)
    q0 = oracle.modularity_fraction(g, labels)
    K = oracle.degrees(g)
    two_m = int(K.sum())
    out, gains = labels.copy(), [0] * n
    for i in range(n):
        d = int(labels[i])
        link = {}
        for e in range(g.offsets[i], g.offsets[i + 1]):
            j = int(g.cols[e])
            if j != i:
                link[int(labels[j])] = link.get(int(labels[j]), 0) + int(g.w[e])
        kid = link.get(d, 0)
        best, bestv = d, None
        for c in sorted(link):
            if c == d:
                continue
            if mode == oracle.MODE_LPA:
                v = link[c]
                if v > kid and (bestv is None or v > bestv):
                    best, bestv = c, v
            else:
                if size[d] == 1 and size[c] == 1 and c > d:
                    continue
                lab2 = labels.copy()
                lab2[i] = c
                dq = oracle.modularity_fraction(g, lab2) - q0
                gain = dq * 2 * Fraction(two_m, 2) ** 2   # Eq. 2 scaled by 2m^2
                assert gain.denominator == 1
                if gain > 0 and (bestv is None or gain > bestv):
                    best, bestv = c, gain
        out[i] = best
        if bestv is not None:
            gains[i] = int(bestv) - (kid if mode == oracle.MODE_LPA else 0)
    return out, gains


def test_two_triangles_first_sweep():
    g, t = two_triangles()
    out, gains = oracle.sweep(g, np.arange(6, dtype=np.uint32), oracle.MODE_LOUVAIN, k=0)
    assert out.tolist() == t["sweep1_labels"]
    assert oracle.gains_as_ints(gains) == t["sweep1_gains"]
    out8, _ = oracle.sweep(g, np.arange(6, dtype=np.uint32), oracle.MODE_LOUVAIN, k=8)
    assert out8.tolist() == t["sweep1_labels"]


@pytest.mark.parametrize("seed", range(16))
@pytest.mark.parametrize("mode", [oracle.MODE_LOUVAIN, oracle.MODE_LPA])
def test_exact_sweep_matches_brute_force(seed, mode):
    rng = np.random.default_rng(300 + seed)
    n = int(rng.integers(3, 16))
    g = gen.random_graph(n, int(rng.integers(2, 50)), 6, seed=300 + seed,
                         self_loops=bool(seed % 3 == 0))
    labels = rng.integers(0, n, size=n).astype(np.uint32)
    if seed % 4 == 0:
        labels = np.arange(n, dtype=np.uint32)
    out, gains = oracle.sweep(g, labels, mode, k=0)
    bout, bgains = brute_sweep(g, labels, mode)
    assert out.tolist() == bout.tolist()
    assert oracle.gains_as_ints(gains) == bgains


@pytest.mark.parametrize("seed", range(8))
def test_mg_with_large_k_equals_exact(seed):
    """k >= number of neighbour communities: the conditional sketch is exact,
    so the MG sweep equals the exact sweep for any stream partition."""
    g = gen.random_graph(60, 300, 9, seed=400 + seed)
    rng = np.random.default_rng(seed)
    labels = rng.integers(0, 60, size=60).astype(np.uint32)
    kmax = int(g.degrees().max())
    k = 1 << int(np.ceil(np.log2(max(kmax, 1))))
    sched = oracle.Schedule([4, 16, 10**9], [1, 2, 8], 2)
    for mode in (oracle.MODE_LOUVAIN, oracle.MODE_LPA):
        a, ga = oracle.sweep(g, labels, mode, k=0)
        b, gb = oracle.sweep(g, labels, mode, k=k, sched=sched)
        assert a.tolist() == b.tolist()
        assert oracle.gains_as_ints(ga) == oracle.gains_as_ints(gb)


def test_sweep_invariants_sigma():
    """Sigma_c = sum of member K_i; sum_c Sigma_c = 2m; moves keep it."""
    g = gen.sbm(500, 10, 0.2, 0.01, wmax=4, seed=9)
    lab = np.arange(g.n, dtype=np.uint32)
    K = oracle.degrees(g)
    for _ in range(3):
        lab, _ = oracle.sweep(g, lab, oracle.MODE_LOUVAIN, k=8)
        Sig, size = oracle.community_totals(g.n, lab, K)
        assert int(Sig.sum()) == int(K.sum())
        assert int(size.sum()) == g.n
        for c in np.unique(lab)[:20]:
            assert int(Sig[c]) == int(K[lab == c].sum())


# ---- whole algorithms and aggregation -------------------------------------------------

def test_aggregate_preserves_weight_and_q():
    g = gen.sbm(400, 8, 0.2, 0.01, wmax=7, seed=5)
    rng = np.random.default_rng(1)
    lab = rng.integers(0, 30, size=g.n).astype(np.uint32)
    G2, dense = oracle.aggregate(g, lab)
    assert int(G2.w.astype(np.uint64).sum()) == int(g.w.astype(np.uint64).sum())
    assert oracle.modularity_fraction(G2, np.arange(G2.n)) == oracle.modularity_fraction(g, lab)
    # K of a super-vertex = Sigma of its community
    K2 = oracle.degrees(G2)
    K = oracle.degrees(g)
    for c in range(G2.n):
        assert int(K2[c]) == int(K[dense == c].sum())


@pytest.mark.parametrize("seed", range(6))
def test_louvain_below_brute_force_optimum(seed):
    g = gen.random_graph(8, 14, 4, seed=500 + seed)
    if g.nnz == 0:
        return
    qstar, _ = oracle.brute_force_best(g)
    for k in (0, 2, 8):
        lab = oracle.louvain_seq(g, k=k, tol=0.0)
        q = oracle.modularity_fraction(g, lab)
        assert q <= qstar


def test_louvain_two_triangles_optimum():
    g, t = two_triangles()
    qstar, _ = oracle.brute_force_best(g)
    assert qstar == Fraction(*t["q_optimum"])
    for k in (0, 8):
        lab = oracle.louvain_seq(g, k=k, tol=0.0)
        assert oracle.modularity_fraction(g, lab) == qstar


def test_louvain_recovers_disjoint_cliques():
    # ring of 6 cliques of size 5, joined by single edges
    src, dst = [], []
    for c in range(6):
        base = 5 * c
        for a, b in itertools.combinations(range(5), 2):
            src.append(base + a)
            dst.append(base + b)
        src.append(base)
        dst.append((base + 5 + 1) % 30)
    g = gen.from_edges(30, src, dst, [1] * len(src))
    for k in (0, 8):
        lab = oracle.louvain_seq(g, k=k, tol=0.0)
        assert len(np.unique(lab)) == 6
        for c in range(6):
            assert len(np.unique(lab[5 * c:5 * c + 5])) == 1


def test_louvain_quality_against_networkx():
    """On the 10k planted-partition SBM (half of the edges cross blocks, so
    the planted partition's Q ~ 0.49 is above what greedy Louvain reaches),
    the exact sequential Louvain must land near networkx's Louvain."""
    nx = pytest.importorskip("networkx")
    g = gen.sbm_10k(1)
    planted = (np.arange(g.n) // 100).astype(np.uint32)
    assert 0.45 < oracle.modularity(g, planted) < 0.53
    G = nx.Graph()
    G.add_nodes_from(range(g.n))
    r = np.repeat(np.arange(g.n), np.diff(g.offsets))
    m = r < g.cols
    G.add_weighted_edges_from(zip(r[m].tolist(), g.cols[m].tolist(), g.w[m].tolist()))
    qnx = np.mean([nx.community.modularity(G, nx.community.louvain_communities(
        G, weight="weight", seed=s, threshold=1e-7)) for s in range(2)])
    q = oracle.modularity(g, oracle.louvain_seq(g, k=0, tol=1e-4))
    assert q > qnx - 0.03
    q8 = oracle.modularity(g, oracle.louvain_seq(g, k=8, tol=1e-4))
    assert 0.8 * q < q8 <= q + 0.01


def test_lpa_converges_on_cliques():
    src, dst = [], []
    for c in range(4):
        for a, b in itertools.combinations(range(6), 2):
            src.append(6 * c + a)
            dst.append(6 * c + b)
    w = [3] * len(src)
    src += [0, 6, 12]
    dst += [6, 12, 18]
    g = gen.from_edges(24, src, dst, w + [1, 1, 1])
    lab = oracle.lpa_seq(g, k=8, tol=0.0)
    assert len(np.unique(lab)) == 4


def lpa_one_scan_case():
    t = load("lpa_one_scan.json")
    e = np.array(t["edges"])
    return gen.from_edges(t["n"], e[:, 0], e[:, 1], e[:, 2]), t


@pytest.mark.parametrize("sched", ["single", "default"])
def test_lpa_one_scan_hand_worked(sched):
    """LPA 1-scan (Section 4.3) against a sweep worked by hand on two stars
    whose 2-slot sketches are lossy: the 1-scan choice differs from the
    2-scan one for both centres, one of them because K_{i->d} comes from the
    sketch (a zeroed slot), not from a second scan."""
    g, t = lpa_one_scan_case()
    s = (oracle.Schedule.single_stream() if sched == "single"
         else oracle.Schedule([2, 4, 8, 16, 32, 64, 128, 256, 512, 1024, 2048, 4096, 16384, 2**62],
                              [1, 1, 1, 1, 1, 1, 1, 2, 4, 4, 8, 8, 32, 256], 4))
    lab = np.array(t["labels_in"], dtype=np.uint32)
    for row, key in ((0, "sketch_row0"), (6, "sketch_row6")):
        keys, vals = oracle.row_sketch(g, row, lab, t["k"], s)
        assert keys.tolist() == t[key]["keys"] and vals.tolist() == t[key]["vals"]
    for one, lk, gk in ((False, "two_scan_labels", "two_scan_gains"), (True, "one_scan_labels", "one_scan_gains")):
        out, gains = oracle.sweep(g, lab, oracle.MODE_LPA, k=t["k"], uncond=t["subtract"], sched=s, one_scan=one)
        assert out.tolist() == t[lk]
        assert oracle.gains_as_ints(gains) == t[gk]


def _lowbias32(x: int) -> int:
    x &= 0xFFFFFFFF
    x ^= x >> 16
    x = (x * 0x7FEB352D) & 0xFFFFFFFF
    x ^= x >> 15
    x = (x * 0x846CA68B) & 0xFFFFFFFF
    x ^= x >> 16
    return x


def test_color_classes_follow_lowbias32():
    n, P = 5000, 8
    c = oracle.color_classes(n, P)
    assert [int(v) for v in c[:300]] == [_lowbias32(i) % P for i in range(300)]
    assert int(c[4999]) == _lowbias32(4999) % P
    counts = np.bincount(c, minlength=P)
    assert counts.min() > 0.8 * n / P
    assert np.all(oracle.color_classes(10, 1) == 0)


@pytest.mark.parametrize("colors", [1, 2, 8])
def test_sync_louvain_invariants(colors):
    g = gen.sbm(600, 12, 0.15, 0.005, wmax=5, seed=6)
    lab = oracle.louvain_sync(g, k=8, colors=colors, threads=2)
    u = np.unique(lab)
    assert u[0] == 0 and u[-1] == len(u) - 1
    q = oracle.modularity_fraction(g, lab)
    assert Fraction(-1, 2) <= q <= 1
    # colour classes tame synchronous oscillation: at least as good as P=1
    if colors == 8:
        q1 = oracle.modularity_fraction(g, oracle.louvain_sync(g, k=8, colors=1, threads=2))
        assert q >= q1 - Fraction(1, 100)


def test_sync_louvain_below_brute_force():
    for seed in range(4):
        g = gen.random_graph(8, 14, 4, seed=700 + seed)
        if g.nnz == 0:
            continue
        qstar, _ = oracle.brute_force_best(g)
        for colors in (1, 8):
            lab = oracle.louvain_sync(g, k=8, colors=colors, tol=0.0)
            assert oracle.modularity_fraction(g, lab) <= qstar


def _components_ok(g, lab):
    """Every label class induces a connected subgraph (BFS)."""
    from collections import deque
    for c in np.unique(lab):
        mem = np.nonzero(lab == c)[0]
        ms = set(mem.tolist())
        seen = {int(mem[0])}
        q = deque([int(mem[0])])
        while q:
            u = q.popleft()
            for e in range(g.offsets[u], g.offsets[u + 1]):
                v = int(g.cols[e])
                if v in ms and v not in seen:
                    seen.add(v)
                    q.append(v)
        if len(seen) != len(mem):
            return False
    return True


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("k", [0, 8])
def test_refinement_nested_and_connected(seed, k):
    """Leiden refinement (Section 3.4): every refined sub-community lies inside
    one community of the bound and is connected (Section 5.1.4: no internally
    disconnected communities); only singletons moved."""
    g = gen.sbm(400, 8, 0.08, 0.01, wmax=6, seed=seed)
    bound = oracle.louvain_sync(g, k=k, max_passes=1, threads=2)
    ref = oracle.refine_sync(g, bound, k=k, threads=2)
    for c in np.unique(ref):
        assert len(np.unique(bound[ref == c])) == 1
    assert _components_ok(g, ref)
    # refinement merges something on a community-rich graph
    assert len(np.unique(ref)) < g.n


def test_refinement_needs_two_colours():
    """With one colour class every singleton target is barred: nothing moves."""
    g = gen.sbm(200, 4, 0.2, 0.01, seed=3)
    bound = oracle.louvain_sync(g, k=8, max_passes=1)
    ref = oracle.refine_sync(g, bound, k=8, colors=1)
    assert np.array_equal(ref, np.arange(g.n))


def test_leiden_quality_and_bounds():
    g = gen.sbm_10k(1)
    q_lei = oracle.modularity(g, oracle.leiden_sync(g, k=0, threads=4))
    q_lou = oracle.modularity(g, oracle.louvain_sync(g, k=0, threads=4))
    assert q_lei >= q_lou - 0.01
    for seed in range(3):
        t = gen.random_graph(8, 14, 4, seed=800 + seed)
        if t.nnz:
            qstar, _ = oracle.brute_force_best(t)
            assert oracle.modularity_fraction(t, oracle.leiden_sync(t, k=8, tol=0.0)) <= qstar


@pytest.mark.parametrize("seed", range(5))
def test_mg_aggregation_pins(seed):
    """MG aggregation (Section 4.1, Fig. 3): equals the exact super-graph when
    every community links to at most k communities; otherwise its weights
    never exceed the exact ones (clamped subtraction only lowers values) and
    the symmetric (Leiden) form is symmetric."""
    g = gen.sbm(600, 12, 0.2, 0.01, wmax=7, seed=seed)
    coarse = (np.arange(g.n) // 100).astype(np.uint32)       # 6 communities
    exact, _ = oracle.aggregate(g, coarse)
    mg, _ = oracle.aggregate_mg(g, coarse, k=8)
    assert np.array_equal(exact.offsets, mg.offsets) and np.array_equal(exact.cols, mg.cols)
    assert np.array_equal(exact.w, mg.w)
    fine = (np.arange(g.n) // 10).astype(np.uint32)          # 60 communities
    exact, _ = oracle.aggregate(g, fine)
    ex = {(r, int(exact.cols[e])): int(exact.w[e]) for r in range(exact.n)
          for e in range(exact.offsets[r], exact.offsets[r + 1])}
    for sym in (False, True):
        mg, _ = oracle.aggregate_mg(g, fine, k=4, symmetric=sym)
        got = {(r, int(mg.cols[e])): int(mg.w[e]) for r in range(mg.n)
               for e in range(mg.offsets[r], mg.offsets[r + 1])}
        for key, val in got.items():
            assert 0 < val <= ex[key]
        if sym:
            assert all(got.get((b, a)) == v for (a, b), v in got.items())
        else:
            assert all(mg.offsets[r + 1] - mg.offsets[r] <= 4 for r in range(mg.n))


# ---- learned skip proposal: the network's oracle ----------------------------------

def _rand_model(seed):
    from oracle import mlp
    rng = np.random.default_rng(seed)
    return (mlp.to_half(rng.normal(0, 0.5, (32, 8))), rng.normal(0, 0.1, 32),
            mlp.to_half(rng.normal(0, 0.3, 32)), float(rng.normal()))


def test_mlp_forward_hand_value():
    """One hidden unit active: z = w2 * relu(W1 x + b1) + b2 by hand."""
    from oracle import mlp
    W1 = np.zeros((32, 8)); W1[0, 0] = 2.0; W1[1, 1] = -1.0
    b1 = np.zeros(32); b1[0] = 0.5
    w2 = np.zeros(32); w2[0] = 3.0; w2[1] = 5.0
    x = np.array([[1.0, 2.0, 0, 0, 0, 0, 0, 1.0]])
    p, z, h = mlp.forward(x, W1, b1, w2, -1.0)
    assert h[0, 0] == 2.5 and h[0, 1] == 0.0
    assert z[0] == 3.0 * 2.5 - 1.0
    assert abs(p[0] - 1 / (1 + np.exp(-6.5))) < 1e-15


@pytest.mark.parametrize("seed", range(3))
def test_mlp_gradient_finite_differences(seed):
    """The analytic gradient of the mean binary cross-entropy matches central
    differences of the loss in float64."""
    from oracle import mlp
    rng = np.random.default_rng(seed)
    W1, b1, w2, b2 = _rand_model(seed)
    x = rng.random((50, 8))
    y = (rng.random(50) < 0.3).astype(np.float64)
    dW1, db1, dw2, db2 = mlp.gradients(x, y, W1, b1, w2, b2)
    eps = 1e-6
    for (j, q) in [(0, 0), (3, 5), (31, 7), (10, 2)]:
        Wp, Wm = W1.copy(), W1.copy()
        Wp[j, q] += eps; Wm[j, q] -= eps
        num = (mlp.loss(x, y, Wp, b1, w2, b2) - mlp.loss(x, y, Wm, b1, w2, b2)) / (2 * eps)
        assert abs(num - dW1[j, q]) < 1e-7 + 1e-5 * abs(num)
    for j in (0, 17, 31):
        bp, bm = b1.copy(), b1.copy(); bp[j] += eps; bm[j] -= eps
        num = (mlp.loss(x, y, W1, bp, w2, b2) - mlp.loss(x, y, W1, bm, w2, b2)) / (2 * eps)
        assert abs(num - db1[j]) < 1e-7 + 1e-5 * abs(num)
        wp, wm = w2.copy(), w2.copy(); wp[j] += eps; wm[j] -= eps
        num = (mlp.loss(x, y, W1, b1, wp, b2) - mlp.loss(x, y, W1, b1, wm, b2)) / (2 * eps)
        assert abs(num - dw2[j]) < 1e-7 + 1e-5 * abs(num)
    num = (mlp.loss(x, y, W1, b1, w2, b2 + eps) - mlp.loss(x, y, W1, b1, w2, b2 - eps)) / (2 * eps)
    assert abs(num - db2) < 1e-7 + 1e-5 * abs(num)


def test_mlp_features_definition():
    from oracle import mlp
    x = mlp.features(deg=[0, 3, 255], K=[0, 6, 1000], size_d=[1, 4, 1], sigma_d=[0, 12, 1000], two_m=4000,
                     moved_last=[1, 0, 1], since_move=[0, 3, 20], attach=[0.0, 0.25, 1.0])
    assert x[1, 0] == 2.0 / 16 and x[2, 0] == 8.0 / 16
    assert x[:, 1].tolist() == [1, 0, 1] and x[:, 2].tolist() == [0, 3 / 8, 1]
    assert x[1, 3] == np.log2(5) / 24 and x[1, 4] == np.sqrt(12 / 4000) and x[1, 5] == 0.5
    assert x[:, 6].tolist() == [0.0, 0.25, 1.0] and np.all(x[:, 7] == 1.0) and x[0, 5] == 0.0


def test_adam_two_steps_by_hand():
    """Adam (Kingma and Ba 2015, Algorithm 1) on one parameter, worked with
    fractions: theta0 = 1, lr = 0.1, g1 = 1/2, g2 = -1/4.  Step 1: m = 1/20,
    v = 1/4000, m_hat = 1/2, v_hat = 1/4, theta1 = 1 - 0.1 (1/2) / (1/2 + 1e-8).
    Step 2: m = 9/10 * 1/20 - 1/40 = 1/50, v = 999/1000 * 1/4000 + 1/16000 =
    1249/4000000, m_hat = (1/50) / (19/100) = 2/19, v_hat = (1249/4000000) /
    (1999/1000000) = 1249/7996, theta2 = theta1 - 0.1 (2/19) / (sqrt(1249/7996)
    + 1e-8)."""
    from oracle import mlp
    p1, m1, m2 = mlp.adam_step([1.0], [0.5], [0.0], [0.0], 1, 0.1)
    assert m1[0] == pytest.approx(1 / 20, rel=1e-15) and m2[0] == pytest.approx(1 / 4000, rel=1e-12)
    assert p1[0] == pytest.approx(1 - 0.1 * 0.5 / (0.5 + 1e-8), rel=1e-15)
    assert abs(p1[0] - 0.900000002) < 1e-15
    p2, m1, m2 = mlp.adam_step(p1, [-0.25], m1, m2, 2, 0.1)
    assert m1[0] == pytest.approx(1 / 50, rel=1e-12) and m2[0] == pytest.approx(1249 / 4000000, rel=1e-12)
    assert abs(p2[0] - 0.8733662987078462) < 1e-12


@pytest.mark.parametrize("seed", range(3))
def test_adam_step_size_and_scale_invariance(seed):
    """Two properties the Adam paper states (Section 2.1): the first step
    moves every parameter by lr in the direction against its gradient
    (m_hat / sqrt(v_hat) = sign(g) at t = 1, up to eps), and the update is
    invariant to a rescaling of the gradients (exactly so with eps = 0)."""
    from oracle import mlp
    rng = np.random.default_rng(seed)
    th = rng.normal(size=20)
    g = rng.normal(size=20) * 10.0 ** rng.uniform(-3, 2, 20)
    p1, _, _ = mlp.adam_step(th, g, np.zeros(20), np.zeros(20), 1, 0.01)
    assert np.allclose(p1 - th, -0.01 * np.sign(g), rtol=1e-5, atol=0)
    p, m1, m2 = th, np.zeros(20), np.zeros(20)
    q, n1, n2 = th, np.zeros(20), np.zeros(20)
    for t in range(1, 6):
        gt = rng.normal(size=20)
        p, m1, m2 = mlp.adam_step(p, gt, m1, m2, t, 0.01, eps=0.0)
        q, n1, n2 = mlp.adam_step(q, 37.5 * gt, n1, n2, t, 0.01, eps=0.0)
        assert np.allclose(p, q, rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("seed", range(8))
@pytest.mark.parametrize("mode", [oracle.MODE_LOUVAIN, oracle.MODE_LPA])
def test_sequential_exact_sweep_is_locally_optimal(seed, mode):
    """The sequential exact local-moving phase (k = 0, run until a sweep moves
    nobody) ends in a state where no single move helps: Louvain, every move
    of a vertex to a neighbouring community leaves Q unchanged or lower (exact
    rationals, Eq. 1); LPA, every vertex's label has the largest linking
    weight among its neighbouring communities (or ties it).  The synchronous
    exact sweep (a separately written candidate scan) then moves nobody."""
    rng = np.random.default_rng(700 + seed)
    n = int(rng.integers(6, 30))
    g = gen.random_graph(n, int(rng.integers(n, 4 * n)), 9, seed=700 + seed, self_loops=bool(seed % 2))
    lab, _ = oracle.local_move_seq(g, np.arange(n, dtype=np.uint32), mode, 0, False, 0.0, 500)
    # ... the phase stopped because a sweep moved nobody
    again, _ = oracle.local_move_seq(g, lab, mode, 0, False, 0.0, 1)
    assert np.array_equal(again, lab)
    q0 = oracle.modularity_fraction(g, lab)
    for i in range(n):
        nb = {int(lab[int(j)]) for j in g.cols[g.offsets[i]:g.offsets[i + 1]] if int(j) != i}
        link = {}
        for e in range(g.offsets[i], g.offsets[i + 1]):
            j = int(g.cols[e])
            if j != i:
                link[int(lab[j])] = link.get(int(lab[j]), 0) + int(g.w[e])
        for c in nb - {int(lab[i])}:
            if mode == oracle.MODE_LOUVAIN:
                moved = lab.copy()
                moved[i] = c
                assert oracle.modularity_fraction(g, moved) <= q0
            else:
                assert link[c] <= link.get(int(lab[i]), 0)
    out, _ = oracle.sweep(g, lab, mode, 0)
    assert np.array_equal(out, lab)
