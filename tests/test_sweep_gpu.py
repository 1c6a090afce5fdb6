"""Parity of the CUDA sweep (through the C ABI) with the CPU oracle.

One synchronous sweep from fixed labels must agree with the oracle element by
element: every output label, the mover count and the 128-bit gain sum, for
every sketch size, subtraction rule, mode, stream schedule (all lane counts
1..256), on ragged graphs, hubs, self-loops, isolated vertices and the
degenerate sizes.  All arithmetic is integer, so the bar is bit-exact.
"""
import numpy as np
import pytest

import oracle
from paper_2411_02268_gb300 import gen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2411_02268_gb300 import _build
    _build.build()
    from paper_2411_02268_gb300 import cd
    return cd, torch


ALL_LANES = ([2, 4, 6, 8, 12, 16, 24, 32, 2**62], [1, 2, 4, 8, 16, 32, 64, 128, 256])
WIDE = ([2**62], [256])
MID = ([3, 40, 2**62], [1, 32, 64])


def sched_for(cd, k, deg, lanes):
    """A test schedule with the kernel's chunk width (the default's vec)."""
    return cd.schedule_from(deg, lanes, cd.cd_default_schedule(k).vec)


def oracle_sched(cd, sched):
    deg, lanes, vec = sched.as_lists()
    return oracle.Schedule(deg, lanes, vec)


def gpu_sweep(cd, torch, g, labels, mode, k, uncond=0, sched=None, active=None, host=False):
    p = cd.make_params(k=k, subtract=uncond, schedule=sched)
    if host:
        G = cd.Graph.host(g)
        out, moved, gain = cd.cd_sweep(G, p, mode, np.ascontiguousarray(labels, dtype=np.uint32),
                                       active=None if active is None else np.ascontiguousarray(active, np.uint8))
        return np.asarray(out, dtype=np.uint32), moved, gain
    G = cd.Graph.to_device(g)
    lab = torch.from_numpy(np.ascontiguousarray(labels, dtype=np.uint32).view(np.int32)).cuda()
    act = None if active is None else torch.from_numpy(np.ascontiguousarray(active, np.uint8)).cuda()
    p.stream = torch.cuda.current_stream().cuda_stream
    out, moved, gain = cd.cd_sweep(G, p, mode, lab, active=act)
    return out.cpu().numpy().view(np.uint32), moved, gain


def oracle_sweep(cd, g, labels, mode, k, uncond=0, sched=None, active=None):
    sch = oracle_sched(cd, sched if sched is not None else cd.cd_default_schedule(k))
    out, gains = oracle.sweep(g, labels, mode, k, int(uncond), sch, active=active, threads=4)
    moved = int(np.count_nonzero(out != np.asarray(labels, dtype=np.uint32)))
    return out, moved, oracle.gain_total(gains)


def check(cd, torch, g, labels, mode, k, uncond=0, sched=None, active=None, host=False):
    a = gpu_sweep(cd, torch, g, labels, mode, k, uncond, sched, active, host)
    b = oracle_sweep(cd, g, labels, mode, k, uncond, sched, active)
    bad = np.nonzero(a[0] != b[0])[0]
    assert len(bad) == 0, f"{len(bad)} labels differ, first at {bad[:5]}: gpu {a[0][bad[:5]]} oracle {b[0][bad[:5]]}"
    assert a[1] == b[1]
    assert a[2] == b[2]
    return a


def label_states(g, seed):
    rng = np.random.default_rng(seed)
    n = g.n
    yield "singletons", np.arange(n, dtype=np.uint32)
    yield "random", rng.integers(0, max(1, n // 7), size=n).astype(np.uint32)
    lab, _ = oracle.sweep(g, np.arange(n, dtype=np.uint32), oracle.MODE_LOUVAIN, 0)
    yield "after_one_sweep", lab


GRAPHS = {
    "sbm10k": lambda: gen.sbm_10k(1),
    "rmat12_w16": lambda: gen.rmat(12, 16, wmax=16, seed=2),
    "rmat11_w255_perm": lambda: gen.rmat(11, 16, wmax=255, seed=3, permute=True),
    "ragged_loops": lambda: gen.random_graph(301, 2500, 9, seed=5, self_loops=True),
    "grid_rewired": lambda: gen.grid(40, 50, 0.05, 16, seed=4),
}


@pytest.mark.parametrize("gname", list(GRAPHS))
@pytest.mark.parametrize("k", [8, 1, 2, 4, 16])
def test_mg_louvain_default_schedule(env, gname, k):
    cd, torch = env
    g = GRAPHS[gname]()
    for _, lab in label_states(g, 1):
        check(cd, torch, g, lab, oracle.MODE_LOUVAIN, k)


@pytest.mark.parametrize("gname", ["rmat12_w16", "ragged_loops", "sbm10k"])
@pytest.mark.parametrize("sched_name", ["all_lanes", "wide", "mid"])
@pytest.mark.parametrize("k", [1, 2, 4, 8, 16])
def test_mg_all_stream_schedules(env, gname, sched_name, k):
    cd, torch = env
    g = GRAPHS[gname]()
    deg, lanes = {"all_lanes": ALL_LANES, "wide": WIDE, "mid": MID}[sched_name]
    s = sched_for(cd, k, deg, lanes)
    for _, lab in label_states(g, 2):
        check(cd, torch, g, lab, oracle.MODE_LOUVAIN, k, sched=s)
        check(cd, torch, g, lab, oracle.MODE_LPA, k, sched=s)


@pytest.mark.parametrize("gname", list(GRAPHS))
@pytest.mark.parametrize("k", [8, 2])
def test_mg_lpa_and_unconditional(env, gname, k):
    cd, torch = env
    g = GRAPHS[gname]()
    s = sched_for(cd, k, *ALL_LANES)
    for _, lab in label_states(g, 3):
        check(cd, torch, g, lab, oracle.MODE_LPA, k)
        check(cd, torch, g, lab, oracle.MODE_LOUVAIN, k, uncond=1)
        check(cd, torch, g, lab, oracle.MODE_LPA, k, uncond=1, sched=s)
        # the weighted Misra-Gries of the literature (subtract = 2)
        check(cd, torch, g, lab, oracle.MODE_LOUVAIN, k, uncond=2)
        check(cd, torch, g, lab, oracle.MODE_LPA, k, uncond=2, sched=s)


@pytest.mark.parametrize("gname", list(GRAPHS))
def test_exact_hashtable(env, gname):
    cd, torch = env
    g = GRAPHS[gname]()
    for _, lab in label_states(g, 4):
        check(cd, torch, g, lab, oracle.MODE_LOUVAIN, 0)
        check(cd, torch, g, lab, oracle.MODE_LPA, 0)


def test_exact_hub_rows_use_global_tables(env):
    """Rows longer than 2048 entries take tables in device scratch."""
    cd, torch = env
    n = 6000
    src = np.concatenate([np.zeros(5000, np.int64), np.arange(1, 3000)])
    dst = np.concatenate([np.arange(1, 5001), np.arange(2, 3001)])
    w = (np.arange(len(src)) % 13 + 1).astype(np.uint64)
    g = gen.from_edges(n, src, dst, w)
    assert g.degrees().max() > 4096
    rng = np.random.default_rng(0)
    for lab in (np.arange(n, dtype=np.uint32), rng.integers(0, 50, n).astype(np.uint32)):
        check(cd, torch, g, lab, oracle.MODE_LOUVAIN, 0)
        check(cd, torch, g, lab, oracle.MODE_LPA, 0)
        check(cd, torch, g, lab, oracle.MODE_LOUVAIN, 8)
    stats = cd.cd_last_stats()
    assert stats.scratch_bytes > 0


def test_active_mask(env):
    cd, torch = env
    g = GRAPHS["rmat12_w16"]()
    rng = np.random.default_rng(7)
    act = (rng.random(g.n) < 0.4).astype(np.uint8)
    for _, lab in label_states(g, 5):
        check(cd, torch, g, lab, oracle.MODE_LOUVAIN, 8, active=act)
        check(cd, torch, g, lab, oracle.MODE_LOUVAIN, 0, active=act)


def test_host_memory_matches_device(env):
    cd, torch = env
    g = GRAPHS["sbm10k"]()
    lab = np.arange(g.n, dtype=np.uint32)
    a = gpu_sweep(cd, torch, g, lab, oracle.MODE_LOUVAIN, 8, host=True)
    b = gpu_sweep(cd, torch, g, lab, oracle.MODE_LOUVAIN, 8, host=False)
    assert np.array_equal(a[0], b[0]) and a[1:] == b[1:]
    check(cd, torch, g, lab, oracle.MODE_LPA, 8, host=True)


def test_sweep_counts_its_kernel_launches(env):
    """One sweep from singletons on a small graph launches seven kernels: the
    bucketing (count, single-block scan, scatter, starts), row sums, totals and
    the sweep."""
    cd, torch = env
    g = GRAPHS["sbm10k"]()
    gpu_sweep(cd, torch, g, np.arange(g.n, dtype=np.uint32), oracle.MODE_LOUVAIN, 8)
    assert cd.cd_last_stats().kernel_launches == 7


def test_wide_sketch_values(env):
    """Weighted degrees above 2^32 switch the sketch to 64-bit values."""
    cd, torch = env
    big = 2**31 + 7
    src = [0, 0, 0, 1, 2, 3, 4, 4]
    dst = [1, 2, 3, 2, 3, 5, 5, 6]
    w = [big, big, big, 3, big - 5, 9, big, 1]
    g = gen.from_edges(7, src, dst, w)
    for lab in (np.arange(7, dtype=np.uint32), np.array([0, 1, 1, 3, 4, 4, 6], np.uint32)):
        for k in (1, 2, 8):
            check(cd, torch, g, lab, oracle.MODE_LOUVAIN, k)
            check(cd, torch, g, lab, oracle.MODE_LPA, k)
        check(cd, torch, g, lab, oracle.MODE_LOUVAIN, 0)


def test_degenerate_graphs(env):
    cd, torch = env
    empty_edges = gen.from_edges(5, [], [], [])
    check(cd, torch, empty_edges, np.arange(5, dtype=np.uint32), oracle.MODE_LOUVAIN, 8)
    one = gen.from_edges(1, [0], [0], [3])       # a single self-loop
    check(cd, torch, one, np.zeros(1, np.uint32), oracle.MODE_LOUVAIN, 8)
    check(cd, torch, one, np.zeros(1, np.uint32), oracle.MODE_LOUVAIN, 0)
    pair = gen.from_edges(2, [0], [1], [5])
    check(cd, torch, pair, np.arange(2, dtype=np.uint32), oracle.MODE_LOUVAIN, 8)
    check(cd, torch, pair, np.arange(2, dtype=np.uint32), oracle.MODE_LPA, 8)
    # n = 0 through the host path
    from paper_2411_02268_gb300 import cd as cdm
    G0 = cdm.Graph(0, np.zeros(1, np.int64), np.zeros(0, np.int32), np.zeros(0, np.uint32))
    out, moved, gain = cdm.cd_sweep(G0, cdm.make_params(k=8), 0, np.zeros(0, np.uint32))
    assert moved == 0 and gain == 0


def test_two_triangles_golden(env):
    import json, os
    cd, torch = env
    t = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "two_triangles.json")))
    e = np.array(t["edges"])
    g = gen.from_edges(t["n"], e[:, 0], e[:, 1], np.ones(len(e)))
    for k in (0, 8):
        out, moved, gain = gpu_sweep(cd, torch, g, np.arange(6, dtype=np.uint32), oracle.MODE_LOUVAIN, k)
        assert out.tolist() == t["sweep1_labels"]
        assert gain == sum(t["sweep1_gains"])


def test_device_detects_bad_columns(env):
    """A column out of range in a device graph is reported, not read."""
    cd, torch = env
    g = gen.sbm(200, 4, 0.2, 0.02, seed=3)
    g.cols[17] = 10_000
    G = cd.Graph.to_device(g)
    lab = torch.arange(g.n, dtype=torch.int32, device="cuda")
    with pytest.raises(cd.CDError) as ei:
        cd.cd_sweep(G, cd.make_params(k=8), 0, lab)
    assert ei.value.code == cd.CD_EINVAL


@pytest.mark.parametrize("mutate", ["col", "w"])
@pytest.mark.parametrize("host", [False, True])
def test_bad_columns_and_weights_rejected(env, mutate, host):
    cd, torch = env
    g = gen.sbm(300, 5, 0.2, 0.02, seed=2)
    if mutate == "col":
        g.cols[3] = 300
    else:
        g.w[5] = 0
    G = cd.Graph.host(g) if host else cd.Graph.to_device(g)
    lab = np.arange(g.n, dtype=np.uint32)
    lab = lab if host else torch.from_numpy(lab.view(np.int32)).cuda()
    for k in (8, 0):
        with pytest.raises(cd.CDError) as ei:
            cd.cd_sweep(G, cd.make_params(k=k), 0, lab)
        assert ei.value.code == cd.CD_EINVAL
    with pytest.raises(cd.CDError):
        cd.cd_louvain(G, cd.make_params(k=8))


@pytest.mark.parametrize("seed", range(3))
def test_modularity_parity(env, seed):
    cd, torch = env
    g = gen.rmat(12, 16, wmax=16, seed=seed + 10)
    rng = np.random.default_rng(seed)
    for lab in (np.arange(g.n, dtype=np.uint32), rng.integers(0, 30, g.n).astype(np.uint32),
                np.zeros(g.n, np.uint32)):
        G = cd.Graph.to_device(g)
        q, parts = cd.cd_modularity(G, torch.from_numpy(lab.view(np.int32)).cuda())
        sin_, sq, tm = oracle.modularity_parts(g, lab)
        assert parts == (sin_, sq, tm)
        assert abs(q - float(oracle.modularity_fraction(g, lab))) <= 1e-15
        qh, parts_h = cd.cd_modularity(cd.Graph.host(g), lab)
        assert parts_h == parts


def test_repeatable(env):
    cd, torch = env
    g = GRAPHS["rmat12_w16"]()
    lab = np.arange(g.n, dtype=np.uint32)
    a = gpu_sweep(cd, torch, g, lab, oracle.MODE_LOUVAIN, 8)
    b = gpu_sweep(cd, torch, g, lab, oracle.MODE_LOUVAIN, 8)
    assert np.array_equal(a[0], b[0]) and a[1:] == b[1:]


@pytest.mark.parametrize("gname", ["sbm10k", "rmat12_w16", "ragged_loops", "grid_rewired"])
@pytest.mark.parametrize("k", [8, 16, 0, 64])
def test_refine_sub_sweep_parity(env, gname, k):
    """One refine-mode sub-sweep (Leiden, Section 3.4): bound filter, the
    singleton-only rule and the same-colour singleton bar, per colour class,
    from singletons and from a partly merged state."""
    cd, torch = env
    g = GRAPHS[gname]()
    colors = 8
    col = oracle.color_classes(g.n, colors)
    bound = oracle.louvain_sync(g, k=8, max_passes=1, threads=4)
    sched = cd.cd_default_schedule(k)
    osched = oracle_sched(cd, sched)
    states = [np.arange(g.n, dtype=np.uint32),
              oracle.sweep(g, np.arange(g.n, dtype=np.uint32), oracle.MODE_REFINE, 8, False, osched,
                           active=(col == 0).astype(np.uint8), bound=bound, colors=colors, sub_color=0)[0]]
    for lab in states:
        for p in (0, 3, 7):
            act = (col == p).astype(np.uint8)
            params = cd.make_params(k=k, colors=colors, sub_color=p, stream=torch.cuda.current_stream().cuda_stream)
            G = cd.Graph.to_device(g)
            out, moved, gain = cd.cd_sweep(G, params, cd.MODE_REFINE,
                                           torch.from_numpy(lab.view(np.int32)).cuda(),
                                           active=torch.from_numpy(act).cuda(),
                                           bound=torch.from_numpy(bound.view(np.int32)).cuda())
            ref, gains = oracle.sweep(g, lab, oracle.MODE_REFINE, k, False, osched, active=act, bound=bound,
                                      threads=4, colors=colors, sub_color=p)
            got = out.cpu().numpy().view(np.uint32)
            assert np.array_equal(got, ref)
            assert moved == int(np.count_nonzero(ref != lab))
            assert gain == oracle.gain_total(gains)


@pytest.mark.parametrize("gname", list(GRAPHS))
@pytest.mark.parametrize("k", [1, 8, 32])
def test_lpa_one_scan_parity(env, gname, k):
    """LPA 1-scan (Section 4.3): decisions on the sketch values alone."""
    cd, torch = env
    g = GRAPHS[gname]()
    osched = oracle_sched(cd, cd.cd_default_schedule(k))
    for _, lab in label_states(g, 9):
        G = cd.Graph.to_device(g)
        p = cd.make_params(k=k, one_scan=True)
        out, moved, gain = cd.cd_sweep(G, p, cd.MODE_LPA, torch.from_numpy(lab.view(np.int32)).cuda())
        ref, gains = oracle.sweep(g, lab, oracle.MODE_LPA, k, False, osched, threads=4, one_scan=True)
        assert np.array_equal(out.cpu().numpy().view(np.uint32), ref)
        assert gain == oracle.gain_total(gains)


def test_lpa_one_scan_golden(env):
    """The hand-worked two-star LPA sweep (k = 2) with and without 1-scan."""
    import json, os
    cd, torch = env
    t = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "lpa_one_scan.json")))
    e = np.array(t["edges"])
    g = gen.from_edges(t["n"], e[:, 0], e[:, 1], e[:, 2])
    lab = torch.from_numpy(np.array(t["labels_in"], dtype=np.int32)).cuda()
    G = cd.Graph.to_device(g)
    for one, lk, gk in ((False, "two_scan_labels", "two_scan_gains"), (True, "one_scan_labels", "one_scan_gains")):
        out, moved, gain = cd.cd_sweep(G, cd.make_params(k=t["k"], one_scan=one), cd.MODE_LPA, lab)
        assert out.cpu().numpy().tolist() == t[lk]
        assert moved == sum(1 for x in t[gk] if x > 0)
        assert gain == sum(t[gk])


# ---- large sketches (k = 32, 64: the paper's Leiden uses 64 slots) --------------------
# These merge inside one warp, so their schedules give a row at most 32 streams.
BIG_LANES = ([1, 2, 4, 8, 16, 40, 2**62], [1, 2, 4, 8, 16, 32, 32])
BIG_NARROW = ([2**62], [8])


@pytest.mark.parametrize("gname", list(GRAPHS))
@pytest.mark.parametrize("k", [32, 64])
def test_large_sketch_default_schedule(env, gname, k):
    cd, torch = env
    g = GRAPHS[gname]()
    assert max(cd.cd_default_schedule(k).as_lists()[1]) <= 32
    for _, lab in label_states(g, 6):
        check(cd, torch, g, lab, oracle.MODE_LOUVAIN, k)
        check(cd, torch, g, lab, oracle.MODE_LPA, k)


@pytest.mark.parametrize("gname", ["rmat12_w16", "ragged_loops", "sbm10k", "rmat11_w255_perm"])
@pytest.mark.parametrize("sched_name", ["big_lanes", "narrow"])
@pytest.mark.parametrize("k", [32, 64])
def test_large_sketch_stream_schedules(env, gname, sched_name, k):
    cd, torch = env
    g = GRAPHS[gname]()
    s = sched_for(cd, k, *{"big_lanes": BIG_LANES, "narrow": BIG_NARROW}[sched_name])
    for _, lab in label_states(g, 7):
        check(cd, torch, g, lab, oracle.MODE_LOUVAIN, k, sched=s)
        check(cd, torch, g, lab, oracle.MODE_LOUVAIN, k, uncond=1, sched=s)
        check(cd, torch, g, lab, oracle.MODE_LPA, k, sched=s)


@pytest.mark.parametrize("k", [32, 64])
def test_large_sketch_wide_values(env, k):
    """Rows whose weighted degree needs 64-bit sketch values."""
    cd, torch = env
    base = gen.rmat(10, 16, wmax=16, seed=8)
    w = (base.w.astype(np.uint64) * (2**27)).astype(np.uint32)  # up to 2^31
    g = gen.Graph(base.n, base.offsets, base.cols, w, "rmat10_heavy")
    assert int(np.max(np.add.reduceat(g.w.astype(np.uint64), g.offsets[:-1][np.diff(g.offsets) > 0]))) >= 2**32
    for _, lab in label_states(g, 8):
        check(cd, torch, g, lab, oracle.MODE_LOUVAIN, k)
        check(cd, torch, g, lab, oracle.MODE_LPA, k)


def test_textbook_summary_limits(env):
    """subtract = 2 is compiled for k <= 8 sweeps only: larger k and MG
    aggregation are refused."""
    cd, torch = env
    g = GRAPHS["sbm10k"]()
    for kw in (dict(k=16, subtract=2), dict(k=64, subtract=2), dict(k=8, subtract=2, agg_k=4)):
        with pytest.raises(cd.CDError) as e:
            cd.cd_louvain(cd.Graph.to_device(g), cd.make_params(**kw))
        assert e.value.code == cd.CD_EINVAL


def test_large_sketch_rejects_wide_streams(env):
    cd, torch = env
    g = GRAPHS["rmat12_w16"]()
    s = sched_for(cd, 64, *WIDE)
    with pytest.raises(cd.CDError):
        gpu_sweep(cd, torch, g, np.arange(g.n, dtype=np.uint32), oracle.MODE_LOUVAIN, 64, sched=s)


def test_modularity_rejects_offsets_short_of_the_entries(env):
    """Device offsets that end before the last entry are reported (the warp
    walk over the entries stops instead of reading past the offsets)."""
    cd, torch = env
    g = GRAPHS["rmat12_w16"]()
    off = g.offsets.copy()
    off[-1] -= 5  # the last row ends 5 entries early
    bad = cd.Graph(g.n, torch.from_numpy(off).cuda(), torch.from_numpy(g.cols).cuda(),
                   torch.from_numpy(g.w.view(np.int32)).cuda())
    lab = torch.arange(g.n, dtype=torch.int32, device="cuda")
    with pytest.raises(cd.CDError) as e:
        cd.cd_modularity(bad, lab)
    assert e.value.code == cd.CD_EINVAL
    # and the well-formed graph still gives the oracle's parts afterwards
    q, parts = cd.cd_modularity(cd.Graph.to_device(g), lab)
    assert parts == oracle.modularity_parts(g, np.arange(g.n, dtype=np.uint32))


@pytest.mark.parametrize("k", [8, 16, 64])
def test_candidate_count_matches_oracle(env, k):
    """cd_stats.candidates (the benchmark's count of Sigma_c gathers) equals
    the number of live sketch slots other than the vertex's own community,
    summed over the vertices that decide, with the oracle's sketches."""
    cd, torch = env
    g = gen.rmat(11, 16, wmax=16, seed=7)
    osched = oracle_sched(cd, cd.cd_default_schedule(k))
    deg = g.degrees()
    for _, lab in label_states(g, 5):
        G = cd.Graph.to_device(g)
        cd.cd_sweep(G, cd.make_params(k=k), cd.MODE_LOUVAIN, torch.from_numpy(lab.view(np.int32)).cuda())
        got = cd.cd_last_stats().candidates
        want = 0
        for i in np.nonzero(deg)[0]:
            keys, vals = oracle.row_sketch(g, int(i), lab, k, osched)
            want += int(np.count_nonzero((vals > 0) & (keys != lab[i])))
        assert got == want


@pytest.mark.parametrize("k", [8, 16, 64])
@pytest.mark.parametrize("bpsm", [1, 4])
def test_resident_grid_same_results(env, k, bpsm):
    """A schedule's blocks_per_sm only changes the launch shape (a resident
    grid striding over the virtual blocks): every sweep result is the
    oracle's, as with one block per virtual block."""
    cd, torch = env
    for gname in ("rmat12_w16", "sbm10k"):
        g = GRAPHS[gname]()
        deg, lanes, vec = cd.cd_default_schedule(k).as_lists()
        s = cd.schedule_from(deg, lanes, vec, blocks_per_sm=bpsm)
        for _, lab in label_states(g, 6):
            check(cd, torch, g, lab, oracle.MODE_LOUVAIN, k, sched=s)
