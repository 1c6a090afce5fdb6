"""Batched Louvain (cd_louvain_batched): a batch of graphs of uneven size is
detected as one padded disjoint union, and every graph of the batch gets
exactly the labels, modularity and sweep count of cd_louvain on that graph
alone (same parameters) -- MG sketches (the union keeps each graph's stream
partition), the exact hashtable (including rows too long for shared
memory), CUDA-graph replay on and off, host and device inputs, degenerate
graphs (no vertices, no edges).  Every graph of the batch is also compared
with the oracle's Louvain of the same schedule (oracle.louvain_sync), so that a
mistake shared by the single and the batched paths cannot pass."""
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


def empty_graph(n):
    return gen.Graph(n, np.zeros(n + 1, dtype=np.int64), np.zeros(0, dtype=np.int32), np.zeros(0, dtype=np.uint32),
                     f"empty{n}")


@pytest.fixture(scope="module")
def graphs():
    gs = gen.sbm_batch(18, seed=3, n_range=(100, 6000), k_range=(4, 200))
    gs.insert(3, gen.rmat(14, 16, wmax=16, seed=9))       # hubs: rows longer than 2048
    gs.insert(7, empty_graph(0))
    gs.insert(8, empty_graph(6))
    gs.append(gen.grid(40, 40, 0.02, 16, seed=2))
    gs.append(gen.sbm_10k(1))
    return gs


def single_runs(cd, dev, params):
    import torch
    out = []
    for G in dev:
        lab, q = cd.cd_louvain(G, params, labels_out=torch.empty(max(G.n, 1), dtype=torch.int32, device="cuda"))
        out.append((lab[:G.n].cpu().numpy().view(np.uint32).copy(), q, cd.cd_last_stats().sweeps))
    return out


def check_equal(cd, graphs, labs, q, sw, ref):
    for i, g in enumerate(graphs):
        l1, q1, s1 = ref[i]
        got = labs[i]
        got = got.cpu().numpy() if hasattr(got, "cpu") else np.asarray(got)
        got = got.view(np.uint32)
        assert np.array_equal(got, l1), f"graph {i} ({g.name}): labels differ"
        assert q[i] == q1, f"graph {i} ({g.name}): Q {q[i]} != {q1}"
        assert sw[i] == s1, f"graph {i} ({g.name}): sweeps {sw[i]} != {s1}"


@pytest.mark.parametrize("k", [8, 0, 4, 16])
def test_batched_equals_single_runs(env, graphs, k):
    cd, torch = env
    dev = [cd.Graph.to_device(g) for g in graphs]
    ref = single_runs(cd, dev, cd.make_params(k=k))
    launches = []
    for capture in (True, False):
        labs, q, sw = cd.cd_louvain_batched(dev, cd.make_params(k=k, capture=capture))
        check_equal(cd, graphs, labs, q, sw, ref)
        launches.append(cd.cd_last_stats().kernel_launches)
    st = cd.cd_last_stats()
    assert st.passes >= 2 and st.sweeps >= max(r[2] for r in ref) // 2
    # a graph replay counts the kernels recorded in it: the same total as launching them
    assert launches[0] == launches[1] > 0


@pytest.mark.parametrize("k", [8, 0, 16])
def test_batched_equals_oracle(env, graphs, k):
    """Every graph of the batch against the CPU oracle's Louvain (same
    default schedule, 8 colour classes): bit-exact labels and the modularity
    of those labels to 1e-15."""
    cd, torch = env
    dev = [cd.Graph.to_device(g) for g in graphs]
    labs, q, _ = cd.cd_louvain_batched(dev, cd.make_params(k=k))
    sched = oracle.Schedule(*cd.cd_default_schedule(k).as_lists())
    for i, g in enumerate(graphs):
        got = labs[i].cpu().numpy().view(np.uint32) if g.n else np.zeros(0, np.uint32)
        ref = oracle.louvain_sync(g, k=k, sched=sched, threads=8)
        assert np.array_equal(got, ref), f"graph {i} ({g.name}): labels differ from the oracle"
        qr = float(oracle.modularity_fraction(g, ref)) if g.nnz else 0.0
        assert q[i] == pytest.approx(qr, abs=1e-15), f"graph {i} ({g.name})"


@pytest.mark.parametrize("opts", [dict(max_passes=1), dict(max_sweeps=2), dict(colors=1),
                                  dict(tolerance=0.0, max_sweeps=50), dict(subtract=1), dict(agg_k=4)])
def test_batched_stopping_rules_per_graph(env, graphs, opts):
    cd, torch = env
    sel = graphs[:8] + graphs[-2:]
    dev = [cd.Graph.to_device(g) for g in sel]
    p = cd.make_params(k=8, **opts)
    ref = single_runs(cd, dev, p)
    labs, q, sw = cd.cd_louvain_batched(dev, p)
    check_equal(cd, sel, labs, q, sw, ref)


def test_batched_host_inputs(env, graphs):
    cd, torch = env
    sel = graphs[:6]
    host = [cd.Graph.host(g) for g in sel]
    p = cd.make_params(k=8)
    ref = single_runs(cd, [cd.Graph.to_device(g) for g in sel], p)
    labs, q, sw = cd.cd_louvain_batched(host, p)
    check_equal(cd, sel, labs, q, sw, ref)


def test_batched_rejects_bad_input(env, graphs):
    cd, torch = env
    dev = [cd.Graph.to_device(g) for g in graphs[:3]]
    mixed = dev[:2] + [cd.Graph.host(graphs[2])]
    with pytest.raises(cd.CDError):
        cd.cd_louvain_batched(mixed, cd.make_params(k=8))
    with pytest.raises(cd.CDError):
        cd.cd_louvain_batched(dev, cd.make_params(k=8, skip_rule=2))
    # a column outside its own graph is reported, not silently remapped
    g = graphs[0]
    bad_cols = g.cols.copy()
    bad_cols[5] = g.n + 3
    bad = cd.Graph(g.n, torch.from_numpy(g.offsets).cuda(), torch.from_numpy(bad_cols).cuda(),
                   torch.from_numpy(g.w.view(np.int32)).cuda())
    with pytest.raises(cd.CDError) as e:
        cd.cd_louvain_batched([dev[1], bad], cd.make_params(k=8))
    assert e.value.code == cd.CD_EINVAL


def test_autotune_picks_valid_schedule_and_k(env, graphs):
    """The tuner returns a valid schedule (the library accepts it), one of the
    candidate k, a tuned sweep no slower than the default schedule's by more
    than timing noise, and a batched run with its choice that keeps the mean
    modularity within the tolerance of the best candidate."""
    cd, torch = env
    dev = [cd.Graph.to_device(g) for g in graphs]
    sched, k, rep = cd.cd_autotune(dev, cd.make_params(k=8), ks=(4, 8, 16), q_tol=0.005)
    assert k in (4, 8, 16) and 0 <= rep.chosen < 3 and rep.trials > 10
    # thresholds ascending, launch shape valid
    dm = list(sched.deg_max[:sched.nbuckets])
    assert all(a < b for a, b in zip(dm, dm[1:])) and sched.blocks_per_sm in (0, 2, 4)
    assert rep.sweep_ms[0] <= rep.default_ms * 1.10
    qbest = max(rep.q_mean[:3])
    assert rep.q_mean[rep.chosen] >= qbest - 0.005 * abs(qbest)
    labs, q, sw = cd.cd_louvain_batched(dev, cd.make_params(k=k, schedule=sched))
    assert abs(float(np.mean(q)) - rep.q_mean[rep.chosen]) < 1e-12
    # and the tuned run is still per-graph identical to single runs with that schedule
    ref = single_runs(cd, dev[:6], cd.make_params(k=k, schedule=sched))
    check_equal(cd, graphs[:6], labs[:6], q[:6], sw[:6], ref)
