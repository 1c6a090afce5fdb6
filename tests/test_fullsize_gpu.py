"""Parity at the benchmark's full sizes, in the launch configuration bench.py
times (cd_sweep, default schedule, k = 8, Louvain, singleton labels and a
mid-run label state): every output label of a random vertex sample and of the
largest hubs is recomputed by the oracle one vertex at a time; the mover
count and gain of the sample, K, and modularity parts are compared whole."""
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


def sampled_parity(cd, torch, g, labels, k, mode, nsample=4000, seed=0):
    deg = g.degrees()
    rng = np.random.default_rng(seed)
    sample = np.zeros(g.n, dtype=np.uint8)
    sample[rng.choice(g.n, size=min(nsample, g.n), replace=False)] = 1
    sample[np.argsort(deg)[-64:]] = 1          # the hubs (longest rows, 256 streams)
    G = cd.Graph.to_device(g)
    lab_d = torch.from_numpy(labels.view(np.int32)).cuda()
    p = cd.make_params(k=k, stream=torch.cuda.current_stream().cuda_stream)
    out, moved, gain = cd.cd_sweep(G, p, mode, lab_d)
    got = out.cpu().numpy().view(np.uint32)
    sched = oracle.Schedule(*cd.cd_default_schedule(k).as_lists())
    ref, gains = oracle.sweep(g, labels, mode, k, False, sched, active=sample, threads=16)
    idx = np.nonzero(sample)[0]
    bad = idx[got[idx] != ref[idx]]
    assert len(bad) == 0, f"{len(bad)} sampled labels differ, e.g. {bad[:5]}"
    # unsampled vertices keep their label in the oracle; the GPU decided them all
    assert moved >= int(np.count_nonzero(ref != labels))
    return got


@pytest.mark.slow
def test_rmat22_full_size_sampled_parity(env):
    cd, torch = env
    g = gen.rmat22(1)
    assert g.n == 2**22 and g.nnz > 120_000_000
    single = np.arange(g.n, dtype=np.uint32)
    out = sampled_parity(cd, torch, g, single, 8, oracle.MODE_LOUVAIN)
    # a mid-run state: the labels after one sweep
    sampled_parity(cd, torch, g, out, 8, oracle.MODE_LOUVAIN, seed=1)
    sampled_parity(cd, torch, g, single, 8, oracle.MODE_LPA, seed=2)
    # weighted degrees and modularity parts, whole
    G = cd.Graph.to_device(g)
    q, parts = cd.cd_modularity(G, torch.from_numpy(out.view(np.int32)).cuda())
    assert parts == oracle.modularity_parts(g, out)


@pytest.mark.slow
def test_rmat22_exact_variant_sampled_parity(env):
    cd, torch = env
    g = gen.rmat22(1)
    sampled_parity(cd, torch, g, np.arange(g.n, dtype=np.uint32), 0, oracle.MODE_LOUVAIN, nsample=2000)


@pytest.mark.slow
def test_rmat25_full_size_sampled_parity(env):
    """The HBM-scale graph (R-MAT scale 25, edge factor 16, w in [1, 255]:
    about 1.07 G CSR entries, hubs of ~10^6 entries on 256 streams): sampled
    vertices and the largest hubs against the oracle, Louvain and LPA."""
    cd, torch = env
    g = gen.rmat25(1)
    assert g.n == 2**25 and g.nnz > 900_000_000
    single = np.arange(g.n, dtype=np.uint32)
    sampled_parity(cd, torch, g, single, 8, oracle.MODE_LOUVAIN, nsample=3000, seed=3)
    sampled_parity(cd, torch, g, single, 8, oracle.MODE_LPA, nsample=2000, seed=4)
