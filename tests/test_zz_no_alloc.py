"""cd_modularity_noalloc: the modularity entry point for callers that cannot
allocate device memory (its scratch is a fixed array inside the library).

Checked through the C ABI against cd_modularity on two calls in a row with
different graphs and labels (the shared array keeps the previous call's
contents, so the second call also checks that it is cleared), plus the size
limit.  Kept in its own file, collected last."""
import numpy as np
import pytest

import oracle
from paper_2411_02268_gb300 import gen

pytestmark = pytest.mark.gpu

MAX_N = 1 << 20


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2411_02268_gb300 import _build
    _build.build()
    from paper_2411_02268_gb300 import cd
    return cd, torch


def test_noalloc_matches_cd_modularity_twice(env):
    cd, torch = env
    cases = [
        (gen.rmat(14, 16, wmax=16, seed=5), np.random.default_rng(1).integers(0, 500, 1 << 14)),
        (gen.sbm(3000, 30, 0.1, 0.002, wmax=9, seed=2), np.arange(3000) // 100),
    ]
    for g, lab in cases:
        G = cd.Graph.to_device(g)
        dlab = torch.from_numpy(lab.astype(np.uint32).view(np.int32)).cuda()
        q_ref, parts_ref = cd.cd_modularity(G, dlab)
        launches_ref = cd.cd_last_stats().kernel_launches
        q, parts = cd.cd_modularity_noalloc(G, dlab)
        st = cd.cd_last_stats()
        assert parts == parts_ref
        assert q == pytest.approx(q_ref, abs=1e-15)
        # and directly against the CPU oracle's integer parts of Eq. 1
        assert parts == oracle.modularity_parts(g, lab.astype(np.uint32))
        # the call's own statistics, not the previous call's
        assert st.modularity == q
        # the same kernels as cd_modularity, counted for this call alone
        assert st.kernel_launches == launches_ref > 0 and st.scratch_bytes == 0


def test_noalloc_size_limit_and_memory_kind(env):
    cd, torch = env
    n = MAX_N + 1
    big = cd.Graph(n, torch.zeros(n + 1, dtype=torch.int64, device="cuda"),
                   torch.zeros(0, dtype=torch.int32, device="cuda"),
                   torch.zeros(0, dtype=torch.int32, device="cuda"))
    with pytest.raises(cd.CDError) as ei:
        cd.cd_modularity_noalloc(big, torch.zeros(n, dtype=torch.int32, device="cuda"))
    assert ei.value.code == cd.CD_ESIZE
    g = gen.sbm(100, 4, 0.2, 0.02, seed=1)
    with pytest.raises(cd.CDError) as ei:
        cd.cd_modularity_noalloc(cd.Graph.host(g), np.zeros(100, np.uint32))
    assert ei.value.code == cd.CD_EINVAL
