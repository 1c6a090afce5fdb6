"""Host-side fault injection on the GPU path: every scratch allocation of a
call is failed in turn (CD_FAIL_ALLOC=n, checked on the host before the
device is asked), and the call must return CD_ENOMEM, release what it took
(no growth of the device memory in use over all the failing calls) and leave
the library in a state where the next call gives the same result as before.
No GPU fault is involved: the failure is made on the host."""
import numpy as np
import pytest

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


def _fail_each(cd, torch, monkeypatch, call, limit=400):
    """Runs call() with CD_FAIL_ALLOC = 1, 2, ... until it succeeds; returns
    the number of allocations the call makes."""
    for n in range(1, limit):
        monkeypatch.setenv("CD_FAIL_ALLOC", str(n))
        try:
            call()
        except cd.CDError as e:
            assert e.code == cd.CD_ENOMEM, (n, str(e))
            assert cd.cd_last_stats().cuda_error == b"injected allocation failure"
            continue
        finally:
            monkeypatch.delenv("CD_FAIL_ALLOC")
        return n - 1
    raise AssertionError("the call never succeeded")


@pytest.mark.parametrize("what", ["sweep_device", "sweep_host", "louvain", "leiden", "batched"])
def test_every_allocation_failure_is_reported_and_released(env, monkeypatch, what):
    cd, torch = env
    g = gen.rmat(16, 16, wmax=16, seed=2)
    G = cd.Graph.to_device(g)
    H = cd.Graph.host(g)
    lab_d = torch.arange(g.n, dtype=torch.int32, device="cuda")
    lab_h = np.arange(g.n, dtype=np.uint32)
    calls = {
        "sweep_device": lambda: cd.cd_sweep(G, cd.make_params(k=8), cd.MODE_LOUVAIN, lab_d)[0].cpu().numpy(),
        "sweep_host": lambda: np.asarray(cd.cd_sweep(H, cd.make_params(k=8), cd.MODE_LOUVAIN, lab_h)[0]).copy(),
        "louvain": lambda: cd.cd_louvain(G, cd.make_params(k=8))[0].cpu().numpy(),
        "leiden": lambda: cd.cd_leiden(G, cd.make_params(k=64))[0].cpu().numpy(),
        "batched": lambda: cd.cd_louvain_batched([G, G], cd.make_params(k=8))[0][1].cpu().numpy(),
    }
    call = calls[what]
    before = call()
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    n = _fail_each(cd, torch, monkeypatch, call)
    assert n >= 3
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    # every failing call released its scratch: the pool did not grow by the
    # scratch of the n failing calls (each holds tens of MB on this graph)
    assert free0 - free1 < 256 * 2**20, (free0, free1, n)
    assert np.array_equal(call(), before)
