"""The C ABI boundary on the CPU: the library builds for sm_103a, loads, and
exports every entry point include/cd.h declares; the ctypes structures match
the C layout; argument checks answer without touching a GPU."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "cd.h")


@pytest.fixture(scope="module")
def cd():
    from paper_2411_02268_gb300 import _build
    _build.build()
    from paper_2411_02268_gb300 import cd as cdmod
    return cdmod


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(cd_[a-z_]+)\s*\(", text)))


def test_header_symbols_exported(cd):
    names = declared_functions()
    assert len(names) >= 9
    out = subprocess.run(["nm", "-D", "--defined-only", cd.SO], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (cd_[a-z_]+)\b", out))
    for name in names:
        assert name in exported, name
        assert hasattr(cd.lib(), name)
    assert set(cd.SYMBOLS) == set(names)


def test_struct_layout_matches_header(cd, tmp_path):
    src = tmp_path / "layout.c"
    src.write_text(r'''
#include <stdio.h>
#include <stddef.h>
#include "cd.h"
int main(void) {
  printf("csr %zu %zu %zu\n", sizeof(cd_csr), offsetof(cd_csr, weights), offsetof(cd_csr, memory));
  printf("sched %zu %zu %zu %zu\n", sizeof(cd_schedule), offsetof(cd_schedule, deg_max), offsetof(cd_schedule, lanes), offsetof(cd_schedule, blocks_per_sm));
  printf("params %zu %zu %zu %zu %zu %zu %zu\n", sizeof(cd_params), offsetof(cd_params, sched), offsetof(cd_params, stream), offsetof(cd_params, timing), offsetof(cd_params, colors), offsetof(cd_params, one_scan), offsetof(cd_params, capture));
  printf("stats %zu %zu %zu %zu %zu %zu %zu\n", sizeof(cd_stats), offsetof(cd_stats, sweep_kernel_ms), offsetof(cd_stats, entries_scanned), offsetof(cd_stats, cuda_error), offsetof(cd_stats, kernel_launches), offsetof(cd_stats, candidates), offsetof(cd_stats, phase_ms));
  printf("mlp %zu %zu\n", sizeof(cd_mlp), offsetof(cd_mlp, b2));
  printf("parts %zu\n", sizeof(cd_modularity_parts));
  printf("tune %zu %zu %zu %zu\n", sizeof(cd_tune_report), offsetof(cd_tune_report, q_mean), offsetof(cd_tune_report, trials), offsetof(cd_tune_report, chosen));
  return 0;
}''')
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    C = ctypes
    exp = [
        f"csr {C.sizeof(cd.CSR)} {cd.CSR.weights.offset} {cd.CSR.memory.offset}",
        f"sched {C.sizeof(cd.Schedule)} {cd.Schedule.deg_max.offset} {cd.Schedule.lanes.offset} {cd.Schedule.blocks_per_sm.offset}",
        f"params {C.sizeof(cd.Params)} {cd.Params.sched.offset} {cd.Params.stream.offset} {cd.Params.timing.offset} {cd.Params.colors.offset} {cd.Params.one_scan.offset} {cd.Params.capture.offset}",
        f"stats {C.sizeof(cd.Stats)} {cd.Stats.sweep_kernel_ms.offset} {cd.Stats.entries_scanned.offset} {cd.Stats.cuda_error.offset} {cd.Stats.kernel_launches.offset} {cd.Stats.candidates.offset} {cd.Stats.phase_ms.offset}",
        f"mlp {C.sizeof(cd.MLP)} {cd.MLP.b2.offset}",
        f"parts {C.sizeof(cd.ModularityParts)}",
        f"tune {C.sizeof(cd.TuneReport)} {cd.TuneReport.q_mean.offset} {cd.TuneReport.trials.offset} {cd.TuneReport.chosen.offset}",
    ]
    assert got[:7] == exp


def test_strerror_and_default_schedule(cd):
    assert cd.cd_strerror(0) == "ok"
    assert cd.cd_strerror(cd.CD_EINVAL) == "invalid argument"
    s = cd.cd_default_schedule(8)
    deg, lanes, vec = s.as_lists()
    assert vec == 4 and len(deg) == len(lanes) >= 2
    assert all(b > a for a, b in zip(deg, deg[1:]))
    assert all(l & (l - 1) == 0 and 1 <= l <= 256 for l in lanes)


def test_argument_checks_without_gpu(cd):
    """Rejected before any CUDA call: bad k, bad subtract flag, bad schedule,
    bad graph header, aliasing labels, unknown mode."""
    from paper_2411_02268_gb300 import gen
    g = gen.sbm(50, 5, 0.3, 0.05, seed=1)
    G = cd.Graph.host(g)
    lab = np.arange(g.n, dtype=np.uint32)
    out = np.empty_like(lab)

    def rc(params, mode=0, li=lab, lo=out, graph=G):
        csr = graph.csr()
        return cd.lib().cd_sweep(ctypes.byref(csr), ctypes.byref(params), mode, li.ctypes.data, None, None,
                                 lo.ctypes.data, None, None)

    assert rc(cd.make_params(k=3)) == cd.CD_EINVAL
    assert rc(cd.make_params(k=128)) == cd.CD_EINVAL
    assert rc(cd.make_params(k=64, schedule=cd.schedule_from([10**9], [64]))) == cd.CD_EINVAL  # > 32 streams
    assert rc(cd.make_params(k=8, subtract=3)) == cd.CD_EINVAL
    assert rc(cd.make_params(k=8), mode=7) == cd.CD_EINVAL
    assert rc(cd.make_params(k=8), lo=lab) == cd.CD_EINVAL
    assert rc(cd.make_params(k=8, one_scan=True), mode=cd.MODE_LOUVAIN) == cd.CD_EINVAL
    assert rc(cd.make_params(k=0, one_scan=True), mode=cd.MODE_LPA) == cd.CD_EINVAL
    assert rc(cd.make_params(k=8), mode=cd.MODE_REFINE) == cd.CD_EINVAL   # refine needs a bound
    assert rc(cd.make_params(k=8, colors=0, sub_color=1)) == cd.CD_EINVAL  # one class in Louvain mode
    assert rc(cd.make_params(k=8, colors=4, sub_color=4)) == cd.CD_EINVAL
    assert rc(cd.make_params(k=8, colors=17)) == cd.CD_EINVAL
    assert rc(cd.make_params(k=16, subtract=2)) == cd.CD_EINVAL           # textbook summary: k <= 8
    assert rc(cd.make_params(k=8, agg_k=3)) == cd.CD_EINVAL
    assert rc(cd.make_params(k=8, skip_rule=1)) == cd.CD_EINVAL           # the learned rule needs a model
    assert rc(cd.make_params(k=8, schedule=cd.schedule_from([10**9], [8], blocks_per_sm=9))) == cd.CD_EINVAL
    bad_sched = cd.schedule_from([4, 2], [1, 2])
    assert rc(cd.make_params(k=8, schedule=bad_sched)) == cd.CD_EINVAL
    bad_sched = cd.schedule_from([4, 10**9], [1, 3])
    assert rc(cd.make_params(k=8, schedule=bad_sched)) == cd.CD_EINVAL
    # host graph with broken offsets (columns and weights are checked on the device)
    for mutate in ("order", "end"):
        g2 = gen.sbm(50, 5, 0.3, 0.05, seed=1)
        if mutate == "order":
            g2.offsets[10] = g2.offsets[11] + 1
        else:
            g2.offsets[-1] += 1
        assert rc(cd.make_params(k=8), graph=cd.Graph.host(g2)) == cd.CD_EINVAL
    # labels out of range (host)
    lab2 = lab.copy()
    lab2[0] = 50
    assert rc(cd.make_params(k=8), li=lab2) == cd.CD_EINVAL
    # null graph
    p = cd.make_params(k=8)
    assert cd.lib().cd_sweep(None, ctypes.byref(p), 0, lab.ctypes.data, None, None, out.ctypes.data,
                             None, None) == cd.CD_EINVAL


def test_product_path_fails_loudly_without_library(tmp_path, monkeypatch):
    from paper_2411_02268_gb300 import cd as cdmod
    monkeypatch.setattr(cdmod, "SO", str(tmp_path / "missing.so"))
    monkeypatch.setattr(cdmod, "_lib", None)
    with pytest.raises(RuntimeError, match="missing"):
        cdmod.lib()


def test_bench_schedule_literal_matches_library(cd):
    """bench.py's oracle legs use a written-out copy of the default schedule
    (so that they never load the CUDA library); it must be the library's."""
    import bench
    for k in (0, 1, 2, 4, 8, 16, 32, 64):
        assert tuple(bench.default_schedule(k)) == tuple(cd.cd_default_schedule(k).as_lists()), k


def test_injected_allocation_failure_without_gpu(cd, monkeypatch):
    """CD_FAIL_ALLOC=1 fails the first scratch allocation of a call on the
    host, before any device request: cd_sweep and cd_louvain on host graphs
    return CD_ENOMEM (this runs without a GPU)."""
    from paper_2411_02268_gb300 import gen
    g = gen.sbm(200, 4, 0.2, 0.02, seed=1)
    G = cd.Graph.host(g)
    lab = np.arange(g.n, dtype=np.uint32)
    monkeypatch.setenv("CD_FAIL_ALLOC", "1")
    for fn in (lambda: cd.cd_sweep(G, cd.make_params(k=8), cd.MODE_LOUVAIN, lab),
               lambda: cd.cd_louvain(G, cd.make_params(k=8))):
        with pytest.raises(cd.CDError) as e:
            fn()
        assert e.value.code == cd.CD_ENOMEM
        assert cd.cd_last_stats().cuda_error == b"injected allocation failure"
