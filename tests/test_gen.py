"""Input generators: determinism, CSR well-formedness, workload shapes."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_2411_02268_gb300 import gen

GOLD = os.path.join(os.path.dirname(__file__), "golden", "gen_checksums.json")


def check_csr(g, self_loops=False):
    off, cols, w = g.offsets, g.cols, g.w
    assert off[0] == 0 and np.all(np.diff(off) >= 0) and off[-1] == len(cols) == len(w)
    assert cols.dtype == np.int32 and w.dtype == np.uint32
    if len(cols):
        assert cols.min() >= 0 and cols.max() < g.n and w.min() >= 1
    rows = np.repeat(np.arange(g.n), np.diff(off))
    # strictly ascending columns within each row
    same = rows[1:] == rows[:-1]
    assert np.all(cols[1:][same] > cols[:-1][same])
    if not self_loops:
        assert not np.any(rows == cols)
    # symmetric with equal weights
    a = np.lexsort((cols, rows))
    b = np.lexsort((rows, cols))
    assert np.array_equal(rows[a], cols[b]) and np.array_equal(cols[a], rows[b])
    assert np.array_equal(w[a], w[b])


def golden():
    with open(GOLD) as f:
        return json.load(f)


def test_checksums_match_golden():
    gd = golden()
    assert gen.checksum(gen.sbm_10k(1)) == gd["sbm_10k_seed1"]
    assert gen.checksum(gen.rmat(16, 16, wmax=16, seed=7)) == gd["rmat16_ef16_w16_seed7"]
    assert gen.checksum(gen.grid(64, 64, 0.02, 16, 3)) == gd["grid64x64_p0.02_w16_seed3"]


def test_thread_count_does_not_change_output():
    code = ("from paper_2411_02268_gb300 import gen;"
            "print(gen.checksum(gen.rmat(15, 8, wmax=9, seed=2)))")
    outs = set()
    for t in ("1", "3"):
        env = dict(os.environ, OMP_NUM_THREADS=t)
        r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                           cwd=os.path.dirname(os.path.dirname(__file__)), check=True)
        outs.add(r.stdout.strip())
    assert len(outs) == 1


def test_sbm_shape():
    g = gen.sbm_10k(1)
    check_csr(g)
    # E[undirected edges] = 100*C(100,2)*0.05 + (C(10^4,2) - 100*C(100,2))*0.0005 ~ 49.5k
    assert 47_000 < g.nnz // 2 < 52_000
    blk = np.arange(g.n) // 100
    rows = np.repeat(np.arange(g.n), g.degrees())
    inside = np.mean(blk[rows] == blk[g.cols])
    assert 0.45 < inside < 0.55
    assert np.all(g.w == 1)


def test_rmat_shape():
    g = gen.rmat(14, 16, wmax=16, seed=3)
    check_csr(g)
    assert g.n == 2**14 and g.nnz < 2 * 16 * 2**14
    d = g.degrees()
    assert d.max() > 20 * d.mean()          # heavy tail
    assert g.w.min() >= 1 and g.w.max() <= 16
    p = gen.rmat(12, 8, wmax=4, seed=3, permute=True)
    check_csr(p)


def test_grid_shape():
    g = gen.grid(32, 48, 0.02, 16, seed=5)
    check_csr(g)
    assert g.n == 32 * 48
    full = 32 * 47 + 31 * 48
    assert 0.97 * full <= g.nnz // 2 <= full
    g0 = gen.grid(8, 8, 0.0, 1, seed=1)
    assert g0.nnz == 2 * (8 * 7 * 2) and np.all(g0.degrees() >= 2) and g0.degrees().max() == 4


def test_from_edges_sums_duplicates_and_keeps_loops():
    g = gen.from_edges(4, [0, 1, 0, 2, 3], [1, 0, 1, 2, 0], [1, 2, 3, 4, 5])
    check_csr(g, self_loops=True)
    r = {(i, int(g.cols[e])): int(g.w[e]) for i in range(4) for e in range(g.offsets[i], g.offsets[i + 1])}
    assert r == {(0, 1): 6, (1, 0): 6, (2, 2): 4, (0, 3): 5, (3, 0): 5}


def test_det_log():
    for x in (1.0, 0.5, 0.1, 1e-9, 0.999999):
        assert abs(gen.det_log(x) - np.log(x)) <= 1e-14 * max(1, abs(np.log(x)))
