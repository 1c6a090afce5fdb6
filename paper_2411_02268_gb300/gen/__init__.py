"""Seeded synthetic graph inputs (CSR), shared by the CUDA path and the oracle.

The generators live in ``graphgen.c`` (compiled with gcc on first use, or by
``__graft_entry__.build()``).  They hold no community-detection arithmetic:
they draw edges, symmetrise, drop self-loops and duplicates, sort each row and
attach integer weights ``w = 1 + H(seed, min(u,v), max(u,v)) mod wmax``.

Workload shapes (stand-ins for the paper's SuiteSparse graphs, Section 5.1.3,
which are not available here):

* ``sbm``  - planted-partition stochastic block model (community-rich, like
  the social graphs);
* ``rmat`` - R-MAT power-law graphs (heavy-tailed web/social degree mix);
* ``grid`` - 2-D grid with a fraction of edges rewired (road / k-mer shape).
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIBDIR = os.path.join(os.path.dirname(_HERE), "lib")
_SO = os.path.join(_LIBDIR, "libgraphgen.so")
_lock = threading.Lock()
_lib = None


class _CSR(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int64),
        ("nnz", ctypes.c_int64),
        ("offsets", ctypes.POINTER(ctypes.c_int64)),
        ("cols", ctypes.POINTER(ctypes.c_int32)),
        ("w", ctypes.POINTER(ctypes.c_uint32)),
    ]


def build(force: bool = False) -> str:
    """Compile graphgen.c into lib/libgraphgen.so (gcc, OpenMP when present)."""
    src = os.path.join(_HERE, "graphgen.c")
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(src):
        return _SO
    os.makedirs(_LIBDIR, exist_ok=True)
    tmp = _SO + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-std=c11", src, "-o", tmp]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_SO)
            P = ctypes.POINTER(_CSR)
            lib.gg_rmat.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                                    ctypes.c_double, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int, P]
            lib.gg_sbm.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                                   ctypes.c_uint32, ctypes.c_uint64, P]
            lib.gg_grid.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_double, ctypes.c_uint32,
                                    ctypes.c_uint64, P]
            lib.gg_free.argtypes = [P]
            lib.gg_checksum.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p,
                                        ctypes.c_void_p, ctypes.c_void_p]
            lib.gg_checksum.restype = ctypes.c_uint64
            lib.gg_rng.argtypes = [ctypes.c_uint64] * 4
            lib.gg_rng.restype = ctypes.c_uint64
            lib.gg_det_log.argtypes = [ctypes.c_double]
            lib.gg_det_log.restype = ctypes.c_double
            lib.gg_num_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


@dataclasses.dataclass
class Graph:
    """Undirected weighted graph in CSR form (both directions stored).

    offsets: int64[n+1]; cols: int32[nnz], each row ascending; w: uint32[nnz].
    """
    n: int
    offsets: np.ndarray
    cols: np.ndarray
    w: np.ndarray
    name: str = ""

    @property
    def nnz(self) -> int:
        return int(self.offsets[-1])

    def degrees(self) -> np.ndarray:
        return np.diff(self.offsets)


def _take(csr: _CSR, name: str) -> Graph:
    lib = _load()
    n, nnz = int(csr.n), int(csr.nnz)
    try:
        off = np.ctypeslib.as_array(csr.offsets, shape=(n + 1,)).copy()
        cols = np.ctypeslib.as_array(csr.cols, shape=(max(nnz, 1),))[:nnz].copy()
        w = np.ctypeslib.as_array(csr.w, shape=(max(nnz, 1),))[:nnz].copy()
    finally:
        lib.gg_free(ctypes.byref(csr))
    return Graph(n, off, cols, w, name)


def _check(rc: int, what: str):
    if rc != 0:
        raise RuntimeError(f"{what} failed with code {rc}")


def rmat(scale: int, edge_factor: int = 16, a: float = 0.57, b: float = 0.19, c: float = 0.19,
         wmax: int = 16, seed: int = 1, permute: bool = False) -> Graph:
    """R-MAT graph with 2**scale vertices and edge_factor * 2**scale drawn edges,
    symmetrised, deduplicated, self-loops removed, w uniform in [1, wmax]."""
    csr = _CSR()
    _check(_load().gg_rmat(scale, edge_factor, a, b, c, wmax, seed, int(permute), ctypes.byref(csr)),
           "gg_rmat")
    return _take(csr, f"rmat{scale}_ef{edge_factor}_w{wmax}_s{seed}" + ("_perm" if permute else ""))


def sbm(n: int, nblocks: int, p_in: float, p_out: float, wmax: int = 1, seed: int = 1) -> Graph:
    """Planted-partition SBM; block b = vertices [ceil(b n/B), ceil((b+1) n/B))."""
    csr = _CSR()
    _check(_load().gg_sbm(n, nblocks, p_in, p_out, wmax, seed, ctypes.byref(csr)), "gg_sbm")
    return _take(csr, f"sbm{n}_b{nblocks}_s{seed}")


def grid(rows: int, cols: int, p_rewire: float = 0.02, wmax: int = 16, seed: int = 1) -> Graph:
    """rows x cols 4-neighbour grid with each edge rewired with probability p."""
    csr = _CSR()
    _check(_load().gg_grid(rows, cols, p_rewire, wmax, seed, ctypes.byref(csr)), "gg_grid")
    return _take(csr, f"grid{rows}x{cols}_p{p_rewire}_s{seed}")


def from_edges(n: int, src, dst, w, name: str = "edges") -> Graph:
    """CSR from an undirected edge list.  Each pair {u, v} adds w to entries
    (u, v) and (v, u); a self-loop {u, u} adds w to the single entry (u, u);
    repeated pairs are summed.  Rows come out ascending by column."""
    src = np.asarray(src, dtype=np.int64)
    dst = np.asarray(dst, dtype=np.int64)
    w = np.asarray(w, dtype=np.uint64)
    loop = src == dst
    s = np.concatenate([src, dst[~loop]])
    d = np.concatenate([dst, src[~loop]])
    ww = np.concatenate([w, w[~loop]])
    key = s * n + d
    order = np.argsort(key, kind="stable")
    key, ww = key[order], ww[order]
    uniq, first = np.unique(key, return_index=True)
    sums = np.add.reduceat(ww, first) if len(ww) else ww
    rows = uniq // n
    cols = (uniq % n).astype(np.int32)
    counts = np.bincount(rows, minlength=n) if len(rows) else np.zeros(n, dtype=np.int64)
    off = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=off[1:])
    if len(sums) and int(sums.max()) >= 2**32:
        raise ValueError("edge weight sum does not fit uint32")
    return Graph(n, off, cols, sums.astype(np.uint32), name)


def random_graph(n: int, n_edges: int, wmax: int, seed: int, self_loops: bool = False) -> Graph:
    """Small uniform random multigraph (pairs drawn with the counter RNG, then
    summed), for parity tests on ragged shapes."""
    lib = _load()
    src = np.empty(n_edges, dtype=np.int64)
    dst = np.empty(n_edges, dtype=np.int64)
    wts = np.empty(n_edges, dtype=np.uint64)
    kept = 0
    for t in range(n_edges):
        u = lib.gg_rng(seed, 100, t, 0) % n
        v = lib.gg_rng(seed, 100, t, 1) % n
        if u == v and not self_loops:
            continue
        src[kept], dst[kept] = u, v
        wts[kept] = 1 + lib.gg_rng(seed, 101, t, 0) % wmax
        kept += 1
    return from_edges(n, src[:kept], dst[:kept], wts[:kept], name=f"rand{n}_{n_edges}_s{seed}")


def checksum(g: Graph) -> int:
    """64-bit checksum over (n, nnz, offsets, cols, w)."""
    off = np.ascontiguousarray(g.offsets, dtype=np.int64)
    cols = np.ascontiguousarray(g.cols, dtype=np.int32)
    w = np.ascontiguousarray(g.w, dtype=np.uint32)
    return int(_load().gg_checksum(g.n, g.nnz, off.ctypes.data, cols.ctypes.data, w.ctypes.data))


def rng(seed: int, stream: int, a: int, b: int) -> int:
    """The counter-based generator: splitmix64 chained over (seed, stream, a, b)."""
    return int(_load().gg_rng(seed, stream, a, b))


def det_log(x: float) -> float:
    return float(_load().gg_det_log(x))


def num_threads() -> int:
    return int(_load().gg_num_threads())


# ---- the named workloads ------------------------------------------------------

def sbm_10k(seed: int = 1) -> Graph:
    """Planted partition: 10,000 vertices in 100 equal blocks, p_in=0.05,
    p_out=0.0005, unit weights, no self-loops."""
    g = sbm(10_000, 100, 0.05, 0.0005, wmax=1, seed=seed)
    g.name = f"sbm10k_s{seed}"
    return g


def rmat22(seed: int = 1) -> Graph:
    """R-MAT scale 22, edge factor 16, (0.57, 0.19, 0.19, 0.05), w in [1, 16]."""
    return rmat(22, 16, 0.57, 0.19, 0.19, wmax=16, seed=seed)


def rmat25(seed: int = 1) -> Graph:
    """R-MAT scale 25, edge factor 16, (0.57, 0.19, 0.19, 0.05), w in [1, 255]."""
    return rmat(25, 16, 0.57, 0.19, 0.19, wmax=255, seed=seed)


def sbm_batch_params(count: int = 512, seed: int = 1, n_range=(1000, 200000), k_range=(10, 2000),
                     d_range=(8.0, 64.0), ratio: float = 10.0):
    """Parameters of a batch of planted-partition graphs of uneven size:
    n log-uniform in n_range, the community count log-uniform in k_range
    (at most n / 2), the average degree d uniform in d_range, and
    p_in = ratio * p_out with p_out = d / (ratio (s - 1) + (n - s)) for
    blocks of s = n / K vertices (so that the expected degree is d).
    Returns a list of (n, K, p_in, p_out, graph_seed)."""
    r = np.random.default_rng([int(seed), 0x5B1])
    out = []
    for g in range(count):
        n = int(round(np.exp(r.uniform(np.log(n_range[0]), np.log(n_range[1])))))
        K = int(round(np.exp(r.uniform(np.log(k_range[0]), np.log(k_range[1])))))
        K = max(1, min(K, n // 2))
        d = float(r.uniform(d_range[0], d_range[1]))
        s = n / K
        p_out = d / (ratio * (s - 1.0) + (n - s))
        p_in = min(1.0, ratio * p_out)
        out.append((n, K, p_in, p_out, (int(seed) << 20) + g))
    return out


def sbm_batch(count: int = 512, seed: int = 1, wmax: int = 16, **kw) -> list[Graph]:
    """A batch of planted-partition graphs (see sbm_batch_params), weights
    uniform in [1, wmax], graph g seeded by (seed, g)."""
    return [sbm(n, K, p_in, p_out, wmax, gs) for (n, K, p_in, p_out, gs) in sbm_batch_params(count, seed, **kw)]
