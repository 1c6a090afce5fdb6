"""CPU oracle for the MG-sketch local-moving sweep (arXiv 2411.02268).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` use it; the library never does.  It shares
no code with the CUDA path.  ``oracle.c`` holds the per-vertex arithmetic
(plain loops, single-threaded per call); this module wraps it with ctypes and
adds the steps that are plain array operations (renumbering and aggregation
by sort, Section 4.1 "aggregation phase"), the pass loops, and a brute-force
optimum for tiny graphs.

Parity status per function (what pins it, tests/test_oracle_pins.py):
  modularity      - Eq. 1; pinned by the textbook double sum, closed forms,
                    networkx, and its [-1/2, 1] range.
  sweep (exact)   - Eq. 2; pinned by exact recomputation of Q for every
                    candidate move and brute-force argmax.
  sketch_update   - Algorithm 1; pinned by hand-worked vectors
                    (tests/golden/sketch_vectors.json) and the textbook
                    Misra-Gries guarantee on unit weights.
  sketch merge / stream partition - no counterpart in the paper (it streams
                    each row on one thread): parity unpinned beyond the
                    exact-sum reduction when a row has <= k communities.
  aggregate       - pinned by weight conservation and Q(G', singletons) =
                    Q(G, C).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor
from fractions import Fraction

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIBDIR = os.path.join(_HERE, "lib")
_SO = os.path.join(_LIBDIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

MODE_LOUVAIN, MODE_LPA, MODE_REFINE = 0, 1, 2
EMPTY_KEY = 0xFFFFFFFF

_p = ctypes.c_void_p
_i64 = ctypes.c_int64


def build(force: bool = False) -> str:
    """Compile oracle.c into oracle/lib/liboracle.so with gcc."""
    src = os.path.join(_HERE, "oracle.c")
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(src):
        return _SO
    os.makedirs(_LIBDIR, exist_ok=True)
    tmp = _SO + f".tmp{os.getpid()}"
    subprocess.run(["gcc", "-O2", "-fPIC", "-shared", "-std=gnu11", src, "-o", tmp],
                   check=True, capture_output=True)
    os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_SO)
            lib.or_degrees.argtypes = [_i64, _p, _p, _p]
            lib.or_community_totals.argtypes = [_i64, _p, _p, _p, _p]
            lib.or_modularity_parts.argtypes = [_i64, _p, _p, _p, _p, _p, _p, _p, _p]
            lib.or_sketch_update.argtypes = [_p, _p, ctypes.c_int, ctypes.c_uint32, ctypes.c_uint64,
                                             ctypes.c_int]
            lib.or_sketch_merge.argtypes = [_p, _p, _p, _p, ctypes.c_int, ctypes.c_int]
            lib.or_sweep.argtypes = ([_i64, _p, _p, _p, _p, _p, _p, _p, ctypes.c_uint64, _p, _p,
                                      ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _p, _p,
                                      ctypes.c_int, _i64, _i64, _p, _p, _p, ctypes.c_int, ctypes.c_int,
                                      ctypes.c_int])
            lib.or_row_sketch.argtypes = [_i64, _p, _p, _p, _p, _p, ctypes.c_int, ctypes.c_int,
                                          ctypes.c_int, _p, _p, ctypes.c_int, _p, _p]
            lib.or_local_move_seq.argtypes = [_i64, _p, _p, _p, _p, ctypes.c_int, ctypes.c_int,
                                              ctypes.c_int, ctypes.c_double, ctypes.c_int]
            lib.or_local_move_seq.restype = ctypes.c_int
            lib.or_aggregate_mg_sketch.argtypes = [_i64, _p, _p, _p, _p, _i64, _p, _p, ctypes.c_int,
                                                   ctypes.c_int, ctypes.c_int, _p, _p, ctypes.c_int, _p, _p]
            _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data


def _csr(g):
    off = np.ascontiguousarray(g.offsets, dtype=np.int64)
    cols = np.ascontiguousarray(g.cols, dtype=np.int32)
    w = np.ascontiguousarray(g.w, dtype=np.uint32)
    return off, cols, w


# ---- Section 3 quantities ---------------------------------------------------

def degrees(g) -> np.ndarray:
    """K_i = sum of w over row i."""
    off, _, w = _csr(g)
    K = np.empty(g.n, dtype=np.uint64)
    _load().or_degrees(g.n, _ptr(off), _ptr(w), _ptr(K))
    return K


def community_totals(n: int, labels, K):
    """Sigma_c = sum of K_i over members, and community sizes."""
    labels = np.ascontiguousarray(labels, dtype=np.uint32)
    K = np.ascontiguousarray(K, dtype=np.uint64)
    Sig = np.empty(n, dtype=np.uint64)
    size = np.empty(n, dtype=np.uint32)
    _load().or_community_totals(n, _ptr(labels), _ptr(K), _ptr(Sig), _ptr(size))
    return Sig, size


def modularity_parts(g, labels):
    """(sum_c sigma_c, sum_c Sigma_c^2, 2m) as Python ints (Eq. 1)."""
    off, cols, w = _csr(g)
    labels = np.ascontiguousarray(labels, dtype=np.uint32)
    if g.n and labels.max(initial=0) >= g.n:
        raise ValueError("labels must be < n")
    out = [ctypes.c_uint64() for _ in range(4)]
    _load().or_modularity_parts(g.n, _ptr(off), _ptr(cols), _ptr(w), _ptr(labels),
                                *[ctypes.byref(o) for o in out])
    sin_, lo, hi, tm = (o.value for o in out)
    return sin_, lo | (hi << 64), tm


def modularity_fraction(g, labels) -> Fraction:
    """Q of Eq. 1 as an exact rational."""
    sin_, sq, tm = modularity_parts(g, labels)
    if tm == 0:
        return Fraction(0)
    return Fraction(tm * sin_ - sq, tm * tm)


def modularity(g, labels) -> float:
    return float(modularity_fraction(g, labels))


# ---- Algorithm 1 ---------------------------------------------------------------

def new_sketch(k: int):
    return np.full(k, EMPTY_KEY, dtype=np.uint32), np.zeros(k, dtype=np.uint64)


def sketch_update(keys, vals, c: int, w: int, uncond: int = 0):
    """One populateSketch update (in place) with community c and weight w."""
    assert keys.dtype == np.uint32 and vals.dtype == np.uint64 and keys.flags.c_contiguous
    _load().or_sketch_update(_ptr(keys), _ptr(vals), len(keys), c, w, int(uncond))


def sketch_merge(akeys, avals, bkeys, bvals, uncond: int = 0):
    _load().or_sketch_merge(_ptr(akeys), _ptr(avals), _ptr(bkeys), _ptr(bvals), len(akeys),
                            int(uncond))


def sketch_stream(stream, k: int, uncond: int = 0):
    """Sketch of a (community, weight) stream processed in order."""
    keys, vals = new_sketch(k)
    for c, w in stream:
        sketch_update(keys, vals, c, w, uncond)
    return keys, vals


# ---- schedules -------------------------------------------------------------------

class Schedule:
    """Streams per row by row length: bucket b takes rows with length
    <= deg_max[b] and splits them into lanes[b] streams; entry e of a row goes
    to stream (e // vec) % lanes."""

    def __init__(self, deg_max, lanes, vec=4):
        self.deg_max = np.ascontiguousarray(deg_max, dtype=np.int64)
        self.lanes = np.ascontiguousarray(lanes, dtype=np.int32)
        self.vec = int(vec)
        assert len(self.deg_max) == len(self.lanes) >= 1

    @staticmethod
    def single_stream():
        return Schedule([2**62], [1], 1)


def row_sketch(g, i: int, labels, k: int, sched: Schedule, uncond=False, bound=None):
    off, cols, w = _csr(g)
    labels = np.ascontiguousarray(labels, dtype=np.uint32)
    keys, vals = new_sketch(k)
    _load().or_row_sketch(i, _ptr(off), _ptr(cols), _ptr(w), _ptr(labels), _ptr(bound), k,
                          int(uncond), len(sched.lanes), _ptr(sched.deg_max), _ptr(sched.lanes),
                          sched.vec, _ptr(keys), _ptr(vals))
    return keys, vals


# ---- one synchronous sweep ----------------------------------------------------------

def sweep(g, labels, mode: int = MODE_LOUVAIN, k: int = 8, uncond: int = 0,
          sched: Schedule | None = None, active=None, bound=None, vertices=None,
          threads: int = 1, state=None, colors: int = 1, sub_color: int = 0, one_scan: bool = False):
    """One synchronous sweep from `labels` (see or_sweep in oracle.c).

    Returns (labels_out, gains) where gains is an object array of Python ints
    (the chosen scaled gain of each mover, 0 for the others).  With
    `vertices=(v0, v1)` only that range is decided (others keep their
    label).  `threads` > 1 splits the range over host threads (each thread
    runs the single-threaded C loop on its own sub-range).
    `state` may pass precomputed (K, Sigma, size, two_m)."""
    sched = sched or Schedule.single_stream()
    off, cols, w = _csr(g)
    n = g.n
    labels = np.ascontiguousarray(labels, dtype=np.uint32)
    if state is None:
        K = degrees(g)
        Sig, size = community_totals(n, labels, K)
        two_m = int(K.sum(dtype=np.uint64))
    else:
        K, Sig, size, two_m = state
    act = None if active is None else np.ascontiguousarray(active, dtype=np.uint8)
    bnd = None if bound is None else np.ascontiguousarray(bound, dtype=np.uint32)
    out = labels.copy()
    glo = np.zeros(n, dtype=np.uint64)
    ghi = np.zeros(n, dtype=np.uint64)
    v0, v1 = (0, n) if vertices is None else vertices
    lib = _load()

    def run(a, b):
        lib.or_sweep(n, _ptr(off), _ptr(cols), _ptr(w), _ptr(labels), _ptr(K), _ptr(Sig),
                     _ptr(size), two_m, _ptr(bnd), _ptr(act), mode, k, int(uncond),
                     len(sched.lanes), _ptr(sched.deg_max), _ptr(sched.lanes), sched.vec,
                     a, b, _ptr(out), _ptr(glo), _ptr(ghi), colors, sub_color, int(one_scan))

    if threads <= 1 or v1 - v0 < 1024:
        run(v0, v1)
    else:
        # interleave small ranges so heavy rows spread over threads
        step = max(256, (v1 - v0) // (threads * 64))
        ranges = [(a, min(a + step, v1)) for a in range(v0, v1, step)]
        with ThreadPoolExecutor(threads) as ex:
            list(ex.map(lambda r: run(*r), ranges))
    return out, (glo, ghi)


def gain_total(gains, idx=None) -> int:
    glo, ghi = gains
    if idx is not None:
        glo, ghi = glo[idx], ghi[idx]
    return int(glo.astype(object).sum()) + (int(ghi.astype(object).sum()) << 64)


def gains_as_ints(gains):
    glo, ghi = gains
    return [int(a) | (int(b) << 64) for a, b in zip(glo, ghi)]


# ---- aggregation (renumber + super-vertex graph) -----------------------------------------

def renumber(labels):
    """Dense ids in ascending order of the old id (the ids in use, in order)."""
    labels = np.asarray(labels, dtype=np.int64)
    used, new = np.unique(labels, return_inverse=True)
    return new.astype(np.uint32), len(used)


def aggregate(g, labels):
    """Super-vertex graph: community c' of every vertex becomes one vertex;
    entry (i, j, w) contributes w to entry (c'_i, c'_j).  Self-loop entries
    hold the summed weight of both directions of internal edges, so every
    K and 2m are preserved.  Returns (G', dense labels)."""
    from types import SimpleNamespace
    dense, nc = renumber(labels)
    off, cols, w = _csr(g)
    rows = np.repeat(np.arange(g.n, dtype=np.int64), np.diff(off))
    ci = dense[rows].astype(np.int64)
    cj = dense[cols].astype(np.int64)
    key = ci * nc + cj
    order = np.argsort(key, kind="stable")
    key = key[order]
    ww = w[order].astype(np.uint64)
    uniq, first = np.unique(key, return_index=True)
    sums = np.add.reduceat(ww, first) if len(ww) else ww
    r = uniq // nc
    counts = np.bincount(r, minlength=nc) if len(r) else np.zeros(nc, dtype=np.int64)
    noff = np.zeros(nc + 1, dtype=np.int64)
    np.cumsum(counts, out=noff[1:])
    if len(sums) and int(sums.max()) >= 2**32:
        raise OverflowError("aggregated weight does not fit uint32")
    G2 = SimpleNamespace(n=nc, offsets=noff, cols=(uniq % nc).astype(np.int32),
                         w=sums.astype(np.uint32), name=getattr(g, "name", "") + "'")
    return G2, dense


def aggregate_mg(g, labels, k: int = 8, uncond: int = 0, sched: Schedule | None = None,
                 symmetric: bool = False):
    """MG aggregation (Section 4.1, Fig. 3): super-vertex c links to the live
    slots of one MG sketch over all edges of c's members (no second pass).
    symmetric=False (Louvain): row c = the live slots of sketch(c), sorted
    by key.  symmetric=True (Leiden, Section 4.2: forward and reverse edge
    both inserted, an edge already present kept): every live slot (c, d, v)
    yields (c, d) and (d, c); when both sketch(c) holds d and sketch(d)
    holds c, the value from the smaller community's sketch is kept (the
    paper's first-inserted edge, with a fixed order).  Returns (G', dense)."""
    from types import SimpleNamespace
    sched = sched or Schedule.single_stream()
    dense, nc = renumber(labels)
    off, cols, w = _csr(g)
    order = np.argsort(dense, kind="stable").astype(np.uint32)
    moff = np.zeros(nc + 1, dtype=np.int64)
    np.cumsum(np.bincount(dense, minlength=nc), out=moff[1:])
    keys = np.empty(nc * k, dtype=np.uint32)
    vals = np.empty(nc * k, dtype=np.uint64)
    _load().or_aggregate_mg_sketch(g.n, _ptr(off), _ptr(cols), _ptr(w), _ptr(dense), nc, _ptr(moff),
                                   _ptr(order), k, int(uncond), len(sched.lanes), _ptr(sched.deg_max),
                                   _ptr(sched.lanes), sched.vec, _ptr(keys), _ptr(vals))
    src = np.repeat(np.arange(nc, dtype=np.int64), k)
    live = vals > 0
    s, d, v = src[live], keys[live].astype(np.int64), vals[live]
    if symmetric:
        own = {(int(a), int(b)): int(x) for a, b, x in zip(s, d, v)}
        edges = {}
        for (a, b), x in own.items():
            lo, hi = (a, b) if a <= b else (b, a)
            if (lo, hi) in edges:
                continue
            # value from the smaller community's sketch when it has the pair
            val = own.get((lo, hi), x) if lo != hi else x
            edges[(lo, hi)] = val
        ss, dd, vv = [], [], []
        for (lo, hi), x in edges.items():
            ss.append(lo); dd.append(hi); vv.append(x)
            if lo != hi:
                ss.append(hi); dd.append(lo); vv.append(x)
        s = np.array(ss, dtype=np.int64)
        d = np.array(dd, dtype=np.int64)
        v = np.array(vv, dtype=np.uint64)
    key = s * nc + d
    o = np.argsort(key, kind="stable")
    s, d, v = s[o], d[o], v[o]
    counts = np.bincount(s, minlength=nc) if len(s) else np.zeros(nc, dtype=np.int64)
    noff = np.zeros(nc + 1, dtype=np.int64)
    np.cumsum(counts, out=noff[1:])
    if len(v) and int(v.max()) >= 2**32:
        raise OverflowError("aggregated weight does not fit uint32")
    G2 = SimpleNamespace(n=nc, offsets=noff, cols=d.astype(np.int32), w=v.astype(np.uint32),
                         name=getattr(g, "name", "") + "'mg")
    return G2, dense


# ---- whole algorithms ------------------------------------------------------------------

def local_move_seq(g, labels, mode=MODE_LOUVAIN, k=8, uncond=False, tol=0.01, max_sweeps=20):
    """Sequential local-moving phase (in place on a copy); returns (labels, sweeps)."""
    off, cols, w = _csr(g)
    lab = np.ascontiguousarray(labels, dtype=np.uint32).copy()
    s = _load().or_local_move_seq(g.n, _ptr(off), _ptr(cols), _ptr(w), _ptr(lab), mode, k,
                                  int(uncond), tol, max_sweeps)
    return lab, s


def louvain_seq(g, k=8, uncond=False, tol=0.01, tol_drop=10.0, max_sweeps=20, max_passes=10,
                agg_tol=0.8):
    """Sequential Louvain: local-move, aggregate, repeat (Section 3.3).  The
    tolerance drops by `tol_drop` after every pass; stops when a pass moves
    nobody, when |V'|/|V| > agg_tol, or after max_passes.  Returns labels of
    the original vertices (dense)."""
    n0 = g.n
    top = np.arange(n0, dtype=np.uint32)
    cur = g
    for p in range(max_passes):
        lab0 = np.arange(cur.n, dtype=np.uint32)
        lab, sweeps = local_move_seq(cur, lab0, MODE_LOUVAIN, k, uncond, tol, max_sweeps)
        dense, nc = renumber(lab)
        top = dense[top]
        if nc == cur.n or nc > agg_tol * cur.n:
            break
        cur, _ = aggregate(cur, lab)
        tol /= tol_drop
    return renumber(top)[0]


def lpa_seq(g, k=8, uncond=False, tol=0.05, max_sweeps=20):
    lab, _ = local_move_seq(g, np.arange(g.n, dtype=np.uint32), MODE_LPA, k, uncond, tol,
                            max_sweeps)
    return renumber(lab)[0]


# ---- brute force (tiny graphs) ------------------------------------------------------------

def set_partitions(n: int):
    """All partitions of range(n) as restricted-growth label lists."""
    lab = [0] * n

    def rec(i, m):
        if i == n:
            yield list(lab)
            return
        for c in range(m + 1):
            lab[i] = c
            yield from rec(i + 1, max(m, c + 1))

    if n == 0:
        yield []
        return
    yield from rec(1, 1)


def brute_force_best(g):
    """Maximum modularity over all set partitions (n <= 10)."""
    best, arg = None, None
    for lab in set_partitions(g.n):
        q = modularity_fraction(g, np.array(lab, dtype=np.uint32))
        if best is None or q > best:
            best, arg = q, lab
    return best, arg


# ---- synchronous whole algorithms (the schedule the CUDA drivers follow) ------------------

def _dq_as_double(gain: int, two_m: int) -> float:
    """Summed scaled gain -> delta-Q in double, rounded the way the library
    does it: high and low 64-bit halves converted separately."""
    hi, lo = gain >> 64, gain & (2**64 - 1)
    return (float(hi) * 18446744073709551616.0 + float(lo)) / (float(two_m) * float(two_m) / 2.0)


def color_classes(n: int, colors: int) -> np.ndarray:
    """Colour class of every vertex: the 32-bit integer hash lowbias32
    (C. Wellons) of the vertex id, modulo the number of classes."""
    if colors <= 1:
        return np.zeros(n, dtype=np.uint32)
    x = np.arange(n, dtype=np.uint32)
    x ^= x >> np.uint32(16)
    x *= np.uint32(0x7FEB352D)
    x ^= x >> np.uint32(15)
    x *= np.uint32(0x846CA68B)
    x ^= x >> np.uint32(16)
    return x % np.uint32(colors)


def local_move_sync(g, mode, k, uncond, tol, max_sweeps, sched, threads=1, colors=8, init=None,
                    one_scan=False):
    """Local-moving phase from singletons, each sweep made of `colors`
    sub-sweeps: sub-sweep p decides the vertices of colour class p, all at
    once, from the state left by the previous sub-sweeps (colors=1: fully
    synchronous sweeps); Louvain's singleton rule bars only singleton targets
    whose id falls in the deciding class (see or_sweep).  Stops when nobody
    moves in a sweep, the sweep's
    summed delta-Q is <= tol (Louvain) or at most tol * n labels changed
    (LPA), or after max_sweeps.  Returns (labels, sweeps)."""
    n = g.n
    labels = np.arange(n, dtype=np.uint32) if init is None else np.array(init, dtype=np.uint32)
    K = degrees(g)
    two_m = int(K.sum(dtype=np.uint64))
    col = color_classes(n, colors)
    masks = [(col == p).astype(np.uint8) for p in range(max(colors, 1))]
    sweeps = 0
    while sweeps < max_sweeps:
        moved, gsum = 0, 0
        for p, act in enumerate(masks):
            Sig, size = community_totals(n, labels, K)
            out, gains = sweep(g, labels, mode, k, uncond, sched, active=act if colors > 1 else None,
                               threads=threads, state=(K, Sig, size, two_m), one_scan=one_scan,
                               colors=max(colors, 1), sub_color=p)
            moved += int(np.count_nonzero(out != labels))
            gsum += gain_total(gains)
            labels = out
        sweeps += 1
        if moved == 0:
            break
        if mode == MODE_LPA:
            if float(moved) <= tol * float(n):
                break
        elif _dq_as_double(gsum, two_m) <= tol:
            break
    return labels, sweeps


def louvain_sync(g, k=8, uncond=False, tol=0.01, tol_drop=10.0, max_sweeps=20, max_passes=10,
                 agg_tol=0.8, sched=None, threads=1, colors=8, agg_k=0, agg_sched=None):
    """Louvain with colour-class sub-sweeps: the exact schedule of cd_louvain
    (agg_k > 0: MG aggregation with agg_k slots)."""
    sched = sched or Schedule.single_stream()
    top = np.arange(g.n, dtype=np.uint32)
    cur = g
    for p in range(max_passes):
        if cur.n == 0:
            break
        lab, _ = local_move_sync(cur, MODE_LOUVAIN, k, uncond, tol, max_sweeps, sched, threads, colors)
        dense, nc = renumber(lab)
        top = dense[top]
        if nc == cur.n or nc > agg_tol * cur.n or p + 1 >= max_passes:
            break
        if agg_k > 0:
            cur, _ = aggregate_mg(cur, dense, agg_k, uncond, agg_sched or sched)
        else:
            cur, _ = aggregate(cur, dense)
        tol /= tol_drop
    return top


def lpa_sync(g, k=8, uncond=False, tol=0.05, max_sweeps=20, sched=None, threads=1, colors=8,
             one_scan=False):
    """LPA with colour-class sub-sweeps: the exact schedule of cd_lpa."""
    sched = sched or Schedule.single_stream()
    lab, _ = local_move_sync(g, MODE_LPA, k, uncond, tol, max_sweeps, sched, threads, colors,
                             one_scan=one_scan)
    return renumber(lab)[0]


def refine_sync(g, bound, k=8, uncond=False, sched=None, threads=1, colors=8):
    """Leiden refinement (Section 3.4): sub-communities start as singletons;
    one sweep of `colors` sub-sweeps in refine mode: only vertices still in
    a singleton move, only to sub-communities inside their own bound, and a
    same-colour singleton is never a target.  Returns sub-community labels."""
    sched = sched or Schedule.single_stream()
    n = g.n
    labels = np.arange(n, dtype=np.uint32)
    K = degrees(g)
    two_m = int(K.sum(dtype=np.uint64))
    bound = np.ascontiguousarray(bound, dtype=np.uint32)
    col = color_classes(n, colors)
    for p in range(colors):
        Sig, size = community_totals(n, labels, K)
        labels, _ = sweep(g, labels, MODE_REFINE, k, uncond, sched, active=(col == p).astype(np.uint8),
                          bound=bound, threads=threads, state=(K, Sig, size, two_m), colors=colors, sub_color=p)
    return labels


def leiden_sync(g, k=8, uncond=False, tol=0.01, tol_drop=10.0, max_sweeps=20, max_passes=10,
                agg_tol=0.8, sched=None, threads=1, colors=8, agg_k=0, agg_sched=None):
    """Leiden (Section 3.4): local-moving (from the previous level's bounds),
    refinement within the communities found, aggregation by the refined
    partition, repeated; the result is the last level's communities mapped
    to the input vertices.  The exact schedule of cd_leiden."""
    sched = sched or Schedule.single_stream()
    top = np.arange(g.n, dtype=np.uint32)
    result = top.copy()
    cur, init = g, None
    for p in range(max_passes):
        if cur.n == 0:
            break
        lab, _ = local_move_sync(cur, MODE_LOUVAIN, k, uncond, tol, max_sweeps, sched, threads, colors, init)
        dc, nc = renumber(lab)
        result = dc[top]
        if nc == cur.n or p + 1 >= max_passes:
            break
        rl = refine_sync(cur, dc, k, uncond, sched, threads, colors)
        dr, nr = renumber(rl)
        if nr == cur.n or nr > agg_tol * cur.n:
            break
        nxt = np.empty(nr, dtype=np.uint32)
        nxt[dr] = dc
        top = dr[top]
        if agg_k > 0:
            cur, _ = aggregate_mg(cur, dr, agg_k, uncond, agg_sched or sched, symmetric=True)
        else:
            cur, _ = aggregate(cur, dr)
        init = nxt
        tol /= tol_drop
    return renumber(result)[0]
