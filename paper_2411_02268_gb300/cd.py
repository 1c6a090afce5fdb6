"""Python binding of the C ABI in include/cd.h (ctypes; argument marshalling only).

Every function here has the name of the C entry point it calls and does no
computation of its own: graphs and labels are passed as device tensors
(``torch`` CUDA tensors, device memory) or as numpy arrays (host memory, the
library copies them in and out).  The library must have been built
(``__graft_entry__.build()``); a missing library raises, there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
SO = os.path.join(_PKG, "lib", "libcd.so")

CD_OK, CD_EINVAL, CD_ENOMEM, CD_ECUDA, CD_ETIMEOUT, CD_EOVERFLOW, CD_ENOTIMPL, CD_ESIZE = 0, -1, -2, -3, -4, -5, -6, -7
MODE_LOUVAIN, MODE_LPA, MODE_REFINE = 0, 1, 2
MEM_DEVICE, MEM_HOST = 0, 1
MAX_BUCKETS = 16

# Symbols declared in include/cd.h.
SYMBOLS = ("cd_strerror", "cd_last_stats", "cd_default_schedule", "cd_sweep", "cd_modularity",
           "cd_louvain", "cd_lpa", "cd_leiden", "cd_aggregate", "cd_aggregate_mg", "cd_modularity_noalloc",
           "cd_features", "cd_mlp_forward", "cd_mlp_gradient", "cd_mlp_train", "cd_trace",
           "cd_louvain_batched", "cd_autotune")


class CSR(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("nnz", ctypes.c_int64), ("offsets", ctypes.c_void_p),
                ("cols", ctypes.c_void_p), ("weights", ctypes.c_void_p), ("memory", ctypes.c_int32)]


class Schedule(ctypes.Structure):
    _fields_ = [("nbuckets", ctypes.c_int32), ("vec", ctypes.c_int32),
                ("deg_max", ctypes.c_int64 * MAX_BUCKETS), ("lanes", ctypes.c_int32 * MAX_BUCKETS),
                ("blocks_per_sm", ctypes.c_int32)]

    def as_lists(self):
        nb = self.nbuckets
        return list(self.deg_max[:nb]), list(self.lanes[:nb]), self.vec


class MLP(ctypes.Structure):
    _fields_ = [("W1", (ctypes.c_float * 8) * 32), ("b1", ctypes.c_float * 32), ("w2", ctypes.c_float * 32),
                ("b2", ctypes.c_float)]

    def to_numpy(self):
        W1 = np.ctypeslib.as_array(self.W1).astype(np.float64).reshape(32, 8)
        return (W1, np.ctypeslib.as_array(self.b1).astype(np.float64),
                np.ctypeslib.as_array(self.w2).astype(np.float64), float(self.b2))

    @staticmethod
    def from_numpy(W1, b1, w2, b2):
        m = MLP()
        np.ctypeslib.as_array(m.W1)[:] = np.asarray(W1, dtype=np.float32).reshape(32, 8)
        np.ctypeslib.as_array(m.b1)[:] = np.asarray(b1, dtype=np.float32)
        np.ctypeslib.as_array(m.w2)[:] = np.asarray(w2, dtype=np.float32)
        m.b2 = float(b2)
        return m

    @staticmethod
    def init(seed=0):
        """Small random initial weights (He-scaled), for training."""
        rng = np.random.default_rng(seed)
        return MLP.from_numpy(rng.normal(0, np.sqrt(2 / 8), (32, 8)), np.zeros(32),
                              rng.normal(0, np.sqrt(1 / 32), 32), 0.0)


class Params(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int32), ("subtract", ctypes.c_int32), ("tolerance", ctypes.c_double),
                ("tolerance_drop", ctypes.c_double), ("aggregation_tolerance", ctypes.c_double),
                ("max_sweeps", ctypes.c_int32), ("max_passes", ctypes.c_int32),
                ("sched", ctypes.POINTER(Schedule)), ("stream", ctypes.c_void_p),
                ("timing", ctypes.c_int32), ("colors", ctypes.c_int32),
                ("sub_color", ctypes.c_int32), ("one_scan", ctypes.c_int32), ("agg_k", ctypes.c_int32),
                ("skip_rule", ctypes.c_int32), ("skip_threshold", ctypes.c_float),
                ("skip_model", ctypes.POINTER(MLP)), ("capture", ctypes.c_int32)]


class Stats(ctypes.Structure):
    _fields_ = [("sweeps", ctypes.c_int64), ("passes", ctypes.c_int64), ("moved", ctypes.c_int64),
                ("gain_lo", ctypes.c_uint64), ("gain_hi", ctypes.c_uint64),
                ("communities", ctypes.c_int64), ("scratch_bytes", ctypes.c_int64),
                ("sweep_kernel_ms", ctypes.c_double), ("sweep_kernel_launches", ctypes.c_int64),
                ("modularity", ctypes.c_double), ("entries_scanned", ctypes.c_int64),
                ("full_sweeps", ctypes.c_int64), ("cuda_error", ctypes.c_char * 128),
                ("kernel_launches", ctypes.c_int64), ("candidates", ctypes.c_int64),
                ("phase_ms", ctypes.c_double * 4)]


TUNE_MAX_K = 8


class TuneReport(ctypes.Structure):
    _fields_ = [("default_ms", ctypes.c_double), ("sweep_ms", ctypes.c_double * TUNE_MAX_K),
                ("run_ms", ctypes.c_double * TUNE_MAX_K), ("q_mean", ctypes.c_double * TUNE_MAX_K),
                ("trials", ctypes.c_int32), ("chosen", ctypes.c_int32)]


class ModularityParts(ctypes.Structure):
    _fields_ = [("sigma_in", ctypes.c_uint64), ("sum_sq_lo", ctypes.c_uint64),
                ("sum_sq_hi", ctypes.c_uint64), ("two_m", ctypes.c_uint64)]


class CDError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        detail = ""
        if code == CD_ECUDA:
            detail = ": " + cd_last_stats().cuda_error.decode(errors="replace")
        super().__init__(f"{where} failed: {cd_strerror(code)} ({code}){detail}")


_lock = threading.Lock()
_lib = None


def lib():
    """The loaded CUDA library; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(SO):
                raise RuntimeError(f"CUDA library {SO} is missing: run __graft_entry__.build()")
            L = ctypes.CDLL(SO)
            P = ctypes.c_void_p
            L.cd_strerror.argtypes = [ctypes.c_int]
            L.cd_strerror.restype = ctypes.c_char_p
            L.cd_last_stats.argtypes = [ctypes.POINTER(Stats)]
            L.cd_default_schedule.argtypes = [ctypes.c_int, ctypes.POINTER(Schedule)]
            L.cd_sweep.argtypes = [ctypes.POINTER(CSR), ctypes.POINTER(Params), ctypes.c_int, P, P, P, P,
                                   ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_uint64)]
            L.cd_modularity.argtypes = [ctypes.POINTER(CSR), P, P, ctypes.POINTER(ctypes.c_double),
                                        ctypes.POINTER(ModularityParts)]
            L.cd_modularity_noalloc.argtypes = L.cd_modularity.argtypes
            L.cd_features.argtypes = [ctypes.POINTER(CSR), P, P, P, P, P, P]
            L.cd_mlp_forward.argtypes = [P, ctypes.c_int64, ctypes.POINTER(MLP), P, P]
            L.cd_mlp_gradient.argtypes = [P, P, ctypes.c_int64, ctypes.POINTER(MLP), ctypes.POINTER(MLP),
                                          ctypes.POINTER(ctypes.c_double), P]
            L.cd_mlp_train.argtypes = [P, P, ctypes.c_int64, ctypes.c_int, ctypes.c_double, ctypes.POINTER(MLP),
                                       ctypes.POINTER(ctypes.c_double), P]
            L.cd_trace.argtypes = [ctypes.POINTER(CSR), ctypes.POINTER(Params), ctypes.c_double, P, P,
                                   ctypes.c_int64, ctypes.POINTER(ctypes.c_int64)]
            for name in ("cd_louvain", "cd_lpa", "cd_leiden"):
                getattr(L, name).argtypes = [ctypes.POINTER(CSR), ctypes.POINTER(Params), P,
                                             ctypes.POINTER(ctypes.c_double)]
            L.cd_aggregate.argtypes = [ctypes.POINTER(CSR), P, P, P, P, P, P,
                                       ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]
            L.cd_aggregate_mg.argtypes = [ctypes.POINTER(CSR), P, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                          ctypes.POINTER(Schedule), P, P, P, P, P,
                                          ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]
            L.cd_louvain_batched.argtypes = [ctypes.POINTER(CSR), ctypes.c_int, ctypes.POINTER(Params), P, P, P]
            L.cd_autotune.argtypes = [ctypes.POINTER(CSR), ctypes.c_int, ctypes.POINTER(Params), P, ctypes.c_int,
                                      ctypes.c_double, ctypes.POINTER(Schedule), ctypes.POINTER(ctypes.c_int),
                                      ctypes.POINTER(TuneReport)]
            for name in SYMBOLS:
                if name != "cd_strerror":
                    getattr(L, name).restype = ctypes.c_int
            _lib = L
    return _lib


def _check(rc: int, where: str):
    if rc != CD_OK:
        raise CDError(rc, where)


# ---- argument marshalling -------------------------------------------------------

def _ptr(x):
    """Address of a torch tensor or numpy array (None -> NULL)."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    return x.ctypes.data


def _is_device(x) -> bool:
    return hasattr(x, "is_cuda") and x.is_cuda


class Graph:
    """A CSR graph handed to the library: device tensors or host arrays."""

    def __init__(self, n, offsets, cols, weights):
        self.n = int(n)
        self.offsets, self.cols, self.weights = offsets, cols, weights
        self.memory = MEM_DEVICE if _is_device(offsets) else MEM_HOST
        if self.memory == MEM_HOST:
            self.offsets = np.ascontiguousarray(offsets, dtype=np.int64)
            self.cols = np.ascontiguousarray(cols, dtype=np.int32)
            self.weights = np.ascontiguousarray(weights, dtype=np.uint32)

    @property
    def nnz(self) -> int:
        return int(self.cols.shape[0])

    def csr(self) -> CSR:
        return CSR(self.n, self.nnz, _ptr(self.offsets), _ptr(self.cols), _ptr(self.weights), self.memory)

    @staticmethod
    def host(g) -> "Graph":
        return Graph(g.n, g.offsets, g.cols, g.w)

    @staticmethod
    def to_device(g, device="cuda") -> "Graph":
        import torch
        return Graph(g.n, torch.from_numpy(np.ascontiguousarray(g.offsets, dtype=np.int64)).to(device),
                     torch.from_numpy(np.ascontiguousarray(g.cols, dtype=np.int32)).to(device),
                     torch.from_numpy(np.ascontiguousarray(g.w, dtype=np.uint32).view(np.int32)).to(device))


def current_stream():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def make_params(k=8, subtract=0, tolerance=0.01, tolerance_drop=10.0, aggregation_tolerance=0.8,
                max_sweeps=20, max_passes=10, schedule: Schedule | None = None, stream=None,
                timing=False, colors=0, sub_color=0, one_scan=False, agg_k=0, skip_rule=0,
                skip_threshold=0.5, skip_model: "MLP | None" = None, capture=True) -> Params:
    p = Params()
    p.k, p.subtract = int(k), int(subtract)
    p.tolerance, p.tolerance_drop, p.aggregation_tolerance = tolerance, tolerance_drop, aggregation_tolerance
    p.max_sweeps, p.max_passes = int(max_sweeps), int(max_passes)
    p.sched = ctypes.pointer(schedule) if schedule is not None else None
    p.stream = stream.value if isinstance(stream, ctypes.c_void_p) else stream
    p.timing = int(bool(timing))
    p.colors = int(colors)
    p.sub_color = int(sub_color)
    p.one_scan = int(bool(one_scan))
    p.agg_k = int(agg_k)
    p.skip_rule = int(skip_rule)
    p.skip_threshold = float(skip_threshold)
    p.skip_model = ctypes.pointer(skip_model) if skip_model is not None else None
    p.capture = int(bool(capture))
    p._keep_model = skip_model
    p._keep = schedule
    return p


def schedule_from(deg_max, lanes, vec=4, blocks_per_sm=0) -> Schedule:
    s = Schedule()
    s.nbuckets, s.vec, s.blocks_per_sm = len(lanes), vec, int(blocks_per_sm)
    for b, (d, l) in enumerate(zip(deg_max, lanes)):
        s.deg_max[b], s.lanes[b] = int(d), int(l)
    return s


# ---- entry points ---------------------------------------------------------------------

def cd_strerror(code: int) -> str:
    return lib().cd_strerror(code).decode()


def cd_last_stats() -> Stats:
    s = Stats()
    _check(lib().cd_last_stats(ctypes.byref(s)), "cd_last_stats")
    return s


def cd_default_schedule(k: int = 8) -> Schedule:
    s = Schedule()
    _check(lib().cd_default_schedule(k, ctypes.byref(s)), "cd_default_schedule")
    return s


def cd_sweep(g: Graph, params: Params, mode: int, labels_in, active=None, bound=None, labels_out=None):
    """One synchronous sweep; returns (labels_out, moved, gain) with gain a Python int."""
    if labels_out is None:
        if g.memory == MEM_DEVICE:
            import torch
            labels_out = torch.empty_like(labels_in)
        else:
            labels_out = np.empty(g.n, dtype=np.uint32)
    moved = ctypes.c_int64()
    gain = (ctypes.c_uint64 * 2)()
    csr = g.csr()
    rc = lib().cd_sweep(ctypes.byref(csr), ctypes.byref(params), mode, _ptr(labels_in), _ptr(active),
                        _ptr(bound), _ptr(labels_out), ctypes.byref(moved), gain)
    _check(rc, "cd_sweep")
    return labels_out, moved.value, int(gain[0]) | (int(gain[1]) << 64)


def cd_modularity(g: Graph, labels, stream=None):
    """Returns (Q, (sigma_in, sum_Sigma2, two_m))."""
    q = ctypes.c_double()
    parts = ModularityParts()
    csr = g.csr()
    st = stream.value if isinstance(stream, ctypes.c_void_p) else stream
    _check(lib().cd_modularity(ctypes.byref(csr), _ptr(labels), st, ctypes.byref(q), ctypes.byref(parts)),
           "cd_modularity")
    return q.value, (parts.sigma_in, parts.sum_sq_lo | (parts.sum_sq_hi << 64), parts.two_m)


def cd_modularity_noalloc(g: Graph, labels, stream=None):
    """As cd_modularity, with the library's fixed scratch array instead of any
    device allocation (device memory only, at most 2^20 vertices)."""
    q = ctypes.c_double()
    parts = ModularityParts()
    csr = g.csr()
    st = stream.value if isinstance(stream, ctypes.c_void_p) else stream
    _check(lib().cd_modularity_noalloc(ctypes.byref(csr), _ptr(labels), st, ctypes.byref(q), ctypes.byref(parts)),
           "cd_modularity_noalloc")
    return q.value, (parts.sigma_in, parts.sum_sq_lo | (parts.sum_sq_hi << 64), parts.two_m)


def _whole(fn_name, g: Graph, params: Params, labels_out=None):
    if labels_out is None:
        if g.memory == MEM_DEVICE:
            import torch
            labels_out = torch.empty(g.n, dtype=torch.int32, device=g.offsets.device)
        else:
            labels_out = np.empty(g.n, dtype=np.uint32)
    q = ctypes.c_double()
    csr = g.csr()
    _check(getattr(lib(), fn_name)(ctypes.byref(csr), ctypes.byref(params), _ptr(labels_out), ctypes.byref(q)),
           fn_name)
    return labels_out, q.value


def cd_louvain(g: Graph, params: Params, labels_out=None):
    return _whole("cd_louvain", g, params, labels_out)


def cd_louvain_batched(graphs, params: Params, labels_out=None):
    """Louvain on a list of graphs (all device or all host) in one batched
    call.  Returns (labels per graph, modularity per graph as a numpy array,
    sweeps per graph as a numpy array)."""
    G = len(graphs)
    if labels_out is None:
        labels_out = []
        for g in graphs:
            if g.memory == MEM_DEVICE:
                import torch
                labels_out.append(torch.empty(max(g.n, 1), dtype=torch.int32, device=g.offsets.device))
            else:
                labels_out.append(np.empty(max(g.n, 1), dtype=np.uint32))
    csrs = (CSR * G)(*[g.csr() for g in graphs])
    outs = (ctypes.c_void_p * G)(*[_ptr(x) for x in labels_out])
    q = np.zeros(G, dtype=np.float64)
    sw = np.zeros(G, dtype=np.int64)
    _check(lib().cd_louvain_batched(csrs, G, ctypes.byref(params), ctypes.addressof(outs), q.ctypes.data,
                                    sw.ctypes.data), "cd_louvain_batched")
    return [x[:g.n] for x, g in zip(labels_out, graphs)], q, sw


def cd_autotune(graphs, params: Params, ks=(4, 8, 16), q_tol=0.005):
    """Tunes the schedule and picks k for a batch (see cd.h).  Returns
    (Schedule, k, TuneReport)."""
    G = len(graphs)
    csrs = (CSR * G)(*[g.csr() for g in graphs])
    karr = (ctypes.c_int * len(ks))(*[int(k) for k in ks])
    sched = Schedule()
    k_out = ctypes.c_int()
    rep = TuneReport()
    _check(lib().cd_autotune(csrs, G, ctypes.byref(params), ctypes.addressof(karr), len(ks), float(q_tol),
                             ctypes.byref(sched), ctypes.byref(k_out), ctypes.byref(rep)), "cd_autotune")
    return sched, k_out.value, rep


def cd_lpa(g: Graph, params: Params, labels_out=None):
    return _whole("cd_lpa", g, params, labels_out)


def cd_leiden(g: Graph, params: Params, labels_out=None):
    return _whole("cd_leiden", g, params, labels_out)


def cd_aggregate(g: Graph, labels, stream=None):
    """Returns (dense labels, super-graph as Graph of device tensors)."""
    import torch
    dev = g.offsets.device
    dense = torch.empty(g.n, dtype=torch.int32, device=dev)
    off = torch.empty(g.n + 1, dtype=torch.int64, device=dev)
    cols = torch.empty(max(g.nnz, 1), dtype=torch.int32, device=dev)
    w = torch.empty(max(g.nnz, 1), dtype=torch.int32, device=dev)
    n_out, nnz_out = ctypes.c_int64(), ctypes.c_int64()
    csr = g.csr()
    st = stream.value if isinstance(stream, ctypes.c_void_p) else stream
    _check(lib().cd_aggregate(ctypes.byref(csr), _ptr(labels), st, _ptr(dense), _ptr(off), _ptr(cols), _ptr(w),
                              ctypes.byref(n_out), ctypes.byref(nnz_out)), "cd_aggregate")
    n2, m2 = n_out.value, nnz_out.value
    return dense, Graph(n2, off[:n2 + 1], cols[:m2], w[:m2])


def cd_aggregate_mg(g: Graph, labels, k=8, subtract=0, symmetric=False, schedule: Schedule | None = None,
                    stream=None):
    """MG aggregation; returns (dense labels, super-graph as Graph of device tensors)."""
    import torch
    dev = g.offsets.device
    dense = torch.empty(g.n, dtype=torch.int32, device=dev)
    off = torch.empty(g.n + 1, dtype=torch.int64, device=dev)
    cap = max(g.nnz, 1)
    cols = torch.empty(cap, dtype=torch.int32, device=dev)
    w = torch.empty(cap, dtype=torch.int32, device=dev)
    n_out, nnz_out = ctypes.c_int64(), ctypes.c_int64()
    csr = g.csr()
    st = stream.value if isinstance(stream, ctypes.c_void_p) else stream
    sp = ctypes.byref(schedule) if schedule is not None else None
    _check(lib().cd_aggregate_mg(ctypes.byref(csr), _ptr(labels), k, subtract, int(symmetric), sp, st, _ptr(dense),
                                 _ptr(off), _ptr(cols), _ptr(w), ctypes.byref(n_out), ctypes.byref(nnz_out)),
           "cd_aggregate_mg")
    n2, m2 = n_out.value, nnz_out.value
    return dense, Graph(n2, off[:n2 + 1], cols[:m2], w[:m2])


def cd_features(g: Graph, labels, moved_last=None, since_move=None, attach=None, stream=None):
    """(n, 8) float16 features (device tensor)."""
    import torch
    x = torch.empty((g.n, 8), dtype=torch.float16, device=g.offsets.device)
    csr = g.csr()
    st = stream.value if isinstance(stream, ctypes.c_void_p) else stream
    _check(lib().cd_features(ctypes.byref(csr), _ptr(labels), _ptr(moved_last), _ptr(since_move), _ptr(attach),
                             _ptr(x), st), "cd_features")
    return x


def cd_mlp_forward(x, model: MLP, stream=None):
    import torch
    p = torch.empty(x.shape[0], dtype=torch.float32, device=x.device)
    _check(lib().cd_mlp_forward(_ptr(x), x.shape[0], ctypes.byref(model), _ptr(p), stream), "cd_mlp_forward")
    return p


def cd_mlp_gradient(x, y, model: MLP, stream=None):
    """Returns (loss, gradient as MLP)."""
    g = MLP()
    loss = ctypes.c_double()
    _check(lib().cd_mlp_gradient(_ptr(x), _ptr(y), x.shape[0], ctypes.byref(model), ctypes.byref(g),
                                 ctypes.byref(loss), stream), "cd_mlp_gradient")
    return loss.value, g


def cd_mlp_train(x, y, model: MLP, steps=200, lr=0.01, stream=None):
    """Trains `model` in place; returns the final loss."""
    loss = ctypes.c_double()
    _check(lib().cd_mlp_train(_ptr(x), _ptr(y), x.shape[0], steps, lr, ctypes.byref(model), ctypes.byref(loss),
                              stream), "cd_mlp_train")
    return loss.value


def cd_trace(g: Graph, params: Params, sample_rate=0.25, capacity=None):
    """Move traces of the plain method: (x float16 (m, 8), y uint8 (m,)) device tensors."""
    import torch
    cap = capacity if capacity is not None else max(1, int(g.n * 20 * sample_rate) + 1024)
    x = torch.empty((cap, 8), dtype=torch.float16, device=g.offsets.device)
    y = torch.empty(cap, dtype=torch.uint8, device=g.offsets.device)
    cnt = ctypes.c_int64()
    csr = g.csr()
    _check(lib().cd_trace(ctypes.byref(csr), ctypes.byref(params), sample_rate, _ptr(x), _ptr(y), cap,
                          ctypes.byref(cnt)), "cd_trace")
    return x[:cnt.value], y[:cnt.value]
