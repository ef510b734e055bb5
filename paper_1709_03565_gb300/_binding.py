"""Thin ctypes binding of ``include/skis.h``: the same entry points, with
argument marshalling only (pointers from numpy arrays or torch tensors,
memory space inferred from them, stream from torch). Every step of the path
runs in ``libskis.so``; there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libskis.so")

SKIS_OK, SKIS_EINVAL, SKIS_ENOMEM, SKIS_ERR_CUDA = 0, 1, 2, 3
SKIS_ERR_RETRY_LIMIT, SKIS_ERR_ARENA_FULL, SKIS_ERR_INTERNAL, SKIS_ERR_EXCHANGE = 4, 5, 6, 7
SKIS_W_EXPLICIT_P, SKIS_W_EXPLICIT_TAU, SKIS_W_WC, SKIS_W_TRI = 0, 1, 2, 3
SKIS_MEM_HOST, SKIS_MEM_DEVICE = 0, 1
SKIS_OPT_RETRY_CAP, SKIS_OPT_CTA_SLOTS, SKIS_OPT_WARP_BLOCKS = 0, 1, 2
SKIS_OPT_THREAD_MAX_DEG, SKIS_OPT_THREAD_BLOCKS, SKIS_OPT_QUERY_INDEX, SKIS_OPT_THREAD_MAX_STEPS = 3, 4, 5, 6
SKIS_OPT_SAMPLER, SKIS_OPT_THREAD_MAX_RETRIES, SKIS_OPT_FIRST_STEP = 7, 8, 9
SKIS_OPT_WARP_MAX_COINS, SKIS_OPT_CTA_HUB_QUADS, SKIS_OPT_FIRST_ID, SKIS_OPT_CTA_QUEUE_CAP = 10, 11, 12, 13
SKIS_OPT_CTA_THREADS = 14
SKIS_DIFF_IC, SKIS_DIFF_LT = 0, 1


class SkisError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"[skis status {code}] {msg}")
        self.code = code


class skis_graph_info(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("m", ctypes.c_int64), ("W", ctypes.c_uint64), ("f", ctypes.c_int32),
                ("row_uniform_tau", ctypes.c_int32), ("Gamma", ctypes.c_double), ("diffusion", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class skis_stats(ctypes.Structure):
    _fields_ = [("T", ctypes.c_uint64), ("entries", ctypes.c_uint64), ("coins", ctypes.c_uint64),
                ("retries", ctypes.c_uint64), ("arena_capacity", ctypes.c_uint64),
                ("arena_reserved", ctypes.c_uint64), ("to_warp", ctypes.c_uint64),
                ("deferred", ctypes.c_uint64), ("last_thread_ms", ctypes.c_double),
                ("last_warp_ms", ctypes.c_double), ("last_cta_ms", ctypes.c_double),
                ("last_sample_ms", ctypes.c_double), ("last_passes", ctypes.c_uint64),
                ("thread_max_deg", ctypes.c_uint64), ("thread_max_steps", ctypes.c_uint64),
                ("warp_max_coins", ctypes.c_uint64), ("cta_hub_quads", ctypes.c_uint64),
                ("first_id", ctypes.c_uint64), ("last_query_ms", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class skis_dssa_result(ctypes.Structure):
    _fields_ = [("rounds", ctypes.c_int32), ("stopped_by", ctypes.c_int32), ("samples", ctypes.c_uint64),
                ("lambda2", ctypes.c_uint64), ("coverage", ctypes.c_int64), ("coverage_c", ctypes.c_int64),
                ("estimate", ctypes.c_double), ("estimate_c", ctypes.c_double), ("eps1", ctypes.c_double),
                ("eps2", ctypes.c_double), ("eps3", ctypes.c_double)]


_lib = None

# (name, restype, argtypes) of every entry point declared in include/skis.h
_P, _I64, _U64, _I32, _INT = ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint64, ctypes.c_int32, ctypes.c_int
_SIGNATURES = [
    ("skis_load_graph", _INT, [_P, _I64, _I64, _P, _P, _P, _INT, _U64, _INT, _P]),
    ("skis_load_graph_lt", _INT, [_P, _I64, _I64, _P, _P, _P, _INT, _U64, _INT, _P]),
    ("skis_graph_get_info", _INT, [_P, _P]),
    ("skis_graph_export", _INT, [_P, _P, _P, _P, _P, _P, _P, _P, _P]),
    ("skis_graph_free", None, [_P]),
    ("skis_sketch_create", _INT, [_P, _P, _U64, _U64, _P]),
    ("skis_sketch_set_option", _INT, [_P, _INT, _U64]),
    ("skis_sketch_autotune", _INT, [_P, _U64, _P, _P, _P, _I32, _P, _P]),
    ("skis_sample", _INT, [_P, _U64, _P, _P]),
    ("skis_sample_to_size", _INT, [_P, _U64, _U64, _P, _P, _P]),
    ("skis_estimate", _INT, [_P, _I32, _P, _P, _P, _P, _INT, _P]),
    ("skis_greedy_maxcover", _INT, [_P, _I32, _P, _P, _P, _P]),
    ("skis_sketch_stats", _INT, [_P, _P]),
    ("skis_sketch_export", _INT, [_P, _U64, _U64, _P, _P, _P, _P, _P, _P, _U64, _P]),
    ("skis_sketch_free", None, [_P]),
    ("skis_estimate_noalloc", _INT, [_P, _I32, _P, _P, _P, _P, _P, _U64, _P]),
    ("skis_dssa_maxinf", _INT, [_P, _U64, _U64, _I32, ctypes.c_double, ctypes.c_double, _U64, _U64, _U64, _P, _P,
                                _P]),
    ("skis_server_create", _INT, [_P, _P, _I32, _I32, _U64]),
    ("skis_server_submit", _INT, [_P, _P, _I32, _P]),
    ("skis_server_progress", _INT, [_P, _I32, _P, _I32, _P]),
    ("skis_server_poll", _INT, [_P, _U64, _P, _P, _P]),
    ("skis_server_counts", _INT, [_P, _P, _P, _P, _P]),
    ("skis_server_free", None, [_P]),
    ("skis_estimate_sharded", _INT, [_P, _I32, _P, _P, _P, _P, _INT, _P, _P, _P, _P]),
    ("skis_greedy_maxcover_sharded", _INT, [_P, _I32, _P, _P, _P, _P, _P, _P, _P]),
    ("skis_philox_rate", _INT, [_U64, _U64, _U64, _INT, _P, _P, _P]),
    ("skis_kernel_launches", ctypes.c_uint64, []),
    ("skis_device_allocations", ctypes.c_uint64, []),
    ("skis_last_error", ctypes.c_char_p, []),
]


def lib():
    """The loaded ``libskis.so`` (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with paper_1709_03565_gb300.build()")
        h = ctypes.CDLL(LIB_PATH)
        for name, res, args in _SIGNATURES:
            f = getattr(h, name)
            f.restype = res
            f.argtypes = args
        _lib = h
    return _lib


def _check(rc: int):
    if rc != SKIS_OK:
        raise SkisError(rc, lib().skis_last_error().decode())


def _is_torch(x):
    return type(x).__module__.startswith("torch")


def _ptr(x, dtype):
    """Pointer and memory space of a contiguous array of the given numpy dtype."""
    if x is None:
        return None, None
    if _is_torch(x):
        import torch

        want = {np.int32: torch.int32, np.int64: torch.int64, np.uint32: torch.uint32,
                np.uint64: torch.uint64, np.float64: torch.float64}[dtype]
        if x.dtype != want:
            raise TypeError(f"expected {want}, got {x.dtype}")
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return ctypes.c_void_p(x.data_ptr()), (SKIS_MEM_DEVICE if x.is_cuda else SKIS_MEM_HOST)
    if not isinstance(x, np.ndarray) or x.dtype != np.dtype(dtype) or not x.flags["C_CONTIGUOUS"]:
        raise TypeError(f"expected a C-contiguous numpy array of {np.dtype(dtype)}")
    return ctypes.c_void_p(x.ctypes.data), SKIS_MEM_HOST


def _numel(x) -> int:
    return int(x.numel()) if _is_torch(x) else int(np.size(x))


def _last(x) -> int:
    return int(x[-1].item()) if _is_torch(x) else int(x[-1])


def _check_queries(seed_offsets, seeds, coverage_out, estimate_out) -> int:
    """Sizes of a query batch against its outputs, before any launch: the
    library writes q coverage counts and estimates and reads seeds
    [0, seed_offsets[q]); CUDA tensors must be on the current device."""
    q = _numel(seed_offsets) - 1
    if q < 0:
        raise ValueError("seed_offsets needs q + 1 >= 1 entries")
    if estimate_out is not None and _numel(estimate_out) < q:
        raise ValueError(f"estimate_out holds {_numel(estimate_out)} entries, {q} queries need {q}")
    if coverage_out is not None and _numel(coverage_out) < q:
        raise ValueError(f"coverage_out holds {_numel(coverage_out)} entries, {q} queries need {q}")
    need = _last(seed_offsets) if q > 0 else 0
    have = 0 if seeds is None else _numel(seeds)
    if need > have:
        raise ValueError(f"seed_offsets[-1] = {need} but seeds holds {have} entries")
    _check_current_device(seed_offsets, seeds, coverage_out, estimate_out)
    return q


def _check_current_device(*xs):
    for x in xs:
        if x is not None and _is_torch(x) and x.is_cuda:
            import torch

            if x.device.index != torch.cuda.current_device():
                raise ValueError(f"tensor on {x.device}, the current device is cuda:{torch.cuda.current_device()}")


def _space(*spaces):
    s = {x for x in spaces if x is not None}
    if len(s) > 1:
        raise ValueError("all arrays of one call must be on the host or all on the device")
    return s.pop() if s else SKIS_MEM_HOST


def _stream(stream):
    if stream is None:
        try:
            import torch

            if torch.cuda.is_available() and torch.cuda.is_initialized():
                return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        except ImportError:
            pass
        return None
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


class _Handle:
    _free = None

    def __init__(self, ptr, keep=None):
        self.ptr = ptr
        self._keep = keep

    def close(self):
        if self.ptr is not None and self.ptr.value:
            getattr(lib(), self._free)(self.ptr)
        self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Graph(_Handle):
    _free = "skis_graph_free"


class Sketch(_Handle):
    _free = "skis_sketch_free"


class Server(_Handle):
    _free = "skis_server_free"

    def __init__(self, ptr, keep=None):
        super().__init__(ptr, keep)
        self._done = np.empty(4096, np.uint64)


# ------------------------------------------------------------ entry points
def _load(fn, n, src, dst, weights, weight_model, weight_seed, stream) -> Graph:
    ps, ss = _ptr(src, np.int32)
    pd, sd = _ptr(dst, np.int32)
    wdt = np.float64 if weight_model == SKIS_W_EXPLICIT_P else np.uint32
    pw, sw = _ptr(weights, wdt) if weight_model in (SKIS_W_EXPLICIT_P, SKIS_W_EXPLICIT_TAU) else (None, None)
    out = ctypes.c_void_p()
    m = int(src.shape[0])
    _check(fn(ctypes.byref(out), int(n), m, ps, pd, pw, int(weight_model), int(weight_seed), _space(ss, sd, sw),
              _stream(stream)))
    return Graph(out)


def skis_load_graph(n, src, dst, weights=None, weight_model=SKIS_W_WC, weight_seed=0, stream=None) -> Graph:
    return _load(lib().skis_load_graph, n, src, dst, weights, weight_model, weight_seed, stream)


def skis_load_graph_lt(n, src, dst, weights=None, weight_model=SKIS_W_WC, weight_seed=0, stream=None) -> Graph:
    """The graph under the Linear Threshold model."""
    return _load(lib().skis_load_graph_lt, n, src, dst, weights, weight_model, weight_seed, stream)


def skis_graph_get_info(g: Graph) -> dict:
    info = skis_graph_info()
    _check(lib().skis_graph_get_info(g.ptr, ctypes.byref(info)))
    return {k: getattr(info, k) for k, _ in info._fields_}


_GRAPH_ARRAYS = ("off", "src", "tau", "perm", "w", "prob", "alias")


def skis_graph_export(g: Graph, stream=None, keys=_GRAPH_ARRAYS) -> dict:
    """The graph's arrays (those named in keys) as host numpy arrays."""
    info = skis_graph_get_info(g)
    n, m = info["n"], info["m"]
    shapes = dict(off=(n + 1, np.int64), src=(m, np.int32), tau=(m, np.uint32), perm=(m, np.int64),
                  w=(n, np.uint64), prob=(n, np.uint64), alias=(n, np.uint32))
    a = {k: np.empty(shapes[k][0], shapes[k][1]) for k in keys}
    P = lambda k: ctypes.c_void_p(a[k].ctypes.data) if k in a else None  # noqa: E731
    _check(lib().skis_graph_export(g.ptr, *[P(k) for k in _GRAPH_ARRAYS], _stream(stream)))
    return a


def skis_graph_free(g: Graph):
    g.close()


def skis_sketch_create(g: Graph, seed: int, arena_entries: int = 0, stream=None) -> Sketch:
    out = ctypes.c_void_p()
    _check(lib().skis_sketch_create(ctypes.byref(out), g.ptr, int(seed), int(arena_entries), _stream(stream)))
    return Sketch(out, keep=g)


def skis_sketch_set_option(s: Sketch, option: int, value: int):
    _check(lib().skis_sketch_set_option(s.ptr, int(option), int(value)))


def skis_sketch_autotune(s: Sketch, pilot_samples: int, stream=None) -> dict:
    """Pick the fastest tier split on a pilot; returns the choice and the
    pilot time of every candidate."""
    d, m, nc = ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_int32()
    ms = np.zeros(32, np.float64)
    _check(lib().skis_sketch_autotune(s.ptr, int(pilot_samples), ctypes.byref(d), ctypes.byref(m),
                                      ctypes.c_void_p(ms.ctypes.data), 32, ctypes.byref(nc), _stream(stream)))
    return dict(max_deg=d.value, max_steps=m.value, warp_max_coins=skis_sketch_stats(s)["warp_max_coins"],
                candidate_ms=ms[: nc.value].tolist())


def skis_sample(s: Sketch, count: int, stream=None) -> int:
    nxt = ctypes.c_uint64()
    _check(lib().skis_sample(s.ptr, int(count), ctypes.byref(nxt), _stream(stream)))
    return nxt.value


def skis_sample_to_size(s: Sketch, target_entries: int, max_count: int = 1 << 40, stream=None):
    """Append samples until their total size reaches target_entries; returns
    (samples appended, new T)."""
    app, nxt = ctypes.c_uint64(), ctypes.c_uint64()
    _check(lib().skis_sample_to_size(s.ptr, int(target_entries), int(max_count), ctypes.byref(app),
                                     ctypes.byref(nxt), _stream(stream)))
    return app.value, nxt.value


def skis_estimate(s: Sketch, seed_offsets, seeds, coverage_out=None, estimate_out=None, stream=None):
    """Eq. 21 for a batch of seed sets (CSR). Host arrays in -> numpy out;
    device tensors in -> the caller's device output tensors are filled."""
    po, so = _ptr(seed_offsets, np.int64)
    pz, sz = _ptr(seeds, np.int32)
    q = _check_queries(seed_offsets, seeds, coverage_out, estimate_out)
    space = _space(so, sz)
    if estimate_out is None:
        if space == SKIS_MEM_DEVICE:
            raise ValueError("device queries need device output tensors")
        estimate_out = np.empty(q, np.float64)
        coverage_out = np.empty(q, np.int64) if coverage_out is None else coverage_out
    pe, se = _ptr(estimate_out, np.float64)
    pc, sc = _ptr(coverage_out, np.int64)
    if _space(space, se, sc) != space:
        raise ValueError("outputs must be in the memory space of the queries")
    _check(lib().skis_estimate(s.ptr, q, po, pz, pc, pe, space, _stream(stream)))
    return coverage_out, estimate_out


def skis_greedy_maxcover(s: Sketch, k: int, stream=None):
    seeds = np.empty(k, np.int32)
    cov = np.empty(k, np.int64)
    est = np.empty(k, np.float64)
    _check(lib().skis_greedy_maxcover(s.ptr, int(k), ctypes.c_void_p(seeds.ctypes.data),
                                      ctypes.c_void_p(cov.ctypes.data), ctypes.c_void_p(est.ctypes.data),
                                      _stream(stream)))
    return seeds, cov, est


def skis_sketch_stats(s: Sketch) -> dict:
    st = skis_stats()
    _check(lib().skis_sketch_stats(s.ptr, ctypes.byref(st)))
    return st.as_dict()


def skis_sketch_export(s: Sketch, first_id: int, count: int, stream=None) -> dict:
    a = dict(src=np.empty(count, np.int32), retries=np.empty(count, np.uint32), len=np.empty(count, np.uint32),
             coins=np.empty(count, np.uint64), member_off=np.empty(count + 1, np.int64))
    P = lambda k: ctypes.c_void_p(a[k].ctypes.data)  # noqa: E731
    st = _stream(stream)
    _check(lib().skis_sketch_export(s.ptr, int(first_id), int(count), P("src"), P("retries"), P("len"),
                                    P("coins"), P("member_off"), None, 0, st))
    total = int(a["member_off"][-1])
    a["members"] = np.empty(max(total, 1), np.int32)
    _check(lib().skis_sketch_export(s.ptr, int(first_id), int(count), None, None, None, None, None,
                                    ctypes.c_void_p(a["members"].ctypes.data), total, st))
    a["members"] = a["members"][:total]
    return a


def skis_sketch_free(s: Sketch):
    s.close()


def skis_estimate_noalloc(s: Sketch, seed_offsets, seeds, coverage_out, estimate_out, stream=None):
    """skis_estimate for callers that cannot allocate: device tensors in and
    out, at most 64 queries, graphs of at most 2^20 vertices; the library's
    static scratch array is used instead of any allocation."""
    po, so = _ptr(seed_offsets, np.int64)
    pz, sz = _ptr(seeds, np.int32)
    pc, sc = _ptr(coverage_out, np.int64)
    pe, se = _ptr(estimate_out, np.float64)
    if estimate_out is None:
        raise ValueError("skis_estimate_noalloc needs an estimate_out tensor")
    q = _check_queries(seed_offsets, seeds, coverage_out, estimate_out)
    if _space(so, sz, sc, se) != SKIS_MEM_DEVICE:
        raise ValueError("skis_estimate_noalloc takes device tensors only")
    buf = ctypes.create_string_buffer(256)
    rc = lib().skis_estimate_noalloc(s.ptr, q, po, pz, pc, pe, buf, 256, _stream(stream))
    if rc != SKIS_OK:
        raise SkisError(rc, buf.value.decode())
    return coverage_out, estimate_out


def skis_dssa_maxinf(g: Graph, seed_r: int, seed_rc: int, k: int, eps: float, delta: float, lambda2: int = 0,
                     n0: int = 1 << 12, n_max: int = 1 << 24, stream=None):
    """DSSA-style doubling influence maximisation; returns (seeds, result dict)."""
    seeds = np.empty(k, np.int32)
    res = skis_dssa_result()
    _check(lib().skis_dssa_maxinf(g.ptr, int(seed_r), int(seed_rc), int(k), float(eps), float(delta), int(lambda2),
                                  int(n0), int(n_max), ctypes.c_void_p(seeds.ctypes.data), ctypes.byref(res),
                                  _stream(stream)))
    return seeds, {f: getattr(res, f) for f, _ in res._fields_}


def skis_server_create(s: Sketch, slots: int = 4, max_batch: int = 64, seed_capacity: int = 1 << 16) -> Server:
    out = ctypes.c_void_p()
    _check(lib().skis_server_create(ctypes.byref(out), s.ptr, int(slots), int(max_batch), int(seed_capacity)))
    return Server(out, keep=s)


def skis_server_submit(srv: Server, seeds) -> int:
    seeds = np.ascontiguousarray(seeds, dtype=np.int32)
    t = ctypes.c_uint64()
    _check(lib().skis_server_submit(srv.ptr, ctypes.c_void_p(seeds.ctypes.data), int(seeds.shape[0]),
                                    ctypes.byref(t)))
    return t.value


def skis_server_progress(srv: Server, wait: bool = False) -> np.ndarray:
    """Retire finished batches and launch new ones; returns completed tickets."""
    nd = ctypes.c_int32()
    buf = srv._done
    _check(lib().skis_server_progress(srv.ptr, 1 if wait else 0, ctypes.c_void_p(buf.ctypes.data),
                                      int(buf.shape[0]), ctypes.byref(nd)))
    return buf[: nd.value].copy()


def skis_server_poll(srv: Server, ticket: int):
    """(state, coverage, estimate); state 0 pending, 1 ready, 2 failed."""
    c, e, st = ctypes.c_int64(), ctypes.c_double(), ctypes.c_int32()
    _check(lib().skis_server_poll(srv.ptr, int(ticket), ctypes.byref(c), ctypes.byref(e), ctypes.byref(st)))
    return st.value, c.value, e.value


def skis_server_counts(srv: Server) -> dict:
    v = [ctypes.c_uint64() for _ in range(4)]
    _check(lib().skis_server_counts(srv.ptr, *[ctypes.byref(x) for x in v]))
    return dict(queued=v[0].value, in_flight=v[1].value, batches=v[2].value, served=v[3].value)


def skis_server_free(srv: Server):
    srv.close()


# ----------------------------------------------------------- sharded sketch
ALLREDUCE_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p)


def _allreduce_cb(allreduce):
    """C callback around allreduce(count): it must sum the caller's exchange
    tensor's first count entries over the ranks in place; an exception is
    reported to the library as a failure."""

    def cb(ctx, buf, count, stream):
        try:
            allreduce(int(count))
            return 0
        except Exception:  # noqa: BLE001 - any failure of the caller's collective
            return 1

    return ALLREDUCE_FN(cb)


def _check_exchange(exchange, need: int):
    if not _is_torch(exchange) or not exchange.is_cuda or exchange.dtype.itemsize != 8 or not exchange.is_contiguous():
        raise TypeError("exchange must be a contiguous int64 CUDA tensor")
    if exchange.numel() < need:
        raise ValueError(f"exchange holds {exchange.numel()} entries, {need} are needed")
    _check_current_device(exchange)


def skis_estimate_sharded(s: Sketch, seed_offsets, seeds, exchange, allreduce, coverage_out=None,
                          estimate_out=None, stream=None):
    """Eq. 21 over a sketch split by sample id across ranks; exchange: int64
    CUDA tensor of >= q + 1 entries that allreduce(count) sums in place."""
    po, so = _ptr(seed_offsets, np.int64)
    pz, sz = _ptr(seeds, np.int32)
    q = _check_queries(seed_offsets, seeds, coverage_out, estimate_out)
    _check_exchange(exchange, q + 1)
    space = _space(so, sz)
    if estimate_out is None:
        if space == SKIS_MEM_DEVICE:
            raise ValueError("device queries need device output tensors")
        estimate_out = np.empty(q, np.float64)
        coverage_out = np.empty(q, np.int64) if coverage_out is None else coverage_out
    pe, se = _ptr(estimate_out, np.float64)
    pc, sc = _ptr(coverage_out, np.int64)
    if _space(space, se, sc) != space:
        raise ValueError("outputs must be in the memory space of the queries")
    cb = _allreduce_cb(allreduce)
    _check(lib().skis_estimate_sharded(s.ptr, q, po, pz, pc, pe, space, ctypes.c_void_p(exchange.data_ptr()), cb,
                                       None, _stream(stream)))
    return coverage_out, estimate_out


def skis_greedy_maxcover_sharded(s: Sketch, k: int, exchange, allreduce, stream=None):
    """Alg. 3 over a sketch split by sample id across ranks; exchange: int64
    CUDA tensor of >= n + 1 entries that allreduce(count) sums in place."""
    n = skis_graph_get_info(s._keep)["n"]
    _check_exchange(exchange, n + 1)
    seeds = np.empty(k, np.int32)
    cov = np.empty(k, np.int64)
    est = np.empty(k, np.float64)
    cb = _allreduce_cb(allreduce)
    _check(lib().skis_greedy_maxcover_sharded(s.ptr, int(k), ctypes.c_void_p(seeds.ctypes.data),
                                              ctypes.c_void_p(cov.ctypes.data), ctypes.c_void_p(est.ctypes.data),
                                              ctypes.c_void_p(exchange.data_ptr()), cb, None, _stream(stream)))
    return seeds, cov, est


def skis_philox_rate(seed: int, threads: int, blocks_per_thread: int, form: int, stream=None):
    """(device ms, XOR of every coin word) of the coin-generator probe."""
    ms, fold = ctypes.c_double(), ctypes.c_uint32()
    _check(lib().skis_philox_rate(int(seed), int(threads), int(blocks_per_thread), int(form), ctypes.byref(ms),
                                  ctypes.byref(fold), _stream(stream)))
    return ms.value, fold.value


def skis_kernel_launches() -> int:
    return int(lib().skis_kernel_launches())


def skis_device_allocations() -> int:
    return int(lib().skis_device_allocations())


def skis_last_error() -> str:
    return lib().skis_last_error().decode()
