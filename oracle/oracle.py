"""ctypes front end of the SKIS oracle (``skis_oracle.c``). Test infrastructure."""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "skis_oracle.c")
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIB_DIR, "libskis_oracle.so")
_lock = threading.Lock()
_handle = None

ORC_OK, ORC_EINVAL, ORC_ENOMEM, ORC_ERETRY = 0, 1, 2, 4
W_P, W_TAU, W_WC, W_TRI = 0, 1, 2, 3
SENT = 0xFFFFFFFF


class OracleError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: oracle status {code}")
        self.code = code


def build(force: bool = False) -> str:
    """Compile the oracle (plain C, -O2, single-threaded) into ``_build/``."""
    with _lock:
        fresh = os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)
        if force or not fresh:
            os.makedirs(_LIB_DIR, exist_ok=True)
            tmp = _LIB + f".{os.getpid()}.tmp"
            subprocess.check_call(["gcc", "-O2", "-shared", "-fPIC", "-Wall", "-o", tmp, _SRC])
            os.replace(tmp, _LIB)
    return _LIB


def _lib():
    global _handle
    if _handle is None:
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        i64, u64, i32, u32 = ctypes.c_int64, ctypes.c_uint64, ctypes.c_int32, ctypes.c_uint32
        lib.orc_philox4x32_10.argtypes = [P, P, P]
        lib.orc_philox4x32_10.restype = None
        lib.orc_graph_build.argtypes = [i64, i64, P, P, P, ctypes.c_int, u64, ctypes.POINTER(P)]
        lib.orc_graph_build.restype = ctypes.c_int
        lib.orc_graph_build_model.argtypes = [i64, i64, P, P, P, ctypes.c_int, u64, ctypes.c_int,
                                              ctypes.POINTER(P)]
        lib.orc_graph_build_model.restype = ctypes.c_int
        lib.orc_graph_free.argtypes = [P]
        lib.orc_graph_free.restype = None
        lib.orc_graph_scalars.argtypes = [P, P, P, P, P]
        lib.orc_graph_scalars.restype = None
        lib.orc_graph_arrays.argtypes = [P] * 8
        lib.orc_graph_arrays.restype = None
        lib.orc_sample_ids.argtypes = [P, u64, P, i64, u32, ctypes.c_int, P, P, P, P, P, P, i64, P]
        lib.orc_sample_ids.restype = ctypes.c_int
        lib.orc_sketch_build.argtypes = [P, u64, i64, u32, ctypes.c_int, ctypes.POINTER(P)]
        lib.orc_sketch_build.restype = ctypes.c_int
        lib.orc_sketch_build_to_size.argtypes = [P, u64, i64, i64, u32, ctypes.c_int, ctypes.POINTER(P)]
        lib.orc_sketch_build_to_size.restype = ctypes.c_int
        lib.orc_sketch_count.argtypes = [P]
        lib.orc_sketch_count.restype = i64
        lib.orc_sketch_free.argtypes = [P]
        lib.orc_sketch_free.restype = None
        lib.orc_sketch_entries.argtypes = [P]
        lib.orc_sketch_entries.restype = i64
        lib.orc_sketch_arrays.argtypes = [P] * 6
        lib.orc_sketch_arrays.restype = None
        lib.orc_coverage.argtypes = [P, i32, P, P, P, P, P, P]
        lib.orc_coverage.restype = ctypes.c_int
        lib.orc_greedy.argtypes = [P, i32, P, P, P]
        lib.orc_greedy.restype = ctypes.c_int
        _handle = lib
    return _handle


def _flags(ris: bool, bucket: bool) -> int:
    """Sampler flags: 1 = plain RIS, 2 = bucket first step."""
    return (1 if ris else 0) | (2 if bucket else 0)


def _p(a):
    return None if a is None else ctypes.c_void_p(a.ctypes.data)


def philox4x32_10(ctr, key) -> np.ndarray:
    """Philox4x32-10 block for a 4-word counter and a 2-word key."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.empty(4, np.uint32)
    _lib().orc_philox4x32_10(_p(c), _p(k), _p(out))
    return out


class OracleGraph:
    """G = (V, E, w) with canonical in-CSR, thresholds, fixed-point gamma and
    the alias table of the source law; lt=True reads the weights under the
    Linear Threshold model (gamma_v = the row's weight sum)."""

    def __init__(self, n, src, dst, weights=None, model=W_WC, weight_seed=0, lt=False):
        src = np.ascontiguousarray(src, dtype=np.int32)
        dst = np.ascontiguousarray(dst, dtype=np.int32)
        m = int(src.shape[0])
        if model == W_P:
            weights = np.ascontiguousarray(weights, dtype=np.float64)
        elif model == W_TAU:
            weights = np.ascontiguousarray(weights, dtype=np.uint32)
        else:
            weights = None
        h = ctypes.c_void_p()
        rc = _lib().orc_graph_build_model(n, m, _p(src), _p(dst), _p(weights), model, weight_seed,
                                          1 if lt else 0, ctypes.byref(h))
        if rc != ORC_OK:
            raise OracleError(rc, "orc_graph_build")
        self._h = h
        nn, mm, W, f = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_uint64(), ctypes.c_int32()
        _lib().orc_graph_scalars(h, ctypes.byref(nn), ctypes.byref(mm), ctypes.byref(W),
                                 ctypes.byref(f))
        self.n, self.m, self.W, self.f = nn.value, mm.value, W.value, f.value

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            _lib().orc_graph_free(h)
            self._h = None

    def arrays(self, keys=("off", "src", "tau", "perm", "w", "prob", "alias")) -> dict:
        """The graph's arrays (those named in keys)."""
        n, m = self.n, self.m
        shapes = dict(off=(n + 1, np.int64), src=(m, np.int32), tau=(m, np.uint32), perm=(m, np.int64),
                      w=(n, np.uint64), prob=(n, np.uint64), alias=(n, np.uint32))
        a = {k: np.empty(shapes[k][0], shapes[k][1]) for k in keys}
        _lib().orc_graph_arrays(self._h, *[_p(a.get(k)) for k in ("off", "src", "tau", "perm", "w", "prob", "alias")])
        return a

    def sample_ids(self, seed, ids, retry_cap=1 << 24, members_cap=None, ris=False, bucket=False):
        """Samples for explicit ids: dict of per-sample arrays plus the
        concatenated members (insertion order) and their offsets."""
        ids = np.ascontiguousarray(ids, dtype=np.uint64)
        c = int(ids.shape[0])
        cap = members_cap if members_cap is not None else max(1024, 64 * c)
        while True:
            out = dict(src=np.empty(c, np.int32), retries=np.empty(c, np.uint32),
                       len=np.empty(c, np.int64), coins=np.empty(c, np.uint64),
                       status=np.empty(c, np.int32))
            mem = np.empty(cap, np.int32)
            used = ctypes.c_int64()
            rc = _lib().orc_sample_ids(self._h, seed, _p(ids), c, retry_cap, _flags(ris, bucket), _p(out["src"]),
                                       _p(out["retries"]), _p(out["len"]), _p(out["coins"]),
                                       _p(out["status"]), _p(mem), cap, ctypes.byref(used))
            if rc == ORC_ENOMEM and members_cap is None:
                cap *= 4
                continue
            if rc != ORC_OK:
                raise OracleError(rc, "orc_sample_ids")
            break
        out["members"] = mem[: used.value].copy()
        out["member_off"] = np.concatenate([[0], np.cumsum(out["len"])]).astype(np.int64)
        return out


class OracleSketch:
    """The SKIS sketch R = {R_1..R_T} (sample ids 0..T-1) with Eq. 21 queries
    and Alg. 3 greedy."""

    def __init__(self, graph: OracleGraph, seed: int, T: int, retry_cap: int = 1 << 24, ris: bool = False,
                 stop_entries: int = 0, bucket: bool = False):
        """T samples; with stop_entries > 0, the first samples whose total
        size reaches stop_entries (T bounds the count)."""
        h = ctypes.c_void_p()
        if stop_entries > 0:
            rc = _lib().orc_sketch_build_to_size(graph._h, seed, stop_entries, T, retry_cap, _flags(ris, bucket),
                                                 ctypes.byref(h))
        else:
            rc = _lib().orc_sketch_build(graph._h, seed, T, retry_cap, _flags(ris, bucket), ctypes.byref(h))
        if rc != ORC_OK:
            raise OracleError(rc, "orc_sketch_build")
        self._h = h
        self.graph = graph
        self.T = int(_lib().orc_sketch_count(h))
        self.seed = seed

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            _lib().orc_sketch_free(h)
            self._h = None

    def arrays(self) -> dict:
        T = self.T
        E = _lib().orc_sketch_entries(self._h)
        a = dict(off=np.empty(T + 1, np.int64), mem=np.empty(E, np.int32),
                 src=np.empty(T, np.int32), retries=np.empty(T, np.uint32),
                 coins=np.empty(T, np.uint64))
        _lib().orc_sketch_arrays(self._h, _p(a["off"]), _p(a["mem"]), _p(a["src"]),
                                 _p(a["retries"]), _p(a["coins"]))
        return a

    def coverage(self, seed_off, seeds, exact=False):
        seed_off = np.ascontiguousarray(seed_off, dtype=np.int64)
        seeds = np.ascontiguousarray(seeds, dtype=np.int32)
        q = int(seed_off.shape[0]) - 1
        cov = np.empty(q, np.int64)
        est = np.empty(q, np.float64)
        num = np.empty(2 * q, np.uint64)
        den = np.empty(2 * q, np.uint64)
        rc = _lib().orc_coverage(self._h, q, _p(seed_off), _p(seeds), _p(cov), _p(est),
                                 _p(num), _p(den))
        if rc != ORC_OK:
            raise OracleError(rc, "orc_coverage")
        if not exact:
            return cov, est
        N = [int(num[2 * b]) | (int(num[2 * b + 1]) << 64) for b in range(q)]
        D = [int(den[2 * b]) | (int(den[2 * b + 1]) << 64) for b in range(q)]
        return cov, est, N, D

    def greedy(self, k: int):
        seeds = np.empty(k, np.int32)
        cov = np.empty(k, np.int64)
        est = np.empty(k, np.float64)
        rc = _lib().orc_greedy(self._h, k, _p(seeds), _p(cov), _p(est))
        if rc != ORC_OK:
            raise OracleError(rc, "orc_greedy")
        return seeds, cov, est
