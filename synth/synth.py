"""ctypes front end of the synthetic input generators (``gen.c``)."""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gen.c")
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIB_DIR, "libskisgen.so")
_lock = threading.Lock()
_handle = None


def build(force: bool = False) -> str:
    """Compile ``gen.c`` into ``_build/libskisgen.so`` (host C, OpenMP)."""
    with _lock:
        fresh = os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)
        if force or not fresh:
            os.makedirs(_LIB_DIR, exist_ok=True)
            tmp = _LIB + f".{os.getpid()}.tmp"
            subprocess.check_call(
                ["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-Wall", "-o", tmp, _SRC, "-lm"]
            )
            os.replace(tmp, _LIB)
    return _LIB


def _lib():
    global _handle
    if _handle is None:
        lib = ctypes.CDLL(build())
        i64, u64, i32, dbl, ptr = (ctypes.c_int64, ctypes.c_uint64, ctypes.c_int32,
                                   ctypes.c_double, ctypes.c_void_p)
        lib.synth_er.argtypes = [i64, i64, u64, ptr, ptr]
        lib.synth_chunglu.argtypes = [i64, i64, dbl, u64, ptr, ptr]
        lib.synth_rmat.argtypes = [ctypes.c_int, i64, dbl, dbl, dbl, u64, ptr, ptr]
        lib.synth_tri.argtypes = [i64, u64, ptr]
        lib.synth_uniform_p.argtypes = [i64, u64, dbl, dbl, ptr]
        lib.synth_seed_sets.argtypes = [i64, i32, ptr, u64, ptr, ptr]
        for f in (lib.synth_er, lib.synth_chunglu, lib.synth_rmat, lib.synth_tri,
                  lib.synth_uniform_p, lib.synth_seed_sets):
            f.restype = ctypes.c_int
        _handle = lib
    return _handle


def _p(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


def er(n: int, m: int, seed: int):
    """Directed Erdos-Renyi: m distinct ordered pairs (u != v), uniform."""
    src = np.empty(m, np.int32)
    dst = np.empty(m, np.int32)
    if _lib().synth_er(n, m, seed, _p(src), _p(dst)) != 0:
        raise ValueError("synth_er: bad arguments")
    return src, dst


def chunglu(n: int, m: int, beta: float, seed: int):
    """Directed Chung-Lu with expected-degree exponent ``beta``; max expected
    degree sqrt(m); self-loops redrawn, parallel edges kept."""
    src = np.empty(m, np.int32)
    dst = np.empty(m, np.int32)
    if _lib().synth_chunglu(n, m, beta, seed, _p(src), _p(dst)) != 0:
        raise ValueError("synth_chunglu: bad arguments")
    return src, dst


def rmat(scale: int, m: int, a: float, b: float, c: float, seed: int):
    """R-MAT over 2^scale vertices with quadrant probabilities (a, b, c, 1-a-b-c)."""
    src = np.empty(m, np.int32)
    dst = np.empty(m, np.int32)
    if _lib().synth_rmat(scale, m, a, b, c, seed, _p(src), _p(dst)) != 0:
        raise ValueError("synth_rmat: bad arguments")
    return src, dst


def tri(m: int, seed: int) -> np.ndarray:
    """Trivalency edge probabilities, uniform over {0.1, 0.01, 0.001}."""
    p = np.empty(m, np.float64)
    _lib().synth_tri(m, seed, _p(p))
    return p


def uniform_p(m: int, seed: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
    """Edge probabilities uniform in [lo, hi) (used by tests)."""
    p = np.empty(m, np.float64)
    _lib().synth_uniform_p(m, seed, lo, hi, _p(p))
    return p


def seed_sets(n: int, sizes, seed: int):
    """Seed sets of the given sizes, each uniform without replacement.

    Returns ``(offsets int64[q+1], seeds int32[sum(sizes)])``."""
    sizes = np.ascontiguousarray(sizes, dtype=np.int32)
    q = int(sizes.shape[0])
    off = np.empty(q + 1, np.int64)
    seeds = np.empty(int(sizes.sum()), np.int32)
    if _lib().synth_seed_sets(n, q, _p(sizes), seed, _p(off), _p(seeds)) != 0:
        raise ValueError("synth_seed_sets: bad arguments")
    return off, seeds


def log_uniform_sizes(q: int, lo: int, hi: int, seed: int) -> np.ndarray:
    """Query sizes floor(10^U) with U uniform on [log10 lo, log10 hi], clamped."""
    rng = np.random.Generator(np.random.PCG64(seed))
    u = rng.uniform(np.log10(lo), np.log10(hi), size=q)
    return np.clip(np.floor(10.0 ** u), lo, hi).astype(np.int32)


# Workloads: the five configurations the benchmark and the parity tests use.
WORKLOADS = {
    "er-1e4-wc": dict(kind="er", n=10_000, m=100_000, seed=1, model="wc",
                      samples=100_000, queries=100, query_size=10),
    "chunglu-1e6-tri": dict(kind="chunglu", n=1_000_000, m=10_000_000, beta=2.1, seed=2,
                            model="tri", samples=10_000_000, k=50),
    "rmat-2^25-wc": dict(kind="rmat", scale=25, n=1 << 25, m=1 << 30, abc=(0.57, 0.19, 0.19),
                         seed=3, model="wc", samples=100_000_000),
    "chunglu-4e6-wc-serve": dict(kind="chunglu", n=4_000_000, m=70_000_000, beta=2.1, seed=4,
                                 model="wc", samples=20_000_000),
    "chunglu-4e7-wc-dssa": dict(kind="chunglu", n=40_000_000, m=1_400_000_000, beta=2.0,
                                seed=5, model="wc"),
}


def workload(name: str):
    """Generate the edge list (and TRI probabilities) of a named workload.

    Returns ``(spec, src, dst, p)`` where ``p`` is None for weighted cascade."""
    spec = dict(WORKLOADS[name])
    kind = spec["kind"]
    if kind == "er":
        src, dst = er(spec["n"], spec["m"], spec["seed"])
    elif kind == "chunglu":
        src, dst = chunglu(spec["n"], spec["m"], spec["beta"], spec["seed"])
    elif kind == "rmat":
        a, b, c = spec["abc"]
        src, dst = rmat(spec["scale"], spec["m"], a, b, c, spec["seed"])
    else:
        raise KeyError(kind)
    p = tri(spec["m"], spec["seed"] + 1000) if spec["model"] == "tri" else None
    return spec, src, dst, p
