"""SKIS oracle — TEST INFRASTRUCTURE ONLY.

A plain single-threaded CPU restatement of the SKIS method (arXiv 1709.03565:
Eq. gamma_v, Eq. probu, Alg. 1, Eq. 21, Alg. 3), written in C in
``skis_oracle.c`` and wrapped here with ctypes. It shares no code with the
CUDA library. Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import it; the product path never does.

Every function is pinned by ``-m "not gpu"`` tests against what the paper and
the mathematics fix (exact enumeration of live-edge worlds, closed forms,
invariants, statistical bounds, brute force); none is "parity unpinned".
"""
from .oracle import (  # noqa: F401
    build,
    philox4x32_10,
    OracleGraph,
    OracleSketch,
    ORC_OK,
    ORC_EINVAL,
    ORC_ENOMEM,
    ORC_ERETRY,
    W_P,
    W_TAU,
    W_WC,
    W_TRI,
    SENT,
    OracleError,
)
