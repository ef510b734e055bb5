"""SKIS on GB300: importance sketching of influence dynamics (arXiv 1709.03565).

The hot path — IIS sampling of non-singular reverse-reachable sets (Alg. 1),
coverage counting with the SKIS estimator (Eq. 21) and greedy max-coverage
(Alg. 3) — runs in hand-written sm_103a CUDA kernels behind the C ABI of
``include/skis.h`` (``libskis.so``). This package is its thin Python binding
(same entry-point names); PyTorch, where used, only supplies device memory
and streams.
"""
from ._binding import *  # noqa: F401,F403
from ._binding import lib, LIB_PATH, SkisError, Graph, Sketch, Server  # noqa: F401


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile ``libskis.so`` in-tree for sm_103a."""
    from ._build import build as _b

    return _b(force=force, verbose=verbose)
