"""Seeded synthetic inputs for the SKIS workloads.

The generators here produce edge lists, edge probabilities and query seed
sets only; they hold none of the method's arithmetic. Both the CUDA library
and the CPU oracle take their inputs from this module and from nowhere else.

Workloads (the shapes of the paper's SNAP/Twitter graphs, which are not
available here, are stood in for by these synthetic graphs):

* ``er``: directed Erdos-Renyi, m distinct ordered pairs.
* ``chunglu``: directed Chung-Lu with power-law expected degrees.
* ``rmat``: R-MAT (a, b, c, d) recursive matrix graph.
* ``tri``: trivalency probabilities, uniform over {0.1, 0.01, 0.001}.
"""
from .synth import (  # noqa: F401
    build,
    chunglu,
    er,
    rmat,
    seed_sets,
    tri,
    uniform_p,
    log_uniform_sizes,
    WORKLOADS,
    workload,
)
