"""Stop-at-size sketches (sample until the total size reaches a target, the
rule of the paper's experiments, Sec. VI "Algorithms compared"): the oracle's
stopping count is the one numpy's searchsorted finds on the cumulative sizes
of a fixed-count sketch, and its samples are that sketch's prefix."""
import numpy as np
import pytest

import oracle
import synth


@pytest.mark.parametrize("ris", [False, True])
def test_stop_count_is_the_first_reaching_prefix(ris):
    n = 2000
    src, dst = synth.chunglu(n, 16000, 2.1, 81)
    g = oracle.OracleGraph(n, src, dst, model=oracle.W_WC)
    seed = 0xABC
    full = oracle.OracleSketch(g, seed, 5000, ris=ris).arrays()
    cum = full["off"][1:]
    for target in (1, 2, 777, int(n * np.log(n)), int(cum[-1])):
        want = int(np.searchsorted(cum, target, side="left")) + 1
        sk = oracle.OracleSketch(g, seed, 5000, ris=ris, stop_entries=target)
        assert sk.T == want
        a = sk.arrays()
        assert np.array_equal(a["off"], full["off"][: want + 1])
        assert np.array_equal(a["mem"], full["mem"][: full["off"][want]])
        assert a["off"][-1] >= target and (want == 1 or a["off"][-2] < target)
    # an unreachable target stops at the sample bound
    assert oracle.OracleSketch(g, seed, 100, ris=ris, stop_entries=10**9).T == 100
