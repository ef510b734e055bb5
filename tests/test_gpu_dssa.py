"""DSSA-style doubling on the device against the oracle's independent driver:
the same rounds, stop reason, seed set, coverages, and bit-identical
estimates and error terms (both form them from exact integers)."""
import numpy as np
import pytest

import oracle
import paper_1709_03565_gb300 as skis
import synth
from oracle.dssa import dssa_maxinf

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    skis.build()


@pytest.mark.parametrize("model,k,eps", [("tri", 10, 0.3), ("wc", 25, 0.2), ("wc", 1, 0.5)])
def test_dssa_matches_the_oracle_driver(model, k, eps):
    n, m = 20_000, 160_000
    src, dst = synth.chunglu(n, m, 2.1, 51)
    if model == "tri":
        p = synth.tri(m, 51)
        g = skis.skis_load_graph(n, src, dst, p, skis.SKIS_W_EXPLICIT_P)
        og = oracle.OracleGraph(n, src, dst, weights=p, model=oracle.W_P)
    else:
        g = skis.skis_load_graph(n, src, dst, weight_model=skis.SKIS_W_WC)
        og = oracle.OracleGraph(n, src, dst, model=oracle.W_WC)
    kw = dict(n0=1024, n_max=1 << 17)
    ds, dr = skis.skis_dssa_maxinf(g, 11, 12, k, eps, 1.0 / n, **kw)
    os_, orr = dssa_maxinf(og, 11, 12, k, eps, 1.0 / n, **kw)
    assert np.array_equal(ds, os_)
    for key in ("rounds", "stopped_by", "samples", "lambda2", "coverage", "coverage_c",
                "estimate", "estimate_c", "eps1", "eps2", "eps3"):
        assert dr[key] == orr[key], key
    g.close()
