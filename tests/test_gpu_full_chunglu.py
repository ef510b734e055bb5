"""Full-size parity on the largest graph of the workloads: the Chung-Lu graph
of the DSSA workload, 40M vertices and 1.4B edges (exponent 2.0, seed 5),
weighted cascade, loaded by the library and by the oracle. Graph structures
(Sec. II-A canonical in-CSR, Eq. gamma_v, Eq. probu) bit-exact: the CSR
source array is 5.6 GB, so both sides index past 2^32 bytes. Samples (Alg. 1,
bucket form) at ids [0, 200) and 20 blocks of 4 ids spread over 10^9."""
import numpy as np
import pytest

import oracle
import paper_1709_03565_gb300 as skis
import synth

from test_gpu_parity import assert_samples_equal

pytestmark = pytest.mark.gpu
SEED = 0x5EED0005


@pytest.fixture(scope="module")
def chunglu_dssa():
    """The Chung-Lu graph of the DSSA workload: 40M vertices, 1.4B edges
    (exponent 2.0, seed 5), weighted cascade, loaded by both sides."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    skis.build()
    spec, src, dst, _ = synth.workload("chunglu-4e7-wc-dssa")
    g = skis.skis_load_graph(spec["n"], src, dst, None, skis.SKIS_W_WC)
    o = oracle.OracleGraph(spec["n"], src, dst, model=oracle.W_WC)
    del src, dst
    yield spec, g, o
    g.close()


def test_full_chunglu_dssa_graph_and_samples(chunglu_dssa):
    # the CSR source array is 5.6 GB: host and device offsets past 2^32 bytes
    spec, g, o = chunglu_dssa
    info = skis.skis_graph_get_info(g)
    assert (info["n"], info["m"]) == (40_000_000, 1_400_000_000) and 4 * info["m"] > 1 << 32
    assert info["W"] == o.W and info["f"] == o.f
    for k in ("off", "src", "tau", "perm", "w", "prob", "alias"):
        a, b = skis.skis_graph_export(g, keys=(k,))[k], o.arrays(keys=(k,))[k]
        assert a.shape == b.shape and np.array_equal(a, b), k
        del a, b
    for first, count in [(0, 200)] + [(i * 50_000_000, 4) for i in range(1, 21)]:
        s = skis.skis_sketch_create(g, SEED)
        skis.skis_sketch_set_option(s, skis.SKIS_OPT_FIRST_STEP, 1)
        skis.skis_sketch_set_option(s, skis.SKIS_OPT_FIRST_ID, first)
        skis.skis_sample(s, count)
        assert_samples_equal(skis.skis_sketch_export(s, first, count),
                             o.sample_ids(SEED, np.arange(first, first + count, dtype=np.uint64), bucket=True))
        s.close()
