"""The coin-generator probe behind the benchmark's measured ALU ceiling draws
the Philox4x32-10 blocks it says it does: the XOR of all its coin words
equals the XOR over the oracle's Philox blocks (BFS domain, counter
(q, 3 << 28, t, 0), key = the seed), in both of its forms (every block in
full, and with the hub loop's per-sample hoisting), with and without a
remainder after its four-block steps."""
import numpy as np
import pytest

import oracle
import paper_1709_03565_gb300 as skis

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    skis.build()


@pytest.mark.parametrize("seed,per", [(0x5EED0003, 16), (0xFFFFFFFF00000001, 7)])
def test_probe_folds_the_oracles_coins(seed, per):
    threads = 48
    key = np.array([seed & 0xFFFFFFFF, seed >> 32], np.uint32)
    want = 0
    for t in range(threads):
        for k in range(per):
            x = oracle.philox4x32_10(np.array([t * per + k, 3 << 28, t, 0], np.uint32), key)
            for word in x:
                want ^= int(word)
    for form in (0, 1):
        ms, fold = skis.skis_philox_rate(seed, threads, per, form)
        assert fold == want and ms > 0
