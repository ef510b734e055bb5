"""skis_estimate_noalloc, the query entry point for callers that cannot
allocate device memory when they query (for instance when another allocator
already holds all of it): through the C ABI it must give the same coverage
counts (exactly) and estimates (relative 1e-12) as skis_estimate, on two
calls in a row, with its static scratch array in place of any allocation.

This file is named so that pytest collects it last."""
import ctypes

import numpy as np
import pytest

import paper_1709_03565_gb300 as skis
import synth

pytestmark = pytest.mark.gpu

REL = 1e-12


@pytest.fixture(scope="module")
def sketch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    skis.build()
    n, m = 20_000, 160_000
    src, dst = synth.chunglu(n, m, 2.1, 31)
    g = skis.skis_load_graph(n, src, dst, synth.tri(m, 31), skis.SKIS_W_EXPLICIT_P)
    s = skis.skis_sketch_create(g, 0x5EED0031)
    skis.skis_sample(s, 200_000)
    yield torch, n, g, s
    s.close()
    g.close()


def _device_queries(torch, n, sizes, seed):
    off, seeds = synth.seed_sets(n, sizes, seed)
    return off, seeds, torch.from_numpy(off).cuda(), torch.from_numpy(seeds).cuda()


def test_noalloc_matches_estimate_on_two_calls_in_a_row(sketch):
    torch, n, g, s = sketch
    # two different batches in a row: the second call must not see the first's state
    for seed, sizes in ((5, [10] * 64), (6, list(synth.log_uniform_sizes(40, 1, 1000, 6)))):
        off, seeds, d_off, d_seeds = _device_queries(torch, n, sizes, seed)
        q = len(sizes)
        cov_ref, est_ref = skis.skis_estimate(s, off, seeds)
        d_cov = torch.full((q,), -1, dtype=torch.int64, device="cuda")
        d_est = torch.full((q,), -1.0, dtype=torch.float64, device="cuda")
        # call through the C ABI directly
        buf = ctypes.create_string_buffer(256)
        stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        rc = skis.lib().skis_estimate_noalloc(s.ptr, q, ctypes.c_void_p(d_off.data_ptr()),
                                             ctypes.c_void_p(d_seeds.data_ptr()), ctypes.c_void_p(d_cov.data_ptr()),
                                             ctypes.c_void_p(d_est.data_ptr()), buf, 256, stream)
        assert rc == skis.SKIS_OK, buf.value
        assert np.array_equal(d_cov.cpu().numpy(), cov_ref)
        np.testing.assert_allclose(d_est.cpu().numpy(), est_ref, rtol=REL, atol=0)


def test_noalloc_makes_no_device_allocation(sketch):
    # the library counts every device allocation it makes: a warm call of the
    # entry point adds none (skis_estimate, for comparison, does)
    torch, n, g, s = sketch
    off, seeds, d_off, d_seeds = _device_queries(torch, n, [10] * 16, 9)
    d_cov = torch.empty(16, dtype=torch.int64, device="cuda")
    d_est = torch.empty(16, dtype=torch.float64, device="cuda")
    skis.skis_estimate_noalloc(s, d_off, d_seeds, d_cov, d_est)  # warm: the array's address is looked up
    before = skis.skis_device_allocations()
    for _ in range(3):
        skis.skis_estimate_noalloc(s, d_off, d_seeds, d_cov, d_est)
    assert skis.skis_device_allocations() == before
    skis.skis_estimate(s, off, seeds)
    assert skis.skis_device_allocations() > before


def test_noalloc_limits_are_rejected_with_a_message(sketch):
    torch, n, g, s = sketch
    off, seeds, d_off, d_seeds = _device_queries(torch, n, [3] * 65, 7)
    d_cov = torch.empty(65, dtype=torch.int64, device="cuda")
    d_est = torch.empty(65, dtype=torch.float64, device="cuda")
    with pytest.raises(skis.SkisError) as e:
        skis.skis_estimate_noalloc(s, d_off, d_seeds, d_cov, d_est)
    assert e.value.code == skis.SKIS_EINVAL and "64" in str(e.value)
    # a repeated seed is rejected like skis_estimate does
    bad_off = torch.tensor([0, 2], dtype=torch.int64, device="cuda")
    bad_seeds = torch.tensor([4, 4], dtype=torch.int32, device="cuda")
    with pytest.raises(skis.SkisError) as e:
        skis.skis_estimate_noalloc(s, bad_off, bad_seeds, d_cov[:1], d_est[:1])
    assert e.value.code == skis.SKIS_EINVAL and "query 0 " in str(e.value)
    # the same message as skis_estimate's, naming the failing query
    two_off = torch.tensor([0, 1, 3], dtype=torch.int64, device="cuda")
    two_seeds = torch.tensor([1, 7, 7], dtype=torch.int32, device="cuda")
    with pytest.raises(skis.SkisError) as e:
        skis.skis_estimate_noalloc(s, two_off, two_seeds, d_cov[:2], d_est[:2])
    with pytest.raises(skis.SkisError) as e2:
        skis.skis_estimate(s, two_off, two_seeds, d_cov[:2], d_est[:2])
    assert "query 1 " in str(e.value) and str(e.value).split(": ", 1)[1] == str(e2.value).split(": ", 1)[1]
    # graphs above 2^20 vertices exceed the static scratch
    big_n = (1 << 20) + 1
    g2 = skis.skis_load_graph(big_n, np.array([1, 2], np.int32), np.array([0, 0], np.int32))
    s2 = skis.skis_sketch_create(g2, 1)
    skis.skis_sample(s2, 10)
    one_off = torch.tensor([0, 1], dtype=torch.int64, device="cuda")
    one_seed = torch.tensor([0], dtype=torch.int32, device="cuda")
    with pytest.raises(skis.SkisError) as e:
        skis.skis_estimate_noalloc(s2, one_off, one_seed, d_cov[:1], d_est[:1])
    assert e.value.code == skis.SKIS_EINVAL and "2^20" in str(e.value)
    s2.close()
    g2.close()
    # and the entry point still answers correctly afterwards
    off, seeds, d_off, d_seeds = _device_queries(torch, n, [10] * 8, 8)
    cov_ref, est_ref = skis.skis_estimate(s, off, seeds)
    skis.skis_estimate_noalloc(s, d_off, d_seeds, d_cov[:8], d_est[:8])
    assert np.array_equal(d_cov[:8].cpu().numpy(), cov_ref)
    np.testing.assert_allclose(d_est[:8].cpu().numpy(), est_ref, rtol=REL, atol=0)
