"""The binding refuses, before any launch, query buffers that the library
would read or write past their ends (q estimates and coverage counts are
written, seeds [0, seed_offsets[q]) are read), and non-device tensors for the
entry point that takes device pointers only. No GPU and no library call is
needed for any of these."""
import numpy as np
import pytest

import paper_1709_03565_gb300 as skis

SK = skis.Sketch(None)  # never reached: every call below fails in the binding


def _q(sizes):
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    return off, np.arange(int(off[-1]), dtype=np.int32)


@pytest.mark.parametrize("case", ["short_est", "short_cov", "short_seeds", "empty_offsets"])
def test_estimate_rejects_short_buffers(case):
    off, seeds = _q([3, 2, 4])
    cov, est = np.empty(3, np.int64), np.empty(3, np.float64)
    if case == "short_est":
        est = np.empty(2, np.float64)
    elif case == "short_cov":
        cov = np.empty(1, np.int64)
    elif case == "short_seeds":
        seeds = seeds[:8]
    else:
        off = np.zeros(0, np.int64)
    with pytest.raises(ValueError):
        skis.skis_estimate(SK, off, seeds, cov, est)


@pytest.mark.parametrize("case", ["short_est", "short_cov", "short_seeds", "host_tensors", "no_est"])
def test_noalloc_rejects_bad_buffers(case):
    torch = pytest.importorskip("torch")
    off, seeds = _q([3, 2, 4])
    t_off, t_seeds = torch.from_numpy(off), torch.from_numpy(seeds)
    cov = torch.empty(3, dtype=torch.int64)
    est = torch.empty(3, dtype=torch.float64)
    if case == "short_est":
        est = torch.empty(2, dtype=torch.float64)
    elif case == "short_cov":
        cov = torch.empty(2, dtype=torch.int64)
    elif case == "short_seeds":
        t_seeds = t_seeds[:5]
    elif case == "no_est":
        est = None
    # host_tensors: right sizes, but host memory where device pointers are required
    with pytest.raises(ValueError):
        skis.skis_estimate_noalloc(SK, t_off, t_seeds, cov, est)


def test_sharded_calls_reject_bad_exchange():
    torch = pytest.importorskip("torch")
    off, seeds = _q([3, 2])
    with pytest.raises(TypeError):  # a host tensor is not a device exchange buffer
        skis.skis_estimate_sharded(SK, off, seeds, torch.zeros(3, dtype=torch.int64), lambda c: None)
    with pytest.raises(TypeError):
        skis.skis_estimate_sharded(SK, off, seeds, np.zeros(3, np.int64), lambda c: None)
