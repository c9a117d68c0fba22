"""Failure detection on the GPU without a fault: a bounded device wait that
runs out reports RIANN_DEV_TIMEOUT through the status word, the kernel
returns, and the context and the index keep working.

riann_test_wait_expiry runs the brute-force kernel with its copy producer
withholding every reference tile, so the MMA issuer's wait for the first one
(a barrier nothing completes) expires after a short limit instead of about a
second.
"""
import time

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rt():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1508_07953_gb300 import riann
    return riann


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("C", [1, 3])
def test_wait_expiry_sets_timeout_and_leaves_the_index_usable(rt, C):
    import torch
    R, KP, frame, _ = synth.random_case(700 + C, 1500, 8, C, 45, 300)
    idx = rt.riann_build_reference_index(_dev(R), _dev(KP))
    fd = _dev(frame)
    shape = (45 - 7, 300 - 7)
    out = torch.empty(shape, dtype=torch.int32, device="cuda")
    assert rt.riann_status(idx) == 0
    t0 = time.monotonic()
    rt.riann_test_wait_expiry(idx, fd, out, 200_000)          # ~0.1 ms of clock cycles
    bits = rt.riann_status(idx)                               # synchronises; clears the word
    waited = time.monotonic() - t0
    assert bits & rt.RIANN_DEV_TIMEOUT, f"status {bits:#x}"
    assert waited < 2.0                                       # the short limit, not the default
    # the next normal calls on the same index and context are exact
    a = torch.empty(shape, dtype=torch.int32, device="cuda")
    d = torch.empty(shape, dtype=torch.int32, device="cuda")
    rt.riann_exact_nn(idx, fd, a, d)
    want_a, want_d, _ = oracle.exact_nn(frame, R)
    assert np.array_equal(a.cpu().numpy(), want_a)
    assert np.array_equal(d.cpu().numpy().view(np.uint32), want_d)
    params = rt.riann_default_params(len(R))
    g = rt.annf(idx, fd, a, params)
    oix = oracle.Index(R, KP)
    o = oracle.riann_frame(oix, frame, want_a, ring_limit=params.ring_limit)
    assert np.array_equal(g[0].cpu().numpy(), o[0])
    assert np.array_equal(g[2].cpu().numpy().view(np.uint32), o[2])
    assert rt.riann_status(idx) == 0
    idx.close()


def test_wait_expiry_rejects_out_of_range_limits(rt):
    import torch
    R, KP, frame, _ = synth.random_case(710, 300, 4, 1, 16, 16)
    idx = rt.riann_build_reference_index(_dev(R), _dev(KP))
    out = torch.empty((9, 9), dtype=torch.int32, device="cuda")
    for bad in (0, 999, 2_000_000_001):
        with pytest.raises(rt.RiannError) as e:
            rt.riann_test_wait_expiry(idx, _dev(frame), out, bad)
        assert e.value.code == rt.RIANN_ERR_INVALID_ARG
    assert rt.riann_status(idx) == 0
    idx.close()
