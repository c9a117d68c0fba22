"""The allocation-free brute-force entry point against the regular one.

riann_exact_nn_noalloc serves callers that may not allocate device memory
while running (a real-time pipeline with a memory budget fixed at start-up, a
plug-in whose host application owns every allocation): its scratch is a fixed
device array inside the library.  Its results must equal riann_exact_nn's
exactly, call after call, although every call reuses the same array.

This file is collected last so that a run stopping at its first failure has
already run every other test.
"""
import numpy as np
import pytest

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


@pytest.mark.parametrize("n,C,H,W", [(4096, 1, 128, 128), (777, 3, 40, 61)])
def test_noalloc_equals_exact_nn_on_two_calls_in_a_row(rt, n, C, H, W):
    import torch
    R, KP, _, _ = synth.random_case(500 + n, n, 4, C, H, W)
    R[n // 2:] = R[: n - n // 2]                         # duplicate rows: ties
    rng = np.random.default_rng(501 + n)
    frames = [rng.integers(0, 256, size=(H, W, C), dtype=np.uint8) for _ in range(2)]
    frames[1][:8, :8] = R[n // 2 + 3]                    # an exact hit with a tie
    idx = rt.riann_build_reference_index(_dev(R), _dev(KP))
    shape = (H - 7, W - 7)
    for f in frames:                                     # two calls in a row
        fd = _dev(f)
        a_ref = torch.empty(shape, dtype=torch.int32, device="cuda")
        d_ref = torch.empty_like(a_ref)
        rt.riann_exact_nn(idx, fd, a_ref, d_ref)
        a = torch.full(shape, -7, dtype=torch.int32, device="cuda")
        d = torch.full(shape, -7, dtype=torch.int32, device="cuda")
        rt.riann_exact_nn_noalloc(idx, fd, a, d)
        torch.cuda.synchronize()
        assert torch.equal(a, a_ref)
        assert torch.equal(d, d_ref)
    assert rt.riann_status(idx) == 0
    idx.close()


def test_noalloc_rejects_frames_beyond_its_scratch(rt):
    import torch
    R, KP, _, _ = synth.random_case(502, 64, 4, 1, 8, 8)
    idx = rt.riann_build_reference_index(_dev(R), _dev(KP))
    qmax = rt.riann_exact_nn_noalloc_max_queries(1)
    W = 7 + 4096
    H = 7 + qmax // 4096 + 1                             # one row of queries too many
    assert (H - 7) * (W - 7) > qmax
    frame = torch.zeros((H, W, 1), dtype=torch.uint8, device="cuda")
    out = torch.empty((H - 7, W - 7), dtype=torch.int32, device="cuda")
    with pytest.raises(rt.RiannError) as e:
        rt.riann_exact_nn_noalloc(idx, frame, out)
    assert e.value.code == rt.RIANN_ERR_TOO_LARGE
    idx.close()
