"""The allocation-free brute-force entry point against the regular one.

riann_exact_nn_noalloc serves callers that may not allocate device memory
while running (a real-time pipeline with a memory budget fixed at start-up, a
plug-in whose host application owns every allocation): its scratch is a fixed
device array inside the library.  Its results must equal riann_exact_nn's
exactly, call after call, although every call reuses the same array.

This file is collected last so that a run stopping at its first failure has
already run every other test.
"""
import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest

import oracle
import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

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
        # and the oracle's brute force itself (lowest index on ties)
        wa, wd, _ = oracle.exact_nn(f, R)
        assert np.array_equal(a.cpu().numpy(), wa)
        assert np.array_equal(d.cpu().numpy().view(np.uint32), wd)
    assert rt.riann_status(idx) == 0
    idx.close()


@pytest.mark.parametrize("C,n", [(1, 4096), (3, 777)])
def test_noalloc_at_exactly_its_limit(rt, C, n):
    # the largest frame it accepts: its last 128-row tile ends exactly at the
    # end of the fixed array and of the tensor map over it
    import torch
    qmax = rt.riann_exact_nn_noalloc_max_queries(C)
    assert qmax % 128 == 0
    H, W = 7 + 128, 7 + qmax // 128
    assert (H - 7) * (W - 7) == qmax
    R, KP, _, _ = synth.random_case(520 + C, n, 4, C, 8, 8)
    frame = np.random.default_rng(521 + C).integers(0, 256, size=(H, W, C), dtype=np.uint8)
    idx = rt.riann_build_reference_index(_dev(R), _dev(KP))
    fd = _dev(frame)
    a_ref = torch.empty((H - 7, W - 7), dtype=torch.int32, device="cuda")
    d_ref = torch.empty_like(a_ref)
    rt.riann_exact_nn(idx, fd, a_ref, d_ref)
    for _ in range(2):
        a = torch.full_like(a_ref, -7)
        d = torch.full_like(a_ref, -7)
        rt.riann_exact_nn_noalloc(idx, fd, a, d)
        torch.cuda.synchronize()
        assert torch.equal(a, a_ref) and torch.equal(d, d_ref)
    assert rt.riann_status(idx) == 0
    idx.close()


def test_noalloc_first_call_inside_a_capture_is_refused():
    # a fresh process: the per-device set-up has not run yet, so a call made
    # while the stream is capturing is refused; the next call outside the
    # capture does the set-up and answers exactly
    script = textwrap.dedent("""
        import sys
        sys.path.insert(0, %r)
        import numpy as np, torch
        import synth
        from paper_1508_07953_gb300 import riann as rt
        R, KP, frame, _ = synth.random_case(530, 500, 4, 1, 40, 50)
        idx = rt.riann_build_reference_index(torch.from_numpy(R).cuda(), torch.from_numpy(KP).cuda())
        f = torch.from_numpy(frame).cuda()
        out = torch.empty((33, 43), dtype=torch.int32, device="cuda")
        ref = torch.empty_like(out)
        rt.riann_exact_nn(idx, f, ref)
        torch.cuda.synchronize()
        s = torch.cuda.Stream()
        g = torch.cuda.CUDAGraph()
        code = None
        with torch.cuda.stream(s):
            g.capture_begin()
            try:
                rt.riann_exact_nn_noalloc(idx, f, out, stream=s)
            except rt.RiannError as e:
                code = e.code
            finally:
                g.capture_end()
        assert code == rt.RIANN_ERR_INVALID_ARG, code
        rt.riann_exact_nn_noalloc(idx, f, out)
        torch.cuda.synchronize()
        assert torch.equal(out, ref)
        assert rt.riann_status(idx) == 0
        print("refused-then-ok")
    """) % ROOT
    r = subprocess.run([sys.executable, "-c", script], capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert r.returncode == 0 and "refused-then-ok" in r.stdout, r.stdout + r.stderr


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
