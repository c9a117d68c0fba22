"""The checked build (libriann_checked.so, RIANN_LIBRARY=checked): every index
a kernel gathers from a table is tested before the access and a failure sets
RIANN_DEV_BOUNDS instead of reading.  On valid input it must give exactly the
oracle's results with a clean status word; a bad previous field still sets
RIANN_DEV_BAD_PREV; cell offsets pushed past a key's rows set RIANN_DEV_BOUNDS.

Each case runs in a child process that loads the checked library.
"""
import os
import subprocess
import sys
import textwrap

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PRELUDE = """
import sys
sys.path.insert(0, %r)
import numpy as np, torch
import oracle, synth
from paper_1508_07953_gb300 import riann as rt
assert rt.library_name() == "libriann_checked.so"
def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()
""" % ROOT


def run_checked(body: str):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    env = dict(os.environ, RIANN_LIBRARY="checked")
    r = subprocess.run([sys.executable, "-c", PRELUDE + textwrap.dedent(body)], capture_output=True, text=True,
                       timeout=600, cwd=ROOT, env=env)
    assert r.returncode == 0 and "checked-ok" in r.stdout, r.stdout + r.stderr


def test_checked_build_tiny_chain_equals_oracle():
    run_checked("""
        w = synth.WORKLOADS["tiny"]
        R = synth.workload_reference(w); KP = synth.workload_keypoints(w, R)
        frames = synth.Video(w.video).frames(0, w.frames)
        oix = oracle.Index(R, KP)
        for scan in (rt.RIANN_SCAN_SINGLE, rt.RIANN_SCAN_PAIRS):
            idx = rt.riann_build_reference_index(dev(R), dev(KP), scan_order=scan)
            params = rt.riann_default_params(len(R))
            prev, oprev = None, None
            for f in frames:
                a, d, c = rt.annf(idx, dev(f), prev, params)
                oa, od, oc, _ = oracle.riann_frame(oix, f, oprev, ring_limit=params.ring_limit)
                assert np.array_equal(a.cpu().numpy(), oa)
                assert np.array_equal(d.cpu().numpy().view(np.uint32), od)
                assert np.array_equal(c.cpu().numpy().view(np.uint32), oc)
                prev, oprev = a, oa
            assert rt.riann_status(idx) == 0
            idx.close()
        print("checked-ok")
    """)


def test_checked_build_random_cases_equal_oracle():
    run_checked("""
        for (n, K, C, H, W) in [(5, 3, 1, 9, 40), (300, 64, 1, 37, 29), (257, 17, 3, 15, 100), (6001, 64, 1, 24, 90)]:
            R, KP, frame, prev = synth.random_case(900 + n, n, K, C, H, W)
            oix = oracle.Index(R, KP)
            for scan in (rt.RIANN_SCAN_SINGLE, rt.RIANN_SCAN_PAIRS):
                for alpha, limit in (((1, 4), -1), ((1, 2), 40)):
                    idx = rt.riann_build_reference_index(dev(R), dev(KP), scan_order=scan)
                    p = rt.riann_default_params(n)
                    p.alpha_num, p.alpha_den, p.ring_limit = alpha[0], alpha[1], limit
                    a, d, c = rt.annf(idx, dev(frame), dev(prev), p)
                    oa, od, oc, _ = oracle.riann_frame(oix, frame, prev, alpha=alpha, ring_limit=limit)
                    assert np.array_equal(a.cpu().numpy(), oa), (n, K, scan, alpha)
                    assert np.array_equal(c.cpu().numpy().view(np.uint32), oc)
                    assert rt.riann_status(idx) == 0
                    idx.close()
        print("checked-ok")
    """)


def test_checked_build_flags_bad_previous_field():
    run_checked("""
        R, KP, frame, prev = synth.random_case(910, 64, 4, 1, 12, 12)
        prev[0, 0] = 64
        prev[2, 3] = -5
        idx = rt.riann_build_reference_index(dev(R), dev(KP))
        a, d, c = rt.annf(idx, dev(frame), dev(prev), rt.riann_default_params(64))
        bits = rt.riann_status(idx)
        assert bits & rt.RIANN_DEV_BAD_PREV and not bits & rt.RIANN_DEV_BOUNDS, bits
        a = a.cpu().numpy()
        assert a[0, 0] == -1 and a[2, 3] == -1
        assert rt.riann_status(idx) == 0
        idx.close()
        print("checked-ok")
    """)


def test_checked_build_flags_offsets_past_the_rows():
    run_checked("""
        w = synth.WORKLOADS["tiny"]
        R = synth.workload_reference(w); KP = synth.workload_keypoints(w, R)
        frames = synth.Video(w.video).frames(0, 2)
        idx = rt.riann_build_reference_index(dev(R), dev(KP), scan_order=rt.RIANN_SCAN_PAIRS)
        params = rt.riann_default_params(len(R))
        a0, _, _ = rt.annf(idx, dev(frames[0]), None, params)
        rt.annf(idx, dev(frames[1]), a0, params)
        assert rt.riann_status(idx) == 0
        for key in range(len(KP) - 1):
            rt.riann_test_corrupt_offsets(idx, key, 8)
        rt.annf(idx, dev(frames[1]), a0, params)
        bits = rt.riann_status(idx)
        assert bits & rt.RIANN_DEV_BOUNDS, bits
        idx.close()
        print("checked-ok")
    """)
