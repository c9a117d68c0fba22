"""Pins of the 3-D spatio-temporal query (Sec. 1: 8x8xT volumes instead of 8x8 patches).

The stacked frame's (dy, dx, c) patches must be the volumes of the three
frames in (dy, dx, tau) order: reference volumes cut from the frames by plain
slicing are found by exact NN at distance 0 and at their own positions, and a
volume with its frames in the other order is not.
"""
import numpy as np

import oracle
import synth
from conftest import read_fixture


def _frames(seed=3, H=20, W=27):
    rng = np.random.default_rng(seed)
    return [rng.integers(0, 256, size=(H, W), dtype=np.uint8) for _ in range(3)]


def test_stacked_patches_are_the_volumes():
    f = _frames()
    st = oracle.stack_frames(*f)
    H, W = f[0].shape
    pos = [(0, 0), (H - 8, W - 8), (5, 11), (12, 3)]
    R = np.stack([np.stack([f[t][y:y + 8, x:x + 8] for t in range(3)], -1) for y, x in pos])   # [n][8][8][3]
    qidx = np.array([y * (W - 7) + x for y, x in pos], np.int64)
    annf, dist, _ = oracle.exact_nn(st, R, qidx=qidx)
    assert list(annf) == list(range(len(pos))) and (dist == 0).all()


def test_time_order_matters():
    f = _frames(4)
    st = oracle.stack_frames(*f)
    W = f[0].shape[1]
    y, x = 6, 9
    rev = np.stack([f[t][y:y + 8, x:x + 8] for t in (2, 1, 0)], -1)[None]
    _, dist, _ = oracle.exact_nn(st, rev, qidx=np.array([y * (W - 7) + x], np.int64))
    assert dist[0] > 0


def test_reference_volumes_are_spatiotemporal_cuts():
    # every reference volume's time slices are 8x8 cuts of three consecutive frames
    R = synth.reference_volumes(21, 40, 2, 48, 64)
    assert R.shape == (40, 8, 8, 3) and R.dtype == np.uint8
    assert len({R[i].tobytes() for i in range(40)}) > 30
    # consecutive frames of a slowly moving video: the slices are close, unlike unrelated patches
    d_t = np.abs(R[..., 0].astype(int) - R[..., 1].astype(int)).mean()
    d_x = np.abs(R[:20, ..., 0].astype(int) - R[20:, ..., 0].astype(int)).mean()
    assert d_t < d_x


def golden_case():
    """(frames, R, KP, prev, alpha, ring_limit, fixture) of
    tests/golden/spatiotemporal_constant_frames.txt."""
    fx = read_fixture("spatiotemporal_constant_frames.txt")

    def vols(s):
        return np.stack([np.broadcast_to(np.array([int(v) for v in t.split(",")], np.uint8), (8, 8, 3))
                         for t in s.split()])

    frames = [np.full((8, 8), int(v), np.uint8) for v in fx["frame_values"].split()]
    prev = np.array([[int(fx["prev"])]], np.int32)
    alpha = tuple(int(x) for x in fx["alpha"].split())
    return frames, vols(fx["ref_volumes"]), vols(fx["key_volumes"]), prev, alpha, int(fx["ring_limit"]), fx


def test_golden_constant_frames():
    frames, R, KP, prev, alpha, limit, fx = golden_case()
    st = oracle.stack_frames(*frames)
    idx = oracle.Index(R, KP)
    for key, pv in (("expect_ring", prev), ("expect_first_frame", None)):
        a, d, c, _ = oracle.riann_frame(idx, st, pv, alpha=alpha, ring_limit=limit, mode="definitional")
        assert [int(a.ravel()[0]), int(d.ravel()[0]), int(c.ravel()[0])] == [int(x) for x in fx[key].split()]
