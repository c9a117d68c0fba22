"""The input generators are seeded and deterministic: the same seed gives the
same bytes (the oracle and the GPU path read identical inputs), different
seeds give different ones, and the workloads have the stated shapes."""
import numpy as np

import synth


def test_video_frames_are_deterministic_and_independent_of_order():
    spec = synth.VideoSpec(48, 64, 1, 123, speeds=(0.5, 2.0), noise_sigma=2.0, cut_every=5)
    a = synth.Video(spec)
    b = synth.Video(spec)
    f7 = a.frame(7)
    assert np.array_equal(f7, b.frame(7))                  # same seed, same bytes
    assert np.array_equal(a.frame(3), b.frame(3))          # any frame without its predecessors
    assert not np.array_equal(a.frame(6), a.frame(7))      # frames move
    c = synth.Video(synth.VideoSpec(48, 64, 1, 124, speeds=(0.5, 2.0), noise_sigma=2.0, cut_every=5))
    assert not np.array_equal(f7, c.frame(7))
    assert f7.shape == (48, 64, 1) and f7.dtype == np.uint8


def test_reference_sets_and_keypoints_are_deterministic():
    r1 = synth.reference_set(9, 500, 3, 64, 80, 3)
    r2 = synth.reference_set(9, 500, 3, 64, 80, 3)
    assert r1.shape == (500, 8, 8, 3) and np.array_equal(r1, r2)
    i1, k1 = synth.keypoints_kmeanspp(r1, 16, 11)
    i2, k2 = synth.keypoints_kmeanspp(r2, 16, 11)
    assert np.array_equal(i1, i2) and np.array_equal(k1, k2)
    assert len(set(i1.tolist())) == 16                       # distinct members of the set
    assert np.array_equal(k1, r1[i1])
    v1 = synth.reference_volumes(5, 100, 2, 40, 48)
    assert np.array_equal(v1, synth.reference_volumes(5, 100, 2, 40, 48))


def test_workload_shapes():
    for name, (H, W) in (("tiny", (128, 128)), ("720p_rgb", (720, 1280)), ("1080p", (1080, 1920))):
        w = synth.WORKLOADS[name]
        assert (w.video.H, w.video.W) == (H, W)
    assert synth.WORKLOADS["1080p"].n == 65536 and synth.WORKLOADS["1080p"].K == 64
    assert synth.WORKLOADS["1080p_st"].C == 3 and synth.WORKLOADS["1080p_st"].volumes
    assert len(synth.BATCH_SIZES) == 32
