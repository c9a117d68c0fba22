"""Pins of the oracle's Sec. 4 reconstruction (patch replacement with averaging
of overlaps, rounded half up to 8 bits, error sums)."""
import os

import numpy as np
import pytest

import oracle
import synth

HERE = os.path.dirname(os.path.abspath(__file__))


def frame_patches(f):
    """All query patches of frame f in query order, (dy, dx, c) vector order."""
    H, W, C = f.shape
    return np.stack([f[y:y + 8, x:x + 8].reshape(-1) for y in range(H - 7) for x in range(W - 7)])


@pytest.mark.parametrize("H,W,C", [(8, 8, 1), (9, 30, 1), (23, 17, 3), (40, 41, 1)])
def test_identity_field_reproduces_frame(H, W, C):
    # every query patch is its own reference: the average of identical bytes is the byte
    f = np.random.default_rng(H * W + C).integers(0, 256, (H, W, C), dtype=np.uint8)
    R = frame_patches(f)
    annf = np.arange(R.shape[0], dtype=np.int32).reshape(H - 7, W - 7)
    out, (e, g) = oracle.reconstruct(R, annf, f)
    assert np.array_equal(out, f)
    assert e == 0 and g == int((f.astype(np.int64) ** 2).sum())


def scatter_reference(R, annf, C):
    """Independent formulation: every patch adds its 8 x 8 block to sum and
    count images; round half up from exact integers."""
    Hq, Wq = annf.shape
    H, W = Hq + 7, Wq + 7
    s = np.zeros((H, W, C), np.int64)
    n = np.zeros((H, W, 1), np.int64)
    Rp = R.reshape(R.shape[0], 8, 8, C).astype(np.int64)
    for py in range(Hq):
        for px in range(Wq):
            r = annf[py, px]
            if 0 <= r < R.shape[0]:
                s[py:py + 8, px:px + 8] += Rp[r]
                n[py:py + 8, px:px + 8] += 1
    return np.where(n > 0, (2 * s + n) // (2 * np.maximum(n, 1)), 0).astype(np.uint8)


@pytest.mark.parametrize("H,W,C,n", [(8, 8, 1, 3), (13, 29, 1, 50), (21, 12, 3, 7), (33, 34, 1, 400)])
def test_matches_scatter_formulation(H, W, C, n):
    rng = np.random.default_rng(7 * H + W)
    R = rng.integers(0, 256, (n, 64 * C), dtype=np.uint8)
    annf = rng.integers(-2, n + 2, (H - 7, W - 7)).astype(np.int32)   # includes entries outside [0, n)
    f = rng.integers(0, 256, (H, W, C), dtype=np.uint8)
    out, (e, g) = oracle.reconstruct(R, annf, f)
    want = scatter_reference(R, annf, C)
    assert np.array_equal(out, want)
    d = f.astype(np.int64) - want.astype(np.int64)
    assert e == int((d * d).sum()) and g == int((f.astype(np.int64) ** 2).sum())


def test_constant_references_closed_form():
    f = synth.Video(synth.VideoSpec(30, 50, 1, 5)).frame(0)
    R = np.full((4, 64), 77, np.uint8)
    annf = np.random.default_rng(3).integers(0, 4, (23, 43)).astype(np.int32)
    out, (e, g) = oracle.reconstruct(R, annf, f)
    assert (out == 77).all()
    ff = f.astype(np.int64)
    assert e == int(((ff - 77) ** 2).sum()) and g == int((ff ** 2).sum())


def test_invalid_field_contributes_nothing():
    R = np.full((2, 64), 9, np.uint8)
    out, _ = oracle.reconstruct(R, np.full((2, 3), 5, np.int32))
    assert (out == 0).all()
    # n itself and -1 are outside [0, n) too (the row after the table holds
    # 200s, so reading it would show)
    table = np.full((3, 64), 9, np.uint8)
    table[2] = 200
    out, _ = oracle.reconstruct(table[:2], np.array([[2, -1, 2]], np.int32))
    assert (out == 0).all()


def load_golden(name):
    d = {}
    for line in open(os.path.join(HERE, "golden", name)):
        line = line.strip()
        if line and not line.startswith("#"):
            k, v = line.split(":", 1)
            d[k.strip()] = [int(t) for t in v.split()]
    return d


def test_golden_two_patches_round_half_up():
    d = load_golden("recon_two_patches.txt")
    H, W = d["H"][0], d["W"][0]
    R = np.stack([np.full(64, v, np.uint8) for v in d["ref_values"]])
    annf = np.array(d["field"], np.int32).reshape(H - 7, W - 7)
    f = np.full((H, W), d["frame_value"][0], np.uint8)
    out, err2 = oracle.reconstruct(R, annf, f)
    assert (out[:, :, 0] == np.array(d["expect_row"], np.uint8)[None]).all()
    assert list(err2) == d["expect_err2"]
