"""Alg. 1 with random anchors on the GPU (riann_full_*, riann_anchor_frame)
against the oracle: the sorted distance matrix and every output
(field, distance, |S|, rings drawn) are bit-identical."""
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


def params(rt, alpha=(1, 4), L=20, max_rings=64, seed=0, frame_id=0):
    p = rt.riann_default_anchor_params()
    p.alpha_num, p.alpha_den, p.L, p.max_rings, p.seed, p.frame_id = alpha[0], alpha[1], L, max_rings, seed, frame_id
    return p


@pytest.mark.parametrize("n,C", [(300, 1), (1000, 1), (2049, 1), (500, 3)])
def test_sorted_matrix_matches_oracle(rt, n, C):
    R = np.random.default_rng(n + C).integers(0, 256, (n, 8, 8, C), dtype=np.uint8)
    R[: n // 10] = R[n // 10: 2 * (n // 10)]          # duplicates: equal distances, ties by index
    idx = rt.riann_build_reference_index(_dev(R), _dev(R[:2]))
    full = rt.riann_full_create(idx)
    assert np.array_equal(rt.riann_full_table(full), oracle.FullIndex(R).T)
    full.close()
    idx.close()


def _check(rt, R, frame, prev, alpha, L, max_rings, seed, frame_id):
    idx = rt.riann_build_reference_index(_dev(R), _dev(R[:2]))
    full = rt.riann_full_create(idx)
    got = rt.anchor(full, _dev(frame), None if prev is None else _dev(prev),
                    params(rt, alpha, L, max_rings, seed, frame_id))
    assert rt.riann_status(idx) == 0
    want = oracle.riann_anchor_frame(oracle.FullIndex(R), frame, prev, alpha=alpha, L=L, max_rings=max_rings,
                                     seed=seed, frame_id=frame_id)
    for g, w in zip(got, want):
        assert np.array_equal(g.cpu().numpy().astype(np.int64), w.astype(np.int64))
    full.close()
    idx.close()


@pytest.mark.parametrize("n,C,H,W", [(400, 1, 20, 40), (1500, 1, 33, 21), (300, 3, 14, 30)])
@pytest.mark.parametrize("alpha,L,max_rings", [((1, 4), 20, 64), ((1, 4), 2, 64), ((1, 2), 5, 3), ((3, 1), 8, 64),
                                               ((1, 8), 1, 64)])
def test_random_frames_match_oracle(rt, n, C, H, W, alpha, L, max_rings):
    R, _, frame, prev = synth.random_case(700 + n + L, n, 1, C, H, W)
    R = (R // 16 * 16).astype(np.uint8)                 # coarse values: rings of many members, ties
    frame = (frame // 16 * 16).astype(np.uint8)
    _check(rt, R, frame, prev, alpha, L, max_rings, seed=0xC0FFEE1234 + n, frame_id=3)


def test_video_chain_matches_oracle_and_alpha_one_is_exact(rt):
    w = synth.WORKLOADS["tiny"]
    R = synth.workload_reference(w)[:2000]
    frames = synth.Video(w.video).frames(0, 4)[:, :48, :80]
    idx = rt.riann_build_reference_index(_dev(R), _dev(R[:2]))
    full = rt.riann_full_create(idx)
    fi = oracle.FullIndex(R)
    for alpha in ((1, 4), (1, 1)):
        prev_g = prev_o = None
        for t in range(4):
            p = params(rt, alpha, 20, 64, seed=77, frame_id=t)
            a, d, c, k = rt.anchor(full, _dev(frames[t]), prev_g, p)
            oa, od, oc, ok = oracle.riann_anchor_frame(fi, frames[t], prev_o, alpha=alpha, L=20, max_rings=64,
                                                       seed=77, frame_id=t)
            for g, o in ((a, oa), (d, od), (c, oc), (k, ok)):
                assert np.array_equal(g.cpu().numpy().astype(np.int64), o.astype(np.int64)), (alpha, t)
            if alpha == (1, 1):
                ea, ed, _ = oracle.exact_nn(frames[t], R)
                assert np.array_equal(oa, ea)
            prev_g, prev_o = a, oa
    assert rt.riann_status(idx) == 0
    full.close()
    idx.close()


def test_bad_prev_sets_status(rt):
    R, _, frame, prev = synth.random_case(901, 200, 1, 1, 12, 12)
    prev[0, 0], prev[2, 3] = 200, -5
    idx = rt.riann_build_reference_index(_dev(R), _dev(R[:2]))
    full = rt.riann_full_create(idx)
    a, d, c, k = rt.anchor(full, _dev(frame), _dev(prev), params(rt))
    assert rt.riann_status(idx) & rt.RIANN_DEV_BAD_PREV
    a = a.cpu().numpy()
    assert a[0, 0] == -1 and a[2, 3] == -1
    full.close()
    idx.close()


def test_random_field_matches_oracle(rt):
    import torch
    for H, W, n, seed, fid in ((8, 8, 1, 0, 0), (37, 100, 65536, 0x5EED, 3), (720, 1280, 16384, 1 << 63, 11)):
        out = torch.empty((H - 7, W - 7), dtype=torch.int32, device="cuda")
        rt.riann_random_field(H, W, n, seed, fid, out)
        assert np.array_equal(out.cpu().numpy(), oracle.random_field(H, W, n, seed, fid))
