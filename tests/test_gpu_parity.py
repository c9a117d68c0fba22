"""GPU path vs the CPU oracle, element by element (bit-exact: all integer work).

Small cases compare every query; full-size workloads (720p RGB with n=16384,
1080p with n=65536) run whole frames on the GPU and compare a seeded sample of
query positions, for which the oracle runs its own chain (a query's step reads
the previous field only at its own position, so a sampled chain is exact).
"""
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


def _np(t, unsigned=False):
    a = t.cpu().numpy()
    return a.view(np.uint32) if unsigned else a


def make_params(rt, n, alpha=(1, 4), ring_limit="default", cap=0):
    p = rt.riann_default_params(n)
    p.alpha_num, p.alpha_den = alpha
    if ring_limit != "default":
        p.ring_limit = ring_limit
    p.cap = cap
    return p


def gpu_chain(rt, R, KP, frames, params, scan_order=None):
    idx = rt.riann_build_reference_index(_dev(R), _dev(KP), scan_order=scan_order)
    outs, prev = [], None
    for f in frames:
        a, d, c = rt.annf(idx, _dev(f), prev, params)
        outs.append((_np(a), _np(d, True), _np(c, True)))
        prev = a
    bits = rt.riann_status(idx)
    idx.close()
    assert bits == 0, f"device status bits {bits:#x}"
    return outs


def oracle_chain(R, KP, frames, params, qidx=None):
    oix = oracle.Index(R, KP)
    outs, prev = [], None
    H, W = frames[0].shape[:2]
    for f in frames:
        a, d, c, _ = oracle.riann_frame(oix, f, prev, alpha=(params.alpha_num, params.alpha_den),
                                        ring_limit=params.ring_limit, qidx=qidx)
        outs.append((a, d, c))
        if qidx is None:
            prev = a
        else:
            prev = np.zeros((H - 7) * (W - 7), np.int32)
            prev[qidx] = a
            prev = prev.reshape(H - 7, W - 7)
    return outs


def assert_same(g, o, qidx=None, what=""):
    for k, name in enumerate(("annf", "dist", "count")):
        a = g[k].ravel() if qidx is None else g[k].ravel()[qidx]
        b = o[k].ravel()
        bad = np.nonzero(a != b)[0]
        assert bad.size == 0, (f"{what} {name}: {bad.size}/{a.size} differ; first at {bad[:5]} "
                               f"gpu={a[bad[:5]]} oracle={b[bad[:5]]}")


# ---------------------------------------------------------------------------
# index build (pre-processing tables)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("n,K,C", [(1, 1, 1), (33, 5, 1), (1000, 7, 3), (4096, 16, 1), (5000, 64, 1)])
def test_index_tables_match_oracle(rt, n, K, C):
    import torch
    R, KP, _, _ = synth.random_case(100 + n, n, K, C, 8, 8)
    if n > 10:
        R[n // 2:] = R[: n - n // 2]            # equal distances: ties ordered by index
    idx = rt.riann_build_reference_index(_dev(R), _dev(KP))
    P = torch.empty(n * K, dtype=torch.int32, device="cuda")
    TA = torch.empty_like(P)
    Tid = torch.empty_like(P)
    rt.riann_index_tables(idx, P, TA, Tid)
    oix = oracle.Index(R, KP)
    assert np.array_equal(_np(P, True).reshape(n, K), oix.P)
    assert np.array_equal(_np(TA, True).reshape(K, n), oix.TA)
    assert np.array_equal(_np(Tid).reshape(K, n), oix.Tid)
    idx.close()


# ---------------------------------------------------------------------------
# brute force (frame 0)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("n,C,H,W", [(4096, 1, 128, 128), (777, 3, 21, 45), (1, 1, 8, 8), (300, 1, 8, 300)])
def test_exact_nn_matches_oracle(rt, n, C, H, W):
    R, KP, frame, _ = synth.random_case(200 + n, n, 3, C, H, W)
    if n > 10:
        R[n // 3: 2 * (n // 3)] = R[: n // 3]
        frame[:8, :8] = R[n // 3 + 1]
    idx = rt.riann_build_reference_index(_dev(R), _dev(KP))
    import torch
    a = torch.empty((H - 7, W - 7), dtype=torch.int32, device="cuda")
    d = torch.empty_like(a)
    rt.riann_exact_nn(idx, _dev(frame), a, d)
    oa, od, _ = oracle.exact_nn(frame, R)
    assert np.array_equal(_np(a), oa) and np.array_equal(_np(d, True), od)
    idx.close()


# ---------------------------------------------------------------------------
# the whole step on the tiny workload (4096 refs, 16 key points, 8 frames)
# ---------------------------------------------------------------------------
@pytest.fixture(scope="module")
def tiny():
    w = synth.WORKLOADS["tiny"]
    R = synth.workload_reference(w)
    KP = synth.workload_keypoints(w, R)
    frames = synth.Video(w.video).frames(0, w.frames)
    return R, KP, frames


@pytest.mark.parametrize("scan", ["auto", "pairs"])
@pytest.mark.parametrize("alpha,limit", [((1, 4), "default"), ((1, 4), -1), ((1, 4), 0),
                                         ((1, 1), -1), ((0, 1), -1), ((3, 8), 64)])
def test_tiny_chain_all_queries(rt, tiny, alpha, limit, scan):
    # "pairs": the scan of a second key's buckets, which the index uses for
    # n >= 16384 only, forced on the tiny index
    R, KP, frames = tiny
    params = make_params(rt, len(R), alpha, limit)
    g = gpu_chain(rt, R, KP, frames, params, None if scan == "auto" else rt.RIANN_SCAN_PAIRS)
    o = oracle_chain(R, KP, frames, params)
    for t in range(len(frames)):
        assert_same(g[t], o[t], what=f"frame {t}")


def test_cap_does_not_change_output(rt, tiny):
    R, KP, frames = tiny
    base = gpu_chain(rt, R, KP, frames[:3], make_params(rt, len(R)))
    for cap in (1, 2, 3, 4):
        other = gpu_chain(rt, R, KP, frames[:3], make_params(rt, len(R), cap=cap))
        for t in range(3):
            for k in range(3):
                assert np.array_equal(base[t][k], other[t][k])


# ---------------------------------------------------------------------------
# ragged / degenerate shapes
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("n,K,C,H,W", [
    (1, 1, 1, 8, 8),          # one query, one reference
    (5, 3, 1, 9, 40),         # fewer references than a warp
    (300, 64, 1, 37, 29),     # maximum K, ragged tile edges
    (257, 17, 3, 15, 100),    # RGB, odd K
    (2049, 5, 1, 8, 300),     # one query row
    (3000, 32, 3, 70, 9),     # one query column pair
    (6001, 64, 1, 24, 90),    # n not a multiple of 4 with K = 64: long seed runs, many drains
])
@pytest.mark.parametrize("alpha,limit", [((1, 4), -1), ((1, 2), 40), ((8, 1), -1)])
@pytest.mark.parametrize("scan", [1, 2])
def test_random_cases(rt, n, K, C, H, W, alpha, limit, scan):
    R, KP, frame, prev = synth.random_case(300 + n + K, n, K, C, H, W)
    params = make_params(rt, n, alpha, limit)
    idx = rt.riann_build_reference_index(_dev(R), _dev(KP), scan_order=scan)
    a, d, c = rt.annf(idx, _dev(frame), _dev(prev), params)
    assert rt.riann_status(idx) == 0
    oix = oracle.Index(R, KP)
    oa, od, oc, _ = oracle.riann_frame(oix, frame, prev, alpha=alpha, ring_limit=limit)
    assert_same((_np(a), _np(d, True), _np(c, True)), (oa, od, oc))
    idx.close()


def test_bad_prev_sets_status(rt):
    import torch
    R, KP, frame, prev = synth.random_case(400, 64, 4, 1, 12, 12)
    prev[0, 0] = 64          # out of range
    prev[1, 1] = -3
    idx = rt.riann_build_reference_index(_dev(R), _dev(KP))
    a, d, c = rt.annf(idx, _dev(frame), _dev(prev), make_params(rt, 64))
    bits = rt.riann_status(idx)
    assert bits & rt.RIANN_DEV_BAD_PREV
    a = _np(a)
    assert a[0, 0] == -1 and a[1, 1] == -1
    assert rt.riann_status(idx) == 0      # cleared by the read
    idx.close()


def test_invalid_arguments_rejected(rt):
    import torch
    R, KP, frame, prev = synth.random_case(401, 64, 4, 1, 12, 12)
    idx = rt.riann_build_reference_index(_dev(R), _dev(KP))
    out = torch.empty((5, 5), dtype=torch.int32, device="cuda")
    for bad in (dict(alpha_den=0), dict(alpha_den=9), dict(alpha_num=-1), dict(alpha_num=65, alpha_den=8),
                dict(ring_limit=-2), dict(cap=-1), dict(cap=5)):
        p = make_params(rt, 64)
        for k, v in bad.items():
            setattr(p, k, v)
        with pytest.raises(rt.RiannError) as e:
            rt.riann_annf_frame(idx, p, _dev(frame), _dev(prev), out)
        assert e.value.code == rt.RIANN_ERR_INVALID_ARG
    small = torch.zeros((7, 12, 1), dtype=torch.uint8, device="cuda")
    with pytest.raises(ValueError):
        rt.riann_annf_frame(idx, make_params(rt, 64), small, None, out)
    idx.close()
    with pytest.raises(rt.RiannError):
        rt.riann_build_reference_index(_dev(R), _dev(np.zeros((65, 8, 8, 1), np.uint8)))
    with pytest.raises(rt.RiannError) as e:
        rt.riann_build_reference_index(_dev(R), _dev(KP), scan_order=3)
    assert e.value.code == rt.RIANN_ERR_INVALID_ARG


# ---------------------------------------------------------------------------
# full-size workloads, sampled queries
# ---------------------------------------------------------------------------
def _sampled_chain(rt, w, t0, t1, nsamp, seed, scan_order=None):
    R = synth.workload_reference(w)
    KP = synth.workload_keypoints(w, R)
    video = synth.Video(w.video)
    frames = [video.frame(t) for t in range(t0, t1)]
    params = make_params(rt, len(R))
    g = gpu_chain(rt, R, KP, frames, params, scan_order)
    H, W = frames[0].shape[:2]
    Q = (H - 7) * (W - 7)
    rng = np.random.default_rng(seed)
    qidx = np.unique(np.concatenate([rng.choice(Q, nsamp, replace=False), [0, Q - 1, W - 8]]))
    o = oracle_chain(R, KP, frames, params, qidx)
    for i in range(len(frames)):
        assert_same(g[i], o[i], qidx, what=f"{w.name} frame {t0 + i}")
    return g


def test_720p_rgb_full_frames_sampled(rt):
    _sampled_chain(rt, synth.WORKLOADS["720p_rgb"], 0, 3, 600, 21)


def test_720p_rgb_single_key_scan_sampled(rt):
    # the single-key scan (used for n < 16384) forced on the 16384-patch RGB index
    _sampled_chain(rt, synth.WORKLOADS["720p_rgb"], 0, 3, 600, 23, rt.RIANN_SCAN_SINGLE)


def test_1080p_single_key_scan_sampled(rt):
    # the single-key scan (used for n < 16384) forced on the 65536-patch index
    _sampled_chain(rt, synth.WORKLOADS["1080p"], 20, 23, 400, 24, rt.RIANN_SCAN_SINGLE)


def test_1080p_across_scene_cut_sampled(rt):
    # frames 38..41 of the 1080p video: dense start, steady frame, scene cut at 40
    g = _sampled_chain(rt, synth.WORKLOADS["1080p"], 38, 42, 400, 22)
    n = synth.WORKLOADS["1080p"].n
    # the cut frame sends far more queries to brute force (count = n) than a steady frame
    assert (g[2][2] == n).mean() > 0.25 and (g[2][2] == n).mean() > 3 * (g[1][2] == n).mean()


def test_candidates_grow_with_temporal_change(rt):
    # Fig. 5 (diagnostic, not parity): regions that move faster give larger
    # rings, so more candidates per query and more queries routed to brute force
    w = synth.WORKLOADS["720p_rgb"]
    R = synth.workload_reference(w)
    KP = synth.workload_keypoints(w, R)
    video = synth.Video(w.video)
    frames = [video.frame(t) for t in (1, 2, 3)]
    g = gpu_chain(rt, R, KP, frames, make_params(rt, len(R)))
    count = g[2][2].astype(np.int64)                       # frame 3
    _, vel, _ = video._scene(0)
    reg = w.video.region
    Hq, Wq = count.shape
    speed = np.hypot(vel[..., 0], vel[..., 1])
    sp = speed[np.arange(Hq)[:, None] // reg, np.arange(Wq)[None, :] // reg]
    ring = count < len(R)
    means, routed = [], []
    for s in sorted(set(np.round(w.video.speeds, 3))):
        m = np.isclose(sp, s)
        if m.sum() < 1000:
            continue
        means.append(count[m & ring].mean())
        routed.append(1.0 - ring[m].mean())
    assert len(means) >= 3
    assert means[-1] > 2 * means[0] and routed[-1] > routed[0]
    assert all(b >= a * 0.9 for a, b in zip(means, means[1:]))   # rising, up to noise
