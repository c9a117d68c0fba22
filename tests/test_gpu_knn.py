"""k-NN output (Sec. 7) on the GPU vs the CPU oracle, bit-exact.

Covers the ring kernel's k-NN variant (warp-wide best-k list over S u {r_p})
and the tensor-core brute force's best-8 lists (frame 0, routed queries,
reference-tile splits when few queries are routed), on whole small frames and
on sampled queries of full-size frames.
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


def _params(rt, n, alpha=(1, 4), limit="default"):
    p = rt.riann_default_params(n)
    p.alpha_num, p.alpha_den = alpha
    if limit != "default":
        p.ring_limit = limit
    return p


def _check(g, o, k, qidx=None, what=""):
    ga, gk, gd, gc = (t.cpu().numpy() for t in g)
    gk = gk.reshape(-1, k)
    gd = gd.reshape(-1, k).view(np.uint32)
    gc = gc.reshape(-1).view(np.uint32)
    ga = ga.reshape(-1)
    if qidx is not None:
        gk, gd, gc, ga = gk[qidx], gd[qidx], gc[qidx], ga[qidx]
    ok, od, oc = o
    ok, od, oc = ok.reshape(-1, k), od.reshape(-1, k), oc.reshape(-1)
    for name, a, b in (("knn", gk, ok), ("knn_dist", gd, od), ("count", gc, oc)):
        bad = np.nonzero((a != b).reshape(len(a), -1).any(1))[0]
        assert bad.size == 0, (f"{what} {name}: {bad.size}/{len(a)} queries differ; first {bad[:4]}: "
                               f"gpu={a[bad[:2]]} oracle={b[bad[:2]]}")
    assert np.array_equal(ga, gk[:, 0]), f"{what}: annf is not the first k-NN entry"


@pytest.mark.parametrize("k", [1, 4, 8])
def test_tiny_chain(rt, k):
    w = synth.WORKLOADS["tiny"]
    R = synth.workload_reference(w)
    KP = synth.workload_keypoints(w, R)
    frames = synth.Video(w.video).frames(0, 3)
    idx = rt.riann_build_reference_index(_dev(R), _dev(KP))
    oix = oracle.Index(R, KP)
    p = _params(rt, len(R))
    prev_g, prev_o = None, None
    for t, f in enumerate(frames):
        g = rt.knn(idx, _dev(f), prev_g, k, p)
        o = oracle.riann_knn(oix, f, prev_o, k, alpha=(1, 4), ring_limit=p.ring_limit)
        _check(g, o, k, what=f"frame {t}")
        prev_g, prev_o = g[0], o[0][..., 0]
    assert rt.riann_status(idx) == 0
    idx.close()


@pytest.mark.parametrize("n,K,C,H,W,k", [
    (1, 1, 1, 8, 8, 8),          # fewer references than k
    (5, 3, 1, 9, 40, 8),
    (300, 64, 1, 37, 29, 3),     # maximum K, ragged tiles
    (257, 17, 3, 15, 100, 5),    # RGB
    (3000, 32, 3, 70, 9, 8),
    (6001, 64, 1, 24, 90, 2),
])
@pytest.mark.parametrize("alpha,limit", [((1, 4), -1), ((1, 2), 40), ((8, 1), -1), ((1, 4), 0)])
def test_random_cases(rt, n, K, C, H, W, k, alpha, limit):
    R, KP, frame, prev = synth.random_case(500 + n + K, n, K, C, H, W)
    if n > 10:
        R[n // 2:] = R[: n - n // 2]             # equal distances: ties by index
    idx = rt.riann_build_reference_index(_dev(R), _dev(KP))
    g = rt.knn(idx, _dev(frame), _dev(prev), k, _params(rt, n, alpha, limit))
    assert rt.riann_status(idx) == 0
    o = oracle.riann_knn(oracle.Index(R, KP), frame, prev, k, alpha=alpha, ring_limit=limit)
    _check(g, o, k)
    idx.close()


def test_frame0_brute_force_with_tile_split(rt):
    # few queries: the brute force splits every query tile's references over work items
    R, KP, frame, _ = synth.random_case(601, 5000, 8, 1, 20, 30)
    R[2500:] = R[:2500]
    idx = rt.riann_build_reference_index(_dev(R), _dev(KP))
    g = rt.knn(idx, _dev(frame), None, 8)
    o = oracle.riann_knn(oracle.Index(R, KP), frame, None, 8)
    _check(g, o, 8)
    idx.close()


def test_matches_the_argmin_path(rt):
    R, KP, frame, prev = synth.random_case(602, 4000, 16, 1, 64, 96)
    idx = rt.riann_build_reference_index(_dev(R), _dev(KP))
    p = _params(rt, 4000, (1, 4), 200)
    a, d, c = rt.annf(idx, _dev(frame), _dev(prev), p)
    ga, gk, gd, gc = rt.knn(idx, _dev(frame), _dev(prev), 6, p)
    assert np.array_equal(a.cpu().numpy(), ga.cpu().numpy())
    assert np.array_equal(d.cpu().numpy(), gd[..., 0].cpu().numpy())
    assert np.array_equal(c.cpu().numpy(), gc.cpu().numpy())
    idx.close()


def test_invalid_k_rejected(rt):
    import torch
    R, KP, frame, prev = synth.random_case(603, 64, 4, 1, 12, 12)
    idx = rt.riann_build_reference_index(_dev(R), _dev(KP))
    out = torch.empty((5, 5), dtype=torch.int32, device="cuda")
    for k in (0, 9, -1):
        kn = torch.empty((5, 5, max(k, 1)), dtype=torch.int32, device="cuda")
        with pytest.raises(rt.RiannError) as e:
            rt.riann_knn_frame(idx, _params(rt, 64), _dev(frame), _dev(prev), k, out, kn)
        assert e.value.code == rt.RIANN_ERR_INVALID_ARG
    idx.close()


def _sampled(rt, w, t0, t1, k, nsamp, seed):
    R = synth.workload_reference(w)
    KP = synth.workload_keypoints(w, R)
    video = synth.Video(w.video)
    frames = [video.frame(t) for t in range(t0, t1)]
    H, W = frames[0].shape[:2]
    Q = (H - 7) * (W - 7)
    rng = np.random.default_rng(seed)
    qidx = np.unique(np.concatenate([rng.choice(Q, nsamp, replace=False), [0, Q - 1, W - 8]]))
    idx = rt.riann_build_reference_index(_dev(R), _dev(KP))
    oix = oracle.Index(R, KP)
    p = _params(rt, len(R))
    prev_g, prev_o = None, None
    for t, f in enumerate(frames):
        g = rt.knn(idx, _dev(f), prev_g, k, p)
        o = oracle.riann_knn(oix, f, prev_o, k, alpha=(1, 4), ring_limit=p.ring_limit, qidx=qidx)
        _check(g, o, k, qidx, what=f"{w.name} frame {t0 + t}")
        # the oracle's next step reads the previous field only at the sampled queries
        prev_g = g[0]
        prev_o = np.zeros(Q, np.int32)
        prev_o[qidx] = o[0][:, 0]
        prev_o = prev_o.reshape(H - 7, W - 7)
    assert rt.riann_status(idx) == 0
    idx.close()


def test_720p_rgb_sampled(rt):
    _sampled(rt, synth.WORKLOADS["720p_rgb"], 0, 3, 4, 200, 31)


def test_1080p_scene_cut_sampled(rt):
    _sampled(rt, synth.WORKLOADS["1080p"], 39, 42, 8, 150, 32)


def test_bad_prev_sets_status_and_empty_lists(rt):
    R, KP, frame, prev = synth.random_case(604, 64, 4, 1, 12, 12)
    prev[0, 0] = 64
    prev[2, 3] = -1
    idx = rt.riann_build_reference_index(_dev(R), _dev(KP))
    a, kn, kd, c = rt.knn(idx, _dev(frame), _dev(prev), 3, _params(rt, 64))
    assert rt.riann_status(idx) & rt.RIANN_DEV_BAD_PREV
    kn = kn.cpu().numpy()
    kd = kd.cpu().numpy().view(np.uint32)
    for (y, x) in ((0, 0), (2, 3)):
        assert (kn[y, x] == -1).all() and (kd[y, x] == 0xFFFFFFFF).all() and a.cpu().numpy()[y, x] == -1
    # every other query matches the oracle on a valid copy of the field
    ok = prev.copy()
    ok[0, 0] = 0
    ok[2, 3] = 0
    o = oracle.riann_knn(oracle.Index(R, KP), frame, ok, 3, alpha=(1, 4), ring_limit=8)
    mask = np.ones(prev.shape, bool)
    mask[0, 0] = mask[2, 3] = False
    assert np.array_equal(kn[mask], o[0][mask])
    idx.close()
