"""Unit-normalised float variant on the GPU vs the oracle, bit-exact (both
sides run the same IEEE fp32 steps in the same order): tables, frame-0 brute
force, chained ring steps on whole small frames, sampled 1080p queries."""
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


def _cmp(g, o, qidx=None, what=""):
    ga, gd, gc = (t.cpu().numpy().reshape(-1) for t in g)
    if qidx is not None:
        ga, gd, gc = ga[qidx], gd[qidx], gc[qidx]
    oa, od, oc = (x.reshape(-1) for x in o)
    for name, x, y in (("annf", ga, oa), ("dist", gd.view(np.uint32), od.view(np.uint32)),
                       ("count", gc.view(np.uint32), oc)):
        bad = np.nonzero(x != y)[0]
        assert bad.size == 0, f"{what} {name}: {bad.size}/{len(x)} differ, first {bad[:4]}: {x[bad[:3]]} vs {y[bad[:3]]}"


def test_tables_are_float_distances(rt):
    import torch
    R, KP, _, _ = synth.random_case(801, 500, 8, 1, 8, 8)
    R[7] = 0                                            # the zero patch
    idx = rt.riann_build_unit_index(_dev(R), _dev(KP))
    P = torch.empty(500 * 8, dtype=torch.int32, device="cuda")
    TA = torch.empty_like(P)
    Tid = torch.empty_like(P)
    rt.riann_index_tables(idx, P, TA, Tid)
    Rn, Kn = oracle.unit_normalize(R), oracle.unit_normalize(KP)
    exp = np.array([[oracle.unit_dist(Kn[m], Rn[r]) for m in range(8)] for r in range(500)], np.float32)
    assert np.array_equal(P.cpu().numpy().view(np.uint32).reshape(500, 8), exp.view(np.uint32))
    ta = TA.cpu().numpy().view(np.float32).reshape(8, 500)
    assert (np.diff(ta, axis=1) >= 0).all()
    assert idx.info().unit == 1
    idx.close()


@pytest.mark.parametrize("n,C,H,W", [(4096, 1, 40, 56), (777, 3, 21, 45), (1, 1, 8, 8), (300, 1, 8, 300)])
def test_frame0_brute_force(rt, n, C, H, W):
    R, KP, frame, _ = synth.random_case(810 + n, n, 3, C, H, W)
    if n > 10:
        R[n // 2:] = R[: n - n // 2]
        frame[:8, :8] = R[n // 2 + 1]
    idx = rt.riann_build_unit_index(_dev(R), _dev(KP))
    g = rt.annf(idx, _dev(frame), None)
    _cmp(g, oracle.riann_unit_frame(R, KP, frame, None))
    idx.close()


@pytest.mark.parametrize("n,K,C,H,W", [(300, 64, 1, 37, 29), (257, 17, 3, 15, 100), (2049, 5, 1, 8, 300),
                                       (3000, 32, 3, 70, 9), (6001, 64, 1, 24, 90), (5, 3, 1, 9, 40)])
@pytest.mark.parametrize("alpha,limit", [((1, 4), -1), ((1, 2), 40), ((1, 1), -1), ((1, 8), 0)])
def test_random_cases(rt, n, K, C, H, W, alpha, limit):
    R, KP, frame, prev = synth.random_case(820 + n + K, n, K, C, H, W)
    idx = rt.riann_build_unit_index(_dev(R), _dev(KP))
    g = rt.annf(idx, _dev(frame), _dev(prev), _params(rt, n, alpha, limit))
    assert rt.riann_status(idx) == 0
    _cmp(g, oracle.riann_unit_frame(R, KP, frame, prev, alpha, limit))
    idx.close()


def test_tiny_chain(rt):
    w = synth.WORKLOADS["tiny"]
    R = synth.workload_reference(w)
    KP = synth.workload_keypoints(w, R)
    frames = synth.Video(w.video).frames(0, 5)
    idx = rt.riann_build_unit_index(_dev(R), _dev(KP))
    p = _params(rt, len(R))
    pg, po = None, None
    for t, f in enumerate(frames):
        g = rt.annf(idx, _dev(f), pg, p)
        o = oracle.riann_unit_frame(R, KP, f, po, (1, 4), p.ring_limit)
        _cmp(g, o, what=f"frame {t}")
        pg, po = g[0], o[0]
    assert rt.riann_status(idx) == 0
    idx.close()


def test_1080p_sampled(rt):
    w = synth.WORKLOADS["1080p"]
    R = synth.workload_reference(w)
    KP = synth.workload_keypoints(w, R)
    video = synth.Video(w.video)
    frames = [video.frame(t) for t in (20, 21, 22)]
    Q = (1080 - 7) * (1920 - 7)
    rng = np.random.default_rng(83)
    qidx = np.unique(np.concatenate([rng.choice(Q, 120, replace=False), [0, Q - 1]])).astype(np.int64)
    idx = rt.riann_build_unit_index(_dev(R), _dev(KP))
    p = _params(rt, len(R))
    pg, po = None, None
    for t, f in enumerate(frames):
        g = rt.annf(idx, _dev(f), pg, p)
        o = oracle.riann_unit_frame(R, KP, f, po, (1, 4), p.ring_limit, qidx=qidx)
        _cmp(g, o, qidx, what=f"frame {20 + t}")
        pg = g[0]
        pv = np.zeros(Q, np.int32)
        pv[qidx] = o[0]
        po = pv.reshape(1073, 1913)
    assert rt.riann_status(idx) == 0
    idx.close()


def test_unsupported_forms(rt):
    import torch
    R, KP, frame, prev = synth.random_case(830, 64, 4, 1, 12, 12)
    idx = rt.riann_build_unit_index(_dev(R), _dev(KP))
    out = torch.empty((5, 5), dtype=torch.int32, device="cuda")
    kn = torch.empty((5, 5, 2), dtype=torch.int32, device="cuda")
    with pytest.raises(rt.RiannError) as e:
        rt.riann_knn_frame(idx, _params(rt, 64), _dev(frame), _dev(prev), 2, out, kn)
    assert e.value.code == rt.RIANN_ERR_UNSUPPORTED
    with pytest.raises(rt.RiannError) as e:
        rt.riann_batch_create(idx, 2, 100)
    assert e.value.code == rt.RIANN_ERR_UNSUPPORTED
    idx.close()


def test_bad_prev_sets_status(rt):
    R, KP, frame, prev = synth.random_case(831, 64, 4, 1, 12, 12)
    prev[1, 1] = 1000
    idx = rt.riann_build_unit_index(_dev(R), _dev(KP))
    a, d, c = rt.annf(idx, _dev(frame), _dev(prev), _params(rt, 64, (1, 4), -1))
    assert rt.riann_status(idx) & rt.RIANN_DEV_BAD_PREV
    a = a.cpu().numpy()
    assert a[1, 1] == -1
    ok = prev.copy()
    ok[1, 1] = 0
    oa, od, oc = oracle.riann_unit_frame(R, KP, frame, ok, (1, 4), -1)
    mask = np.ones(prev.shape, bool)
    mask[1, 1] = False
    assert np.array_equal(a[mask], oa[mask])
    idx.close()


@pytest.mark.parametrize("alpha,limit", [((0, 1), -1), ((1, 4), -1), ((1, 1), 30)])
def test_zero_patches_and_alpha_zero(rt, alpha, limit):
    # all-zero query patches and references (a zero patch stays zero), and
    # alpha = 0, where a ring holds only the references at exactly B
    R, KP, frame, prev = synth.random_case(832, 500, 12, 1, 30, 40)
    R[:3] = 0
    R[100:140] = R[:40]                         # duplicates: ties by index
    frame[4:20, 6:22] = 0                       # a block of zero queries
    prev[5:9, 7:11] = 1                         # their previous match: a zero reference
    idx = rt.riann_build_unit_index(_dev(R), _dev(KP))
    g = rt.annf(idx, _dev(frame), _dev(prev), _params(rt, 500, alpha, limit))
    assert rt.riann_status(idx) == 0
    _cmp(g, oracle.riann_unit_frame(R, KP, frame, prev, alpha, limit), what=f"alpha {alpha}")
    g0 = rt.annf(idx, _dev(frame), None)
    _cmp(g0, oracle.riann_unit_frame(R, KP, frame, None), what="frame 0")
    idx.close()
