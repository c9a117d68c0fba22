"""Served form: every stream's field in the continuous-batching mix equals the
field of the same stream run alone; admission follows the memory budget."""
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


@pytest.fixture(scope="module")
def indexes(rt):
    out = {}
    for C, seed in ((1, 60), (3, 61)):
        R = synth.reference_set(seed, 3000, 8, 96, 96, C)
        KP = synth.keypoints_kmeanspp(R, 12, 11)[1]
        out[C] = (rt.riann_build_reference_index(_dev(R), _dev(KP)), R, KP)
    yield out
    for v in out.values():
        v[0].close()


def alone(rt, idx, frames, params):
    outs, prev = [], None
    for f in frames:
        a, _, _ = rt.annf(idx, _dev(f), prev, params)
        outs.append(a.cpu().numpy())
        prev = a
    return outs


@pytest.mark.parametrize("plain", [False, True])
def test_mix_equals_alone(rt, indexes, plain):
    import torch
    params = rt.riann_default_params(3000)
    fmts = [(40, 64, 1), (72, 100, 1), (33, 47, 3), (64, 64, 3), (96, 128, 1)]
    vids = [synth.Video(synth.VideoSpec(H, W, C, 70 + i, speeds=(0.5, 2.0))) for i, (H, W, C) in enumerate(fmts)]
    T = 5
    frames = [[v.frame(t) for t in range(T)] for v in vids]
    refs = [alone(rt, indexes[C][0], frames[i], params) for i, (H, W, C) in enumerate(fmts)]
    srv = rt.RiannServer(indexes[1][0], indexes[3][0], budget_bytes=1 << 30, max_tick_queries=1 << 20,
                         max_streams=8, params=params, plain=plain)
    sids = [srv.open(H, W, C) for H, W, C in fmts]
    assert all(s is not None for s in sids)
    for t in range(T):
        # streams join late and skip ticks: stream 4 starts at t = 2, stream 1 idles at t = 3
        for i, sid in enumerate(sids):
            if (i == 4 and t < 2) or (i == 1 and t == 3):
                continue
            srv.submit(sid, frames[i][t], t, rt.riann_server_clock())
        assert srv.step(wait=True) > 0
        srv.step(wait=True)                     # completes the tick
        done = {sid: fid for sid, fid, _, _ in srv.poll()}
        for i, (H, W, C) in enumerate(fmts):
            if (i == 4 and t < 2) or (i == 1 and t == 3):
                assert sids[i] not in done
                continue
            assert done[sids[i]] == t
            got = torch.empty((H - 7, W - 7), dtype=torch.int32)
            srv.field(sids[i], got)
            if i == 4:
                want = alone(rt, indexes[C][0], frames[i][2:t + 1], params)[-1]
            elif i == 1 and t > 3:
                want = alone(rt, indexes[C][0], frames[i][:3] + frames[i][4:t + 1], params)[-1]
            else:
                want = refs[i][t]
            assert np.array_equal(got.numpy(), want), (plain, t, i)
    info = srv.info()
    assert info["dropped"] == 0 and info["open_streams"] == len(fmts)
    srv.close()


def test_admission_budget_and_replacement(rt, indexes):
    params = rt.riann_default_params(3000)
    idx = indexes[1][0]
    one = rt.riann_session_state_bytes(idx, 64, 64)
    srv = rt.RiannServer(idx, None, budget_bytes=2 * one + one // 2, max_tick_queries=1 << 20, max_streams=8,
                         params=params)
    a, b = srv.open(64, 64, 1), srv.open(64, 64, 1)
    assert a is not None and b is not None
    assert srv.open(64, 64, 1) is None                      # third does not fit the budget
    with pytest.raises(rt.RiannError):
        srv.open(64, 64, 3)                                 # no RGB index
    srv.close_stream(a)
    c = srv.open(64, 64, 1)                                 # freed budget admits it
    assert c is not None
    f = synth.Video(synth.VideoSpec(64, 64, 1, 90)).frame(0)
    srv.submit(b, f, 0, 0.0)
    srv.submit(b, f, 1, 0.0)                                # replaces frame 0 before dispatch
    assert srv.step(wait=True) == 1
    srv.step(wait=True)
    res = srv.poll()
    assert [(r[0], r[1]) for r in res] == [(b, 1)]
    info = srv.info()
    assert info["dropped"] == 1 and info["rejected"] == 1
    srv.close()


def test_rate_admission(rt, indexes):
    """With a load limit, a stream that declares a frame rate claims
    fps * queries * (measured GPU time per query); claims must fit the limit."""
    params = rt.riann_default_params(3000)
    idx = indexes[1][0]
    srv = rt.RiannServer(idx, None, budget_bytes=1 << 30, max_tick_queries=1 << 20, max_streams=8,
                         params=params, load_limit=0.5)
    a = srv.open(64, 64, 1, fps=30.0)
    assert a is not None                                    # no measurement yet: the first one enters
    assert srv.open(64, 64, 1, fps=30.0) is None            # ... and only the first
    free = srv.open(64, 64, 1)                              # declares no rate: memory budget only
    assert free is not None
    v = synth.Video(synth.VideoSpec(64, 64, 1, 91))
    for t in range(3):
        srv.submit(a, v.frame(t), t, 0.0)
        srv.step(wait=True)
        srv.step(wait=True)
    info = srv.info()
    ns = info["ns_per_query"][0]
    assert ns > 0 and info["ns_per_query"][1] == 0
    q = 57 * 57
    assert abs(info["load"] - 30.0 * q * ns * 1e-9) <= 1e-9 + 1e-6 * info["load"]
    # a stream whose claim alone exceeds the limit is rejected, a small one fits
    huge_fps = 2.0 * 0.5 / (q * ns * 1e-9)
    assert srv.open(64, 64, 1, fps=huge_fps) is None
    assert srv.open(64, 64, 1, fps=1.0) is not None
    assert srv.info()["rejected"] == 2
    srv.close()
