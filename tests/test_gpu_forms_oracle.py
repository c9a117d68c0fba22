"""The batched and served forms against the CPU oracle itself, and one whole
1080p ring step compared at every query.

Each stream of a batched tick or a served mix must carry exactly the field the
oracle computes for that stream alone (Alg. 1 per query: the previous match at
the same position, the rings, the argmin over S u {r_p}).  A query's step reads
the previous field only at its own position, so an oracle chain restricted to
sampled positions follows the GPU's stream exactly; it restarts with brute
force wherever the stream restarts (a reset, a late join) and skips the frames
the stream skipped.
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


def _sample(H, W, nsamp, seed):
    """nsamp seeded query positions plus the four corners of the field."""
    Hq, Wq = H - 7, W - 7
    Q = Hq * Wq
    rng = np.random.default_rng(seed)
    pick = rng.choice(Q, min(nsamp, Q), replace=False)
    return np.unique(np.concatenate([pick, [0, Wq - 1, Q - Wq, Q - 1]])).astype(np.int64)


class OracleStream:
    """The oracle's chain of one stream at sampled positions."""

    def __init__(self, oix, H, W, params, qidx):
        self.oix, self.H, self.W, self.params, self.qidx = oix, H, W, params, qidx
        self.prev = None

    def reset(self):
        self.prev = None

    def step(self, frame):
        prev = None
        if self.prev is not None:
            prev = np.zeros((self.H - 7) * (self.W - 7), np.int32)
            prev[self.qidx] = self.prev
            prev = prev.reshape(self.H - 7, self.W - 7)
        a, d, c, _ = oracle.riann_frame(self.oix, frame, prev, alpha=(self.params.alpha_num, self.params.alpha_den),
                                        ring_limit=self.params.ring_limit, qidx=self.qidx)
        self.prev = a
        return a, d, c


def _check_sampled(got, want, qidx, what):
    for k, name in enumerate(("annf", "dist", "count")[:len(got)]):
        a = got[k].ravel()[qidx]
        b = want[k].ravel()
        if k:
            a, b = a.view(np.uint32), b.view(np.uint32)
        bad = np.nonzero(a != b)[0]
        assert bad.size == 0, (f"{what} {name}: {bad.size}/{a.size} sampled queries differ; first at "
                               f"{qidx[bad[:5]]}: gpu {a[bad[:5]]} oracle {b[bad[:5]]}")


def test_batched_tick_shaped_like_32_streams_matches_oracle(rt):
    # the 32-stream batched workload's index (n = 16384, K = 32) and six of its
    # streams: one 1080p and one 720p among 480p and 240p ones, three ticks
    # through one captured graph, one stream restarting at the third
    w = synth.BATCH_INDEX
    R = synth.workload_reference(w)
    KP = synth.workload_keypoints(w, R)
    idx = rt.riann_build_reference_index(_dev(R), _dev(KP))
    params = rt.riann_default_params(len(R))
    oix = oracle.Index(R, KP)
    which = [24, 16, 8, 9, 0, 1]
    vids = [synth.Video(synth.batch_stream_spec(s)) for s in which]
    sizes = [synth.BATCH_SIZES[s] for s in which]
    sess = [rt.riann_session_create(idx, H, W) for H, W in sizes]
    ors = [OracleStream(oix, H, W, params, _sample(H, W, 400, 300 + i)) for i, (H, W) in enumerate(sizes)]
    b = rt.riann_batch_create(idx, 8, sum((H - 7) * (W - 7) for H, W in sizes))
    reset = {2: 2}                                  # stream 2 restarts at tick 2
    routed = 0
    for t in range(3):
        frames = [v.frame(t) for v in vids]
        for i, tt in reset.items():
            if t == tt:
                rt.riann_session_reset(sess[i])
                ors[i].reset()
        rt.riann_batch_run(b, params, sess, [_dev(f) for f in frames])
        for i in range(len(which)):
            got = [x.cpu().numpy() for x in rt.session_result(sess[i])]
            want = ors[i].step(frames[i])
            _check_sampled(got, want, ors[i].qidx, f"batched tick {t} stream {which[i]} {sizes[i]}")
            if t > 0:
                routed += int((want[2] == len(R)).sum())
    assert b.info().graph_builds == 1
    assert rt.riann_status(idx) == 0
    assert routed > 0                               # brute-force routing is exercised inside the batch
    b.close()
    for s in sess:
        s.close()
    idx.close()


def test_served_mix_with_1080p_matches_oracle(rt):
    import torch
    # the served workload's two indexes (n = 65536, K = 64, gray and RGB; one
    # parameter set for both); a 1080p gray stream from the start, a 720p
    # stream that joins late, a 480p stream that skips a tick, a 480p RGB stream
    w = synth.WORKLOADS["1080p"]
    Rg = synth.workload_reference(w)
    KPg = synth.workload_keypoints(w, Rg)
    Rc = synth.workload_reference(synth.SERVE_RGB_INDEX)
    KPc = synth.workload_keypoints(synth.SERVE_RGB_INDEX, Rc)
    gidx = rt.riann_build_reference_index(_dev(Rg), _dev(KPg))
    cidx = rt.riann_build_reference_index(_dev(Rc), _dev(KPc))
    ogix, ocix = oracle.Index(Rg, KPg), oracle.Index(Rc, KPc)
    pg = rt.riann_default_params(len(Rg))
    fmts = [(1080, 1920, 1), (720, 1280, 1), (480, 640, 1), (480, 640, 3)]
    joins = [0, 1, 0, 0]
    skips = {2: {2}}                                # stream 2 sends nothing at tick 2
    vids = [synth.Video(synth.VideoSpec(H, W, C, 400 + i, speeds=(0.0, 0.5, 2.0, 6.0), noise_sigma=2.0))
            for i, (H, W, C) in enumerate(fmts)]
    srv = rt.RiannServer(gidx, cidx, budget_bytes=1 << 32, max_tick_queries=1 << 23, max_streams=8, params=pg)
    sids = [srv.open(H, W, C) for H, W, C in fmts]
    assert all(s is not None for s in sids)
    ors = [OracleStream(ogix if C == 1 else ocix, H, W, pg, _sample(H, W, 400, 500 + i))
           for i, (H, W, C) in enumerate(fmts)]
    T = 4
    for t in range(T):
        sent = []
        for i, sid in enumerate(sids):
            if t < joins[i] or t in skips.get(i, ()):
                continue
            f = vids[i].frame(t)
            srv.submit(sid, f, t, rt.riann_server_clock())
            sent.append((i, f))
        assert srv.step(wait=True) > 0
        srv.step(wait=True)                         # completes the tick
        done = {sid: fid for sid, fid, _, _ in srv.poll()}
        assert sorted(done) == sorted(sids[i] for i, _ in sent)
        for i, f in sent:
            H, W, C = fmts[i]
            assert done[sids[i]] == t
            got = torch.empty((H - 7, W - 7), dtype=torch.int32)
            srv.field(sids[i], got)
            want = ors[i].step(f)
            _check_sampled([got.numpy()], want, ors[i].qidx, f"served tick {t} stream {i} {fmts[i]}")
    assert srv.info()["dropped"] == 0
    srv.close()
    assert rt.riann_status(gidx) == 0 and rt.riann_status(cidx) == 0
    gidx.close()
    cidx.close()


def test_whole_1080p_ring_step_matches_oracle(rt):
    # every one of the 2,052,649 queries of a 1080p frame, ring step and brute
    # force for the routed ones, against the oracle's indexed mode on all host
    # cores.  The previous field is the oracle's exact NN of frame 20 over the
    # first 4096 references (a valid field of this index that the oracle
    # computes in seconds; its temporal changes route a few percent of the
    # queries, as a chained field does).
    w = synth.WORKLOADS["1080p"]
    R = synth.workload_reference(w)
    KP = synth.workload_keypoints(w, R)
    video = synth.Video(w.video)
    f20, f21 = video.frame(20), video.frame(21)
    prev = oracle.exact_nn(f20, R[:4096])[0]
    idx = rt.riann_build_reference_index(_dev(R), _dev(KP))
    params = rt.riann_default_params(len(R))
    a, d, c = rt.annf(idx, _dev(f21), _dev(prev), params)
    got = [a.cpu().numpy(), d.cpu().numpy().view(np.uint32), c.cpu().numpy().view(np.uint32)]
    assert rt.riann_status(idx) == 0
    idx.close()
    oix = oracle.Index(R, KP)
    want = oracle.riann_frame(oix, f21, prev, alpha=(1, 4), ring_limit=params.ring_limit)[:3]
    for k, name in enumerate(("annf", "dist", "count")):
        bad = np.flatnonzero(got[k].ravel() != want[k].ravel())
        assert bad.size == 0, f"whole 1080p frame {name}: {bad.size} of {got[k].size} queries differ, first {bad[:5]}"
    routed = float((want[2] == len(R)).mean())
    assert 0.005 < routed < 0.5                      # both paths carry real work
