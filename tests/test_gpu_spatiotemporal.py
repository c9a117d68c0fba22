"""3-D spatio-temporal patches on the GPU vs the oracle (bit-exact).

The interleaving kernel against the oracle's stacking (aligned and unaligned
buffers, ragged pixel counts), then the query step on stacked frames against
the oracle's 3-channel step: whole frames of a 128x128 video against 4096
reference volumes, and sampled queries of 1080p against 65536.
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


@pytest.mark.parametrize("H,W", [(1, 1), (8, 8), (9, 13), (37, 29), (1080, 1920)])
@pytest.mark.parametrize("offset", [0, 1])
def test_stack_matches_oracle(rt, H, W, offset):
    import torch
    rng = np.random.default_rng(H * 7 + W + offset)
    f = [rng.integers(0, 256, size=(H, W), dtype=np.uint8) for _ in range(3)]
    # offset 1: frames and output start one byte into their buffers (byte path)
    bufs = [torch.zeros(H * W + 8, dtype=torch.uint8, device="cuda") for _ in range(3)]
    views = []
    for b, x in zip(bufs, f):
        v = b[offset:offset + H * W]
        v.copy_(torch.from_numpy(x.reshape(-1)))
        views.append(v.view(H, W))
    ob = torch.full((3 * H * W + 8,), 7, dtype=torch.uint8, device="cuda")
    out = ob[offset:offset + 3 * H * W]
    rt.riann_stack_frames(*views, out=out)
    got = out.cpu().numpy().reshape(H, W, 3)
    assert np.array_equal(got, oracle.stack_frames(*f))
    rest = ob.cpu().numpy()
    assert (rest[:offset] == 7).all() and (rest[offset + 3 * H * W:] == 7).all()   # nothing written outside


def test_invalid_arguments(rt):
    import torch
    f = torch.zeros((8, 8), dtype=torch.uint8, device="cuda")
    o = torch.zeros((8, 8, 3), dtype=torch.uint8, device="cuda")
    with pytest.raises(rt.RiannError) as e:          # output aliasing an input
        rt.riann_stack_frames(o.view(-1)[:64].view(8, 8), f, f, out=o)
    assert e.value.code == rt.RIANN_ERR_INVALID_ARG


def _chain(rt, w, t0, t1, qidx=None):
    R = synth.workload_reference(w)
    KP = synth.workload_keypoints(w, R)
    video = synth.Video(w.video)
    gray = [video.frame(t)[..., 0] for t in range(t0 - 2, t1)]
    idx = rt.riann_build_reference_index(_dev(R), _dev(KP))
    oix = oracle.Index(R, KP)
    p = rt.riann_default_params(len(R))
    H, W = gray[0].shape
    Q = (H - 7) * (W - 7)
    prev_g, prev_o = None, None
    for t in range(2, len(gray)):
        st_g = rt.riann_stack_frames(_dev(gray[t - 2]), _dev(gray[t - 1]), _dev(gray[t]))
        st_o = oracle.stack_frames(gray[t - 2], gray[t - 1], gray[t])
        a, d, c = rt.annf(idx, st_g, prev_g, p)
        if prev_o is None:
            oa, od, oc = oracle.exact_nn(st_o, R, qidx=qidx)
        else:
            oa, od, oc, _ = oracle.riann_frame(oix, st_o, prev_o, alpha=(1, 4), ring_limit=p.ring_limit, qidx=qidx)
        g = [x.cpu().numpy().reshape(-1) for x in (a, d, c)]
        if qidx is not None:
            g = [x[qidx] for x in g]
        for name, x, y in zip(("annf", "dist", "count"), g, (oa, od, oc)):
            bad = np.nonzero(x.view(np.uint32) != y.reshape(-1).view(np.uint32))[0]
            assert bad.size == 0, f"{w.name} frame {t0 + t - 2} {name}: {bad.size} differ, first {bad[:4]}"
        prev_g = a
        if qidx is None:
            prev_o = oa
        else:
            pv = np.zeros(Q, np.int32)
            pv[qidx] = oa
            prev_o = pv.reshape(H - 7, W - 7)
    assert rt.riann_status(idx) == 0
    idx.close()


def test_tiny_volumes_all_queries(rt):
    _chain(rt, synth.WORKLOADS["tiny_st"], 2, 7)


def test_1080p_volumes_sampled(rt):
    w = synth.WORKLOADS["1080p_st"]
    Q = (1080 - 7) * (1920 - 7)
    rng = np.random.default_rng(41)
    qidx = np.unique(np.concatenate([rng.choice(Q, 150, replace=False), [0, Q - 1]])).astype(np.int64)
    _chain(rt, w, 21, 24, qidx)
