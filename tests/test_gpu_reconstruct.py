"""Sec. 4 reconstruction on the GPU (riann_reconstruct) against the oracle:
the rebuilt frame and the error sums are bit-identical."""
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


def _gpu(rt, idx, annf, frame):
    import torch
    H, W = annf.shape[0] + 7, annf.shape[1] + 7
    out = torch.empty((H, W, idx.C), dtype=torch.uint8, device="cuda")
    err2 = torch.zeros(2, dtype=torch.int64, device="cuda")
    rt.riann_reconstruct(idx, _dev(annf), _dev(frame), out, err2)
    return out.cpu().numpy(), tuple(int(v) for v in err2.cpu())


@pytest.mark.parametrize("n,C,H,W", [(5, 1, 8, 8), (300, 1, 9, 33), (777, 3, 21, 45), (4096, 1, 100, 140),
                                     (64, 3, 40, 8), (1000, 1, 71, 300)])
def test_random_fields_match_oracle(rt, n, C, H, W):
    R, KP, frame, _ = synth.random_case(500 + n + H, n, 2, C, H, W)
    annf = np.random.default_rng(n * W).integers(0, n, (H - 7, W - 7)).astype(np.int32)
    idx = rt.riann_build_reference_index(_dev(R), _dev(KP))
    out, err2 = _gpu(rt, idx, annf, frame)
    want, werr2 = oracle.reconstruct(R, annf, frame)
    assert np.array_equal(out, want)
    assert err2 == werr2
    assert rt.riann_status(idx) == 0
    idx.close()


def test_identity_field_reproduces_frame(rt):
    f = synth.Video(synth.VideoSpec(36, 52, 3, 17)).frame(0)
    R = np.stack([f[y:y + 8, x:x + 8] for y in range(29) for x in range(45)])   # [n][8][8][3]
    KP = R[:3]
    idx = rt.riann_build_reference_index(_dev(R), _dev(KP))
    annf = np.arange(R.shape[0], dtype=np.int32).reshape(29, 45)
    out, (e, g) = _gpu(rt, idx, annf, f)
    assert np.array_equal(out, f) and e == 0 and g == int((f.astype(np.int64) ** 2).sum())
    idx.close()


def test_entries_outside_the_index_are_skipped_and_flagged(rt):
    import torch
    R, KP, frame, _ = synth.random_case(601, 50, 2, 1, 20, 30)
    annf = np.random.default_rng(2).integers(0, 50, (13, 23)).astype(np.int32)
    annf[3, 4], annf[0, 0], annf[12, 22] = -1, 50, 1 << 30
    idx = rt.riann_build_reference_index(_dev(R), _dev(KP))
    out, err2 = _gpu(rt, idx, annf, frame)
    want, werr2 = oracle.reconstruct(R, annf, frame)
    assert np.array_equal(out, want) and err2 == werr2
    assert rt.riann_status(idx) & rt.RIANN_DEV_BAD_PREV
    # output only, no error sums; and error sums only, no output
    o2 = torch.empty_like(torch.from_numpy(want)).cuda()
    rt.riann_reconstruct(idx, _dev(annf), out=o2)
    e2 = torch.zeros(2, dtype=torch.int64, device="cuda")
    rt.riann_reconstruct(idx, _dev(annf), _dev(frame), None, e2)
    assert np.array_equal(o2.cpu().numpy(), want) and tuple(int(v) for v in e2.cpu()) == werr2
    rt.riann_status(idx)
    idx.close()


def test_1080p_ring_field_full_frame(rt):
    """Reconstruction of a full 1080p frame from the ring step's field (the
    bench's quality number) equals the oracle's."""
    w = synth.WORKLOADS["1080p"]
    R = synth.workload_reference(w)
    KP = synth.workload_keypoints(w, R)
    v = synth.Video(w.video)
    f0, f1 = v.frame(20), v.frame(21)
    idx = rt.riann_build_reference_index(_dev(R), _dev(KP))
    p = rt.riann_default_params(w.n)
    a0, _, _ = rt.annf(idx, _dev(f0), None, p)
    a1, _, _ = rt.annf(idx, _dev(f1), a0, p)
    field = a1.cpu().numpy()
    out, err2 = _gpu(rt, idx, field, f1)
    want, werr2 = oracle.reconstruct(R, field, f1)
    assert np.array_equal(out, want) and err2 == werr2
    assert 0.0 < (err2[0] / err2[1]) ** 0.5 < 0.5
    idx.close()
