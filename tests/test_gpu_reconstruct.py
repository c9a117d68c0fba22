"""Sec. 4 reconstruction on the GPU (riann_reconstruct) and the Sec. 5
effects by patch replacement (riann_reconstruct_payload) against the oracle:
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


def _gpu_payload(rt, idx, payload, annf, frame):
    import torch
    H, W = annf.shape[0] + 7, annf.shape[1] + 7
    C = payload.shape[3]
    out = torch.empty((H, W, C), dtype=torch.uint8, device="cuda")
    err2 = torch.zeros(2, dtype=torch.int64, device="cuda")
    rt.riann_reconstruct_payload(idx, _dev(payload), _dev(annf), _dev(frame), out, err2)
    return out.cpu().numpy(), tuple(int(v) for v in err2.cpu())


@pytest.mark.parametrize("n,C,Cp,H,W", [(300, 1, 3, 21, 45), (777, 3, 1, 30, 40), (1000, 1, 1, 71, 300),
                                        (64, 3, 3, 9, 8)])
def test_payload_matches_oracle(rt, n, C, Cp, H, W):
    """Sec. 5: the rows come from a transformed table T(R) with its own channel count."""
    R, KP, _, _ = synth.random_case(700 + n, n, 2, C, 8, 8)
    rng = np.random.default_rng(n + Cp)
    payload = rng.integers(0, 256, size=(n, 8, 8, Cp), dtype=np.uint8)
    target = rng.integers(0, 256, size=(H, W, Cp), dtype=np.uint8)
    annf = rng.integers(0, n, (H - 7, W - 7)).astype(np.int32)
    annf[0, 0] = n                                  # outside the index: skipped and flagged
    idx = rt.riann_build_reference_index(_dev(R), _dev(KP))
    out, err2 = _gpu_payload(rt, idx, payload, annf, target)
    want, werr2 = oracle.reconstruct(payload, annf, target)
    assert np.array_equal(out, want) and err2 == werr2
    assert rt.riann_status(idx) & rt.RIANN_DEV_BAD_PREV
    # the index's own references as the payload: riann_reconstruct exactly
    if Cp == C:
        annf[0, 0] = 0
        o1, e1 = _gpu_payload(rt, idx, R, annf, target)
        o2, e2 = _gpu(rt, idx, annf, target)
        assert np.array_equal(o1, o2) and e1 == e2
    idx.close()


def test_payload_colours_a_gray_video(rt):
    """Colourisation as Sec. 5 sets it up: a gray index of reference cuts whose
    colour versions are the payload; the field of a gray frame then rebuilds a
    colour frame."""
    import torch
    video = synth.Video(synth.VideoSpec(48, 64, 3, 23))
    ref_rgb = video.frame(0)
    to_gray = lambda f: ((f[..., 0].astype(np.uint32) * 77 + f[..., 1].astype(np.uint32) * 150
                          + f[..., 2].astype(np.uint32) * 29) >> 8).astype(np.uint8)
    pos = [(y, x) for y in range(0, 41, 2) for x in range(0, 57, 2)]
    payload = np.stack([ref_rgb[y:y + 8, x:x + 8] for y, x in pos])                 # [n][8][8][3]
    R = to_gray(payload)[..., None]                                                  # [n][8][8][1]
    idx = rt.riann_build_reference_index(_dev(R), _dev(R[:4]))
    f_rgb = video.frame(2)
    field = torch.empty((41, 57), dtype=torch.int32, device="cuda")
    rt.riann_exact_nn(idx, _dev(to_gray(f_rgb)), field)
    annf = field.cpu().numpy()
    out, err2 = _gpu_payload(rt, idx, payload, annf, f_rgb)
    want, werr2 = oracle.reconstruct(payload, annf, f_rgb)
    assert np.array_equal(out, want) and err2 == werr2
    assert rt.riann_status(idx) == 0
    idx.close()


def test_payload_arguments_rejected(rt):
    import torch
    R, KP, frame, _ = synth.random_case(711, 40, 2, 1, 12, 12)
    idx = rt.riann_build_reference_index(_dev(R), _dev(KP))
    annf = _dev(np.zeros((5, 5), np.int32))
    raw = torch.zeros(40 * 64 + 16, dtype=torch.uint8, device="cuda")
    shifted = raw[1:1 + 40 * 64].view(40, 8, 8, 1)                   # not 16-byte aligned
    with pytest.raises(rt.RiannError) as e:
        rt.riann_reconstruct_payload(idx, shifted, annf, out=torch.empty((12, 12, 1), dtype=torch.uint8,
                                                                         device="cuda"))
    assert e.value.code == rt.RIANN_ERR_INVALID_ARG
    with pytest.raises(ValueError):                                   # n rows of the index
        rt.riann_reconstruct_payload(idx, raw[:39 * 64].view(39, 8, 8, 1), annf)
    with pytest.raises(ValueError):                                   # C' in {1, 3}
        rt.riann_reconstruct_payload(idx, torch.zeros((40, 8, 8, 2), dtype=torch.uint8, device="cuda"), annf)
    assert rt.riann_status(idx) == 0
    idx.close()
