"""The hand-worked fixtures of tests/golden/ through the CUDA path.

The same small cases that pin the oracle by hand (constant or 16-pixel
patches and constant volumes, whose ring sets, lists, trees and averages
are derived in each file's header) run here through the C-ABI: ring steps
(Sec. 3.2, Alg. 1), k-NN lists (Sec. 7), the unit-length variant (Sec. 3.4),
the regression-tree clustering (Sec. 3.4), 3-D spatio-temporal volumes
(Sec. 1), the random-anchor loop (Alg. 1) and the Sec. 4 reconstruction.
Expected values come from the fixture files alone.
"""
import numpy as np
import pytest

import test_oracle_cluster as cluster_pins
import test_oracle_knn as knn_pins
import test_oracle_pins as pins
import test_oracle_spatiotemporal as st_pins
import test_oracle_unit as unit_pins
from conftest import read_fixture

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


def _params(rt, n, alpha, limit):
    p = rt.riann_default_params(n)
    p.alpha_num, p.alpha_den = alpha
    p.ring_limit = limit
    return p


def _gray(values):
    return np.stack([np.full((8, 8, 1), int(v), np.uint8) for v in values])


@pytest.mark.parametrize("name", pins.GOLDEN)
def test_ring_fixture(rt, name):
    fx, R, KP, frame, prev, alpha, limit = pins.fixture_case(name)
    idx = rt.riann_build_reference_index(_dev(R), _dev(KP))
    a, d, c = rt.annf(idx, _dev(frame), _dev(prev), _params(rt, len(R), alpha, limit))
    assert rt.riann_status(idx) == 0
    assert a.item() == int(fx["expect_annf"])
    assert d.cpu().numpy().view(np.uint32).item() == int(fx["expect_dist"])
    assert c.cpu().numpy().view(np.uint32).item() == int(fx["expect_count"])
    idx.close()


@pytest.mark.parametrize("name", knn_pins.GOLDEN)
def test_knn_fixture(rt, name):
    fx = read_fixture(name)
    R, KP = _gray(fx["ref_values"].split()), _gray(fx["key_values"].split())
    frame = np.full((8, 8), int(fx["query_value"]), np.uint8)
    prev = np.array([[int(fx["prev"])]], np.int32)
    alpha = tuple(int(x) for x in fx["alpha"].split())
    k = int(fx["k"])
    idx = rt.riann_build_reference_index(_dev(R), _dev(KP))
    a, kn, kd, c = rt.knn(idx, _dev(frame), _dev(prev), k, _params(rt, len(R), alpha, int(fx["ring_limit"])))
    assert rt.riann_status(idx) == 0
    assert kn.cpu().numpy().ravel().tolist() == [int(x) for x in fx["expect_knn"].split()]
    assert kd.cpu().numpy().view(np.uint32).ravel().tolist() == [int(x) for x in fx["expect_knn_dist"].split()]
    assert c.cpu().numpy().view(np.uint32).ravel().tolist() == [int(fx["expect_count"])]
    assert a.item() == int(fx["expect_knn"].split()[0])
    idx.close()


@pytest.mark.parametrize("case", ["limit_-1", "limit_5", "limit_6", "zero_query_limit_-1"])
def test_unit_fixture(rt, case):
    fx = read_fixture("unit_16_pixel_sets.txt")
    R = np.stack([unit_pins._set_patch(s) for s in fx["refs"].split(";")])
    KP = np.stack([unit_pins._set_patch(s) for s in fx["keys"].split(";")])
    frame = np.zeros((8, 8, 1), np.uint8) if case.startswith("zero") else unit_pins._set_patch(fx["query"])
    prev = np.array([[int(fx["prev"])]], np.int32)
    alpha = tuple(int(x) for x in fx["alpha"].split())
    idx = rt.riann_build_unit_index(_dev(R), _dev(KP))
    a, d, c = rt.annf(idx, _dev(frame[:, :, 0]), _dev(prev), _params(rt, len(R), alpha, int(case.rsplit("_", 1)[1])))
    assert rt.riann_status(idx) == 0
    e_annf, e_d2, e_count = fx["expect_" + case].split()
    num, _, den = e_d2.partition("/")
    assert a.item() == int(e_annf)
    assert d.cpu().numpy().view(np.uint32).item() == unit_pins._f32_sqrt(int(num), int(den or 1)).view(np.uint32)
    assert c.cpu().numpy().view(np.uint32).item() == int(e_count)
    idx.close()


@pytest.mark.parametrize("name", cluster_pins.GOLDEN)
def test_cluster_fixture(rt, name):
    fx = read_fixture(name)
    X = cluster_pins._golden_patches(fx, "values" if "values" in fx else "patches")
    reps, assign = rt.riann_cluster_references(_dev(X.reshape(-1, 8, 8, 1)), int(fx["leaf"]))
    want = cluster_pins._golden_patches(fx, "expect_reps")
    assert tuple(reps.shape) == (len(want), 8, 8, 1)
    assert np.array_equal(reps.cpu().numpy().reshape(len(want), 64), want)
    assert assign.cpu().numpy().tolist() == [int(x) for x in fx["expect_assign"].split()]


def _ints(name):
    return {k: [int(t) for t in v.split()] for k, v in read_fixture(name).items()}


@pytest.mark.parametrize("seed", [0, 1, 2, 3, 12345])
def test_anchor_fixture(rt, seed):
    d = _ints("anchor_loop_at_L.txt")
    R = _gray(d["ref_values"])
    H, W = d["H"][0], d["W"][0]
    frame = np.full((H, W), d["query_value"][0], np.uint8)
    prev = np.full((H - 7, W - 7), d["prev"][0], np.int32)
    idx = rt.riann_build_reference_index(_dev(R), _dev(R[:1]))
    full = rt.riann_full_create(idx)
    p = rt.riann_default_anchor_params()
    p.alpha_num, p.alpha_den = d["alpha"]
    p.L, p.seed = d["L"][0], seed
    a, dist, c, k = rt.anchor(full, _dev(frame), _dev(prev), p)
    assert rt.riann_status(idx) == 0
    got = (a.item(), dist.cpu().numpy().view(np.uint32).item(), c.cpu().numpy().view(np.uint32).item(),
           k.cpu().numpy().view(np.uint32).item())
    assert got == (d["expect_annf"][0], d["expect_dist"][0], d["expect_count"][0], d["expect_rings"][0])
    full.close()
    idx.close()


def test_reconstruct_fixture(rt):
    import torch
    d = _ints("recon_two_patches.txt")
    H, W = d["H"][0], d["W"][0]
    R = _gray(d["ref_values"])
    idx = rt.riann_build_reference_index(_dev(R), _dev(R[:1]))
    annf = np.array(d["field"], np.int32).reshape(H - 7, W - 7)
    frame = np.full((H, W), d["frame_value"][0], np.uint8)
    out = torch.empty((H, W, 1), dtype=torch.uint8, device="cuda")
    err2 = torch.zeros(2, dtype=torch.int64, device="cuda")
    rt.riann_reconstruct(idx, _dev(annf), _dev(frame), out, err2)
    assert (out.cpu().numpy()[:, :, 0] == np.array(d["expect_row"], np.uint8)[None]).all()
    assert err2.cpu().numpy().tolist() == d["expect_err2"]
    idx.close()


def test_spatiotemporal_fixture(rt):
    frames, R, KP, prev, alpha, limit, fx = st_pins.golden_case()
    st = rt.riann_stack_frames(*(_dev(f) for f in frames))
    idx = rt.riann_build_reference_index(_dev(R), _dev(KP))
    for key, pv in (("expect_ring", _dev(prev)), ("expect_first_frame", None)):
        a, d, c = rt.annf(idx, st, pv, _params(rt, len(R), alpha, limit))
        got = [a.item(), d.cpu().numpy().view(np.uint32).item(), c.cpu().numpy().view(np.uint32).item()]
        assert got == [int(x) for x in fx[key].split()], key
    assert rt.riann_status(idx) == 0
    idx.close()
