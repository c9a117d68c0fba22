"""Pins of the oracle's k-NN output (Sec. 7: more than one match per query).

Each check derives the expected lists independently of ``oracle_riann_knn``:
numpy brute force with an explicit (distance, index) sort, the pinned argmin
of the 1-NN step, the alpha = 1 guarantee (every reference at least as close
as the previous match lies in every ring), and a Python assembly of
S u {r_p} from the separately pinned ring predicate.
"""
import numpy as np
import pytest

import oracle
import synth
from conftest import read_fixture


def np_sorted_lists(frame, R):
    """Per query, every reference as (d, index) sorted by distance then index (int64)."""
    f = frame if frame.ndim == 3 else frame[:, :, None]
    C = f.shape[2]
    Q = np.lib.stride_tricks.sliding_window_view(f, (8, 8, C)).reshape(-1, 64 * C).astype(np.int64)
    Rm = R.reshape(R.shape[0], -1).astype(np.int64)
    d = ((Q[:, None, :] - Rm[None, :, :]) ** 2).sum(-1)           # [Q][n]
    idx = np.broadcast_to(np.arange(R.shape[0]), d.shape)
    order = np.lexsort((idx, d), axis=-1)
    return np.take_along_axis(d, order, -1), order


def cut(d_sorted, i_sorted, k):
    n = d_sorted.shape[-1]
    kk = min(k, n)
    ids = np.full(d_sorted.shape[:-1] + (k,), -1, np.int64)
    ds = np.full(d_sorted.shape[:-1] + (k,), 0xFFFFFFFF, np.int64)
    ids[..., :kk] = i_sorted[..., :kk]
    ds[..., :kk] = d_sorted[..., :kk]
    return ids, ds


GOLDEN = ["knn_1d_two_keys.txt", "knn_1d_limit_bruteforce.txt", "knn_1d_limit_equal.txt",
          "knn_1d_prev_kept.txt"]


@pytest.mark.parametrize("name", GOLDEN)
def test_golden_fixture(name):
    """Hand-worked lists on constant gray patches (tests/golden/knn_*.txt)."""
    fx = read_fixture(name)
    assert int(fx["channels"]) == 1

    def patches(s):
        return np.stack([np.full((8, 8, 1), int(v), np.uint8) for v in s.split()])

    R, KP = patches(fx["ref_values"]), patches(fx["key_values"])
    frame = np.full((8, 8), int(fx["query_value"]), np.uint8)
    prev = np.array([[int(fx["prev"])]], np.int32)
    k = int(fx["k"])
    alpha = tuple(int(x) for x in fx["alpha"].split())
    knn, kd, count = oracle.riann_knn(oracle.Index(R, KP), frame, prev, k, alpha=alpha,
                                      ring_limit=int(fx["ring_limit"]))
    assert knn.ravel().tolist() == [int(x) for x in fx["expect_knn"].split()]
    assert kd.ravel().tolist() == [int(x) for x in fx["expect_knn_dist"].split()]
    assert count.ravel().tolist() == [int(fx["expect_count"])]


@pytest.mark.parametrize("n,C,H,W,k", [(300, 1, 12, 20, 8), (5, 1, 9, 9, 8), (257, 3, 10, 13, 3), (1, 1, 8, 8, 2)])
def test_frame0_is_sorted_brute_force(n, C, H, W, k):
    R, KP, frame, _ = synth.random_case(900 + n, n, min(4, n), C, H, W)
    if n > 10:
        R[n // 2:] = R[: n - n // 2]                  # equal distances: ties by index
    oix = oracle.Index(R, KP)
    knn, kd, count = oracle.riann_knn(oix, frame, None, k)
    ds, ids = np_sorted_lists(frame, R)
    ei, ed = cut(ds, ids, k)
    assert np.array_equal(knn.reshape(-1, k), ei) and np.array_equal(kd.reshape(-1, k).astype(np.int64), ed)
    assert (count == n).all()


@pytest.mark.parametrize("alpha,limit", [((1, 4), -1), ((1, 2), 40), ((0, 1), -1), ((1, 1), 0), ((3, 8), 10)])
def test_k1_is_the_argmin_step(alpha, limit):
    R, KP, frame, prev = synth.random_case(910, 400, 6, 1, 14, 22)
    R[200:] = R[:200]
    oix = oracle.Index(R, KP)
    knn, kd, count = oracle.riann_knn(oix, frame, prev, 1, alpha=alpha, ring_limit=limit)
    a, d, c, _ = oracle.riann_frame(oix, frame, prev, alpha=alpha, ring_limit=limit, mode="definitional")
    assert np.array_equal(knn[..., 0], a) and np.array_equal(kd[..., 0], d) and np.array_equal(count, c)


def test_routing_at_the_limit_follows_the_argmin_step():
    # ring_limit equal to some queries' smallest ring: those stay on the rings
    R, KP, frame, prev = synth.random_case(915, 300, 5, 1, 12, 16)
    oix = oracle.Index(R, KP)
    _, _, _, nseed = oracle.riann_frame(oix, frame, prev, alpha=(1, 2), ring_limit=-1, mode="definitional")
    for limit in (int(np.median(nseed)), int(nseed.min()), int(nseed.max())):
        knn, kd, count = oracle.riann_knn(oix, frame, prev, 2, alpha=(1, 2), ring_limit=limit)
        a, d, c, _ = oracle.riann_frame(oix, frame, prev, alpha=(1, 2), ring_limit=limit, mode="definitional")
        assert (nseed == limit).any()
        assert np.array_equal(knn[..., 0], a) and np.array_equal(kd[..., 0], d) and np.array_equal(count, c)


def test_routed_queries_are_sorted_brute_force():
    R, KP, frame, prev = synth.random_case(911, 300, 5, 1, 12, 16)
    oix = oracle.Index(R, KP)
    k = 5
    knn, kd, count = oracle.riann_knn(oix, frame, prev, k, alpha=(8, 1), ring_limit=0)   # every ring too wide
    ds, ids = np_sorted_lists(frame, R)
    ei, ed = cut(ds, ids, k)
    assert (count == 300).all()
    assert np.array_equal(knn.reshape(-1, k), ei) and np.array_equal(kd.reshape(-1, k).astype(np.int64), ed)


def test_alpha_one_prefix_is_exact_knn():
    # alpha = 1: every r with ||q - r|| <= ||q - r_p|| is in every ring (triangle
    # inequality), so the listed entries up to distance C are the exact k-NN ones
    R, KP, frame, prev = synth.random_case(912, 500, 8, 1, 13, 19)
    R[250:] = R[:250]
    oix = oracle.Index(R, KP)
    k = 8
    knn, kd, _ = oracle.riann_knn(oix, frame, prev, k, alpha=(1, 1), ring_limit=-1)
    ds, ids = np_sorted_lists(frame, R)
    Qm = ds.shape[0]
    prevf = prev.reshape(-1)
    checked = 0
    for i in range(Qm):
        Cd = ds[i][np.nonzero(ids[i] == prevf[i])[0][0]]
        t = min(k, int((ds[i] <= Cd).sum()))
        assert t >= 1
        assert np.array_equal(knn.reshape(-1, k)[i, :t], ids[i, :t]), i
        assert np.array_equal(kd.reshape(-1, k)[i, :t].astype(np.int64), ds[i, :t]), i
        checked += t
    assert checked > Qm


@pytest.mark.parametrize("alpha", [(1, 4), (1, 2), (3, 4)])
def test_matches_set_assembled_from_the_ring_predicate(alpha):
    # S from the pinned scalar ring test, r_p added once, sorted in Python
    R, KP, frame, prev = synth.random_case(913, 120, 4, 1, 10, 12)
    R[60:] = R[:60]
    prev[0, 0] = 3
    oix = oracle.Index(R, KP)
    k = 6
    knn, kd, count = oracle.riann_knn(oix, frame, prev, k, alpha=alpha, ring_limit=-1)
    Qp = np.lib.stride_tricks.sliding_window_view(frame, (8, 8, 1)).reshape(-1, 64).astype(np.int64)
    Rm = R.reshape(len(R), -1).astype(np.int64)
    Km = KP.reshape(len(KP), -1).astype(np.int64)
    A = ((Rm[:, None, :] - Km[None, :, :]) ** 2).sum(-1)
    prevf = prev.reshape(-1)
    for i, q in enumerate(Qp):
        B = ((Km - q) ** 2).sum(-1)
        d = ((Rm - q) ** 2).sum(-1)
        rp = int(prevf[i])
        Cd = int(d[rp])
        S = [r for r in range(len(R))
             if all(oracle.ring_member(int(A[r, m]), int(B[m]), Cd, *alpha) for m in range(len(Km)))]
        cand = sorted(set(S) | {rp}, key=lambda r: (int(d[r]), r))
        exp = (cand + [-1] * k)[:k]
        assert list(knn.reshape(-1, k)[i]) == exp, i
        assert list(kd.reshape(-1, k)[i]) == [int(d[r]) if r >= 0 else 0xFFFFFFFF for r in exp], i
        assert int(count.reshape(-1)[i]) == len(S)


def test_lists_are_sorted_unique_and_padded():
    R, KP, frame, prev = synth.random_case(914, 64, 6, 3, 11, 15)
    oix = oracle.Index(R, KP)
    k = 8
    knn, kd, count = oracle.riann_knn(oix, frame, prev, k, alpha=(1, 8), ring_limit=-1)
    knn = knn.reshape(-1, k)
    kd = kd.reshape(-1, k).astype(np.int64)
    for i in range(len(knn)):
        valid = knn[i] >= 0
        nv = int(valid.sum())
        assert valid[:nv].all() and not valid[nv:].any()            # padding only at the end
        c = int(count.reshape(-1)[i])
        assert nv == k or c in (nv, nv - 1)                          # |S u {r_p}| = nv when not cut
        key = kd[i, :nv] * 1000 + knn[i, :nv]
        assert (np.diff(key) > 0).all()                              # ascending (dist, index), unique
        assert (kd[i, nv:] == 0xFFFFFFFF).all()
        assert prev.reshape(-1)[i] in knn[i] or nv == k              # r_p is a candidate
