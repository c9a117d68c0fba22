"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

None of these compare the oracle with itself: each checks it against an
independent derivation (hand-worked fixtures, numpy brute force, a decimal
square-root evaluation, the triangle inequality, a reduction to a special case).
"""
import decimal
import itertools

import numpy as np
import pytest

import oracle
import synth
from conftest import read_fixture


# --------------------------------------------------------------------------
# independent helpers (numpy / decimal; no code from the oracle)
# --------------------------------------------------------------------------
def np_patches(frame):
    f = frame if frame.ndim == 3 else frame[:, :, None]
    C = f.shape[2]
    w = np.lib.stride_tricks.sliding_window_view(f, (8, 8, C))
    return w.reshape(-1, 64 * C).astype(np.int64)


def np_exact_nn(frame, R):
    """Exact NN by float64 (integer-exact here) norm expansion; argmin keeps the first index."""
    Qm = np_patches(frame).astype(np.float64)
    Rm = R.reshape(R.shape[0], -1).astype(np.float64)
    rn = (Rm * Rm).sum(1)
    out_i = np.empty(len(Qm), np.int64)
    out_d = np.empty(len(Qm), np.int64)
    for s in range(0, len(Qm), 2048):
        q = Qm[s:s + 2048]
        d = (q * q).sum(1)[:, None] + rn[None, :] - 2.0 * (q @ Rm.T)
        i = d.argmin(1)
        out_i[s:s + 2048] = i
        out_d[s:s + 2048] = np.rint(d[np.arange(len(q)), i]).astype(np.int64)
    return out_i, out_d


decimal.getcontext().prec = 90


def dec_member(A, B, C, p, q):
    """|sqrt A - sqrt B| <= (p/q) sqrt C by 90-digit decimal square roots.

    Returns None when the two sides agree to 1e-60 (an equality that decimal
    cannot separate from a near miss); those cases are pinned separately by
    construction.
    """
    D = decimal.Decimal
    lhs = abs(D(A).sqrt() - D(B).sqrt())
    rhs = D(p) / D(q) * D(C).sqrt()
    if abs(lhs - rhs) < D(10) ** -60:
        return None
    return lhs < rhs


def fixture_case(name):
    fx = read_fixture(name)
    C = int(fx["channels"])

    def vals(s):
        return [tuple(int(x) for x in t.split(",")) for t in s.split()]

    R = np.stack([np.broadcast_to(np.array(v, np.uint8), (8, 8, C)) for v in vals(fx["ref_values"])])
    KP = np.stack([np.broadcast_to(np.array(v, np.uint8), (8, 8, C)) for v in vals(fx["key_values"])])
    frame = np.ascontiguousarray(np.broadcast_to(np.array(vals(fx["query_value"])[0], np.uint8), (8, 8, C)))
    prev = np.array([[int(fx["prev"])]], np.int32)
    a = tuple(int(x) for x in fx["alpha"].split())
    return fx, R, KP, frame, prev, a, int(fx["ring_limit"])


GOLDEN = ["ring_1d_two_keys.txt", "ring_1d_exact_boundary.txt", "ring_1d_prev_kept.txt",
          "ring_1d_limit_bruteforce.txt", "ring_1d_limit_equal.txt", "ring_rgb_two_keys.txt"]


# --------------------------------------------------------------------------
# hand-worked fixtures (Sec. 3.2 rings, Alg. 1)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("name", GOLDEN)
@pytest.mark.parametrize("mode", ["definitional", "indexed"])
def test_golden_fixture(name, mode):
    fx, R, KP, frame, prev, alpha, limit = fixture_case(name)
    idx = oracle.Index(R, KP)
    annf, dist, count, nseed = oracle.riann_frame(idx, frame, prev, alpha=alpha,
                                                  ring_limit=limit, mode=mode)
    assert annf.ravel()[0] == int(fx["expect_annf"])
    assert dist.ravel()[0] == int(fx["expect_dist"])
    assert count.ravel()[0] == int(fx["expect_count"])
    assert nseed.ravel()[0] == int(fx["expect_nseed"])


# --------------------------------------------------------------------------
# the exact ring predicate
# --------------------------------------------------------------------------
def test_ring_member_vs_decimal_random():
    rng = np.random.default_rng(5)
    checked = 0
    for _ in range(4000):
        hi = int(rng.choice([50, 5000, 12_484_800]))
        A, B, C = (int(x) for x in rng.integers(0, hi + 1, size=3))
        q = int(rng.integers(1, 9))
        p = int(rng.integers(0, 8 * q + 1))
        want = dec_member(A, B, C, p, q)
        if want is None:
            continue
        assert oracle.ring_member(A, B, C, p, q) == want, (A, B, C, p, q)
        checked += 1
    assert checked > 3900


def test_ring_member_near_boundary():
    """Cases a few units from the ring edge, where rounding would show."""
    rng = np.random.default_rng(6)
    for _ in range(3000):
        q = int(rng.integers(1, 9))
        p = int(rng.integers(1, 8 * q + 1))
        B = int(rng.integers(0, 12_000_000))
        C = int(rng.integers(0, 12_000_000 // max(1, (p * p) // (q * q) + 1)))
        # real edge of the ring on the upper side: (sqrt B + alpha sqrt C)^2
        edge = (B ** 0.5 + p / q * C ** 0.5) ** 2
        for A in range(max(0, int(edge) - 3), int(edge) + 4):
            if A > 12_484_800 * 4:
                continue
            want = dec_member(A, B, C, p, q)
            if want is not None:
                assert oracle.ring_member(A, B, C, p, q) == want, (A, B, C, p, q)


def test_ring_member_exact_equalities_by_construction():
    """A = a^2 s, B = b^2 s, C = c^2 s: the test is |a - b| q <= p c exactly,
    including irrational square roots (s not a square) and exact equality."""
    rng = np.random.default_rng(7)
    n_eq = 0
    for _ in range(3000):
        s = int(rng.integers(1, 40))
        a, b = (int(x) for x in rng.integers(0, 500, size=2))
        q = int(rng.integers(1, 9))
        p = int(rng.integers(0, 8 * q + 1))
        # pick c so that equality holds when possible, else random
        if p > 0 and (abs(a - b) * q) % p == 0 and rng.random() < 0.7:
            c = abs(a - b) * q // p
        else:
            c = int(rng.integers(0, 500))
        A, B, C = a * a * s, b * b * s, c * c * s
        if max(A, B, C) > 12_484_800:
            continue
        want = abs(a - b) * q <= p * c
        n_eq += abs(a - b) * q == p * c
        assert oracle.ring_member(A, B, C, p, q) == want, (A, B, C, p, q)
    assert n_eq > 100


def test_ring_member_small_grid_exhaustive():
    for A, B, C in itertools.product(range(0, 30), range(0, 30), range(0, 30)):
        for p, q in [(1, 4), (1, 1), (0, 1), (3, 2)]:
            want = dec_member(A, B, C, p, q)
            if want is None:
                # equal to 60 digits: decide by the construction A,B,C perfect-square multiples
                continue
            assert oracle.ring_member(A, B, C, p, q) == want


# --------------------------------------------------------------------------
# exact NN (frame-0 initialisation) vs independent numpy brute force
# --------------------------------------------------------------------------
def test_exact_nn_vs_numpy_random_with_ties():
    rng = np.random.default_rng(8)
    R = rng.integers(0, 256, size=(300, 8, 8, 1), dtype=np.uint8)
    R[150:] = R[:150]                          # duplicates: ties must go to the lower index
    frame = rng.integers(0, 256, size=(24, 30, 1), dtype=np.uint8)
    frame[:8, :8, 0] = R[7, :, :, 0]           # one exact hit
    a, d, c = oracle.exact_nn(frame, R)
    ei, ed = np_exact_nn(frame, R)
    assert (a.ravel() == ei).all() and (d.ravel() == ed).all()
    assert (a.ravel() < 150).all()
    assert a[0, 0] == 7 and d[0, 0] == 0
    assert (c == 300).all()


def test_exact_nn_vs_numpy_rgb():
    rng = np.random.default_rng(9)
    R = rng.integers(0, 256, size=(200, 8, 8, 3), dtype=np.uint8)
    frame = rng.integers(0, 256, size=(16, 20, 3), dtype=np.uint8)
    a, d, _ = oracle.exact_nn(frame, R)
    ei, ed = np_exact_nn(frame, R)
    assert (a.ravel() == ei).all() and (d.ravel() == ed).all()


def test_exact_nn_vs_numpy_tiny_workload():
    w = synth.WORKLOADS["tiny"]
    R = synth.workload_reference(w)
    f = synth.Video(w.video).frame(0)
    a, d, _ = oracle.exact_nn(f, R)
    ei, ed = np_exact_nn(f, R)
    assert (a.ravel() == ei).all() and (d.ravel() == ed).all()


def test_frame0_is_brute_force():
    R, KP, frame, _ = synth.random_case(10, 200, 6, 1, 20, 20)
    idx = oracle.Index(R, KP)
    a0, d0, c0 = oracle.exact_nn(frame, R)
    for mode in ("definitional", "indexed"):
        a, d, c, _ = oracle.riann_frame(idx, frame, None, mode=mode)
        assert (a == a0).all() and (d == d0).all() and (c == 200).all()


# --------------------------------------------------------------------------
# closed-form invariants
# --------------------------------------------------------------------------
@pytest.fixture(scope="module")
def tiny():
    w = synth.WORKLOADS["tiny"]
    R = synth.workload_reference(w)
    KP = synth.workload_keypoints(w, R)
    frames = synth.Video(w.video).frames(0, w.frames)
    return R, KP, frames, oracle.Index(R, KP)


def test_alpha_one_is_exact_nn_every_frame(tiny):
    """alpha = 1: by the triangle inequality every exact NN r* (dist(q, r*) <=
    dist(q, r_p) = eps) lies in every ring, so the field equals exact NN on
    every frame, ties included."""
    R, KP, frames, idx = tiny
    prev = None
    for t in range(len(frames)):
        a, d, c, _ = oracle.riann_frame(idx, frames[t], prev, alpha=(1, 1))
        ei, ed = np_exact_nn(frames[t], R)
        assert (a.ravel() == ei).all(), t
        assert (d.ravel() == ed).all(), t
        prev = a


def test_alpha_zero_profile_match():
    """alpha = 0: a ring keeps exactly the references whose key distance equals
    the query's, so S = references with the query's whole key-distance profile."""
    rng = np.random.default_rng(11)
    base = rng.integers(0, 4, size=(40, 8, 8, 1), dtype=np.uint8) * 60
    R = np.concatenate([base, base[::-1]])       # repeated profiles
    KP = R[[0, 5, 17]].copy()
    frame = np.zeros((8, 16, 1), np.uint8)
    frame[:, :8] = R[3]
    frame[:, 8:] = R[22]
    prev = rng.integers(0, len(R), size=(1, 9)).astype(np.int32)
    idx = oracle.Index(R, KP)
    a, d, c, _ = oracle.riann_frame(idx, frame, prev, alpha=(0, 1))
    Qm = np_patches(frame)
    Rm = R.reshape(len(R), -1).astype(np.int64)
    Km = KP.reshape(len(KP), -1).astype(np.int64)
    for i, q in enumerate(Qm):
        prof_q = ((Km - q) ** 2).sum(1)
        prof_r = ((Km[None] - Rm[:, None]) ** 2).sum(2)
        S = np.nonzero((prof_r == prof_q[None]).all(1))[0]
        rp = int(prev.ravel()[i])
        cand = sorted(set(S.tolist()) | {rp})
        dd = [int(((Rm[r] - q) ** 2).sum()) for r in cand]
        best = min(zip(dd, cand))
        assert a.ravel()[i] == best[1] and d.ravel()[i] == best[0]
        assert c.ravel()[i] == len(S)


def test_monotone_never_worse_than_previous(tiny):
    """r_p is always verified, so dist(q, ANNF_t) <= dist(q, r_p)."""
    R, KP, frames, idx = tiny
    prev, _, _ = oracle.exact_nn(frames[0], R)
    for t in range(1, 4):
        a, d, c, _ = oracle.riann_frame(idx, frames[t], prev)
        Qm = np_patches(frames[t])
        Rm = R.reshape(len(R), -1).astype(np.int64)
        dprev = ((Qm - Rm[prev.ravel()]) ** 2).sum(1)
        assert (d.ravel() <= dprev).all()
        prev = a


def test_keypoint_permutation_invariance(tiny):
    R, KP, frames, idx = tiny
    perm = np.random.default_rng(12).permutation(len(KP))
    idx2 = oracle.Index(R, KP[perm])
    prev, _, _ = oracle.exact_nn(frames[0], R)
    o1 = oracle.riann_frame(idx, frames[1], prev)
    o2 = oracle.riann_frame(idx2, frames[1], prev)
    for x, y in zip(o1, o2):
        assert (x == y).all()


def test_count_bounded_by_smallest_ring(tiny):
    R, KP, frames, idx = tiny
    prev, _, _ = oracle.exact_nn(frames[0], R)
    a, d, c, ns = oracle.riann_frame(idx, frames[1], prev)
    assert (c <= ns).all()


# --------------------------------------------------------------------------
# the index tables; the two oracle modes agree
# --------------------------------------------------------------------------
@pytest.mark.parametrize("C", [1, 3])
def test_index_tables_vs_numpy(C):
    """Sec. 3.3 pre-processing: P = squared distances of every reference to
    every key point, and per key the references sorted by (distance, index),
    derived here with numpy (int64 sums, lexsort)."""
    R, KP, _, _ = synth.random_case(40 + C, 301, 6, C, 8, 8)
    R[200:260] = R[0:60]                       # equal distances: ties by index
    idx = oracle.Index(R, KP)
    Rm = R.reshape(len(R), -1).astype(np.int64)
    Km = KP.reshape(len(KP), -1).astype(np.int64)
    P = ((Rm[:, None, :] - Km[None, :, :]) ** 2).sum(-1)             # [n][K]
    assert np.array_equal(idx.P.reshape(len(R), len(KP)).astype(np.int64), P)
    for m in range(len(KP)):
        order = np.lexsort((np.arange(len(R)), P[:, m]))
        assert np.array_equal(idx.Tid[m], order)
        assert np.array_equal(idx.TA[m].astype(np.int64), P[order, m])


@pytest.mark.parametrize("C", [1, 3])
@pytest.mark.parametrize("alpha", [(1, 4), (1, 2), (0, 1), (1, 1), (7, 8)])
def test_definitional_equals_indexed_random(C, alpha):
    R, KP, frame, prev = synth.random_case(13 + C, 257, 5, C, 19, 23)
    R[100:140] = R[0:40]
    idx = oracle.Index(R, KP)
    for limit in (-1, 0, 30):
        o1 = oracle.riann_frame(idx, frame, prev, alpha=alpha, ring_limit=limit, mode="definitional")
        o2 = oracle.riann_frame(idx, frame, prev, alpha=alpha, ring_limit=limit, mode="indexed")
        for x, y in zip(o1, o2):
            assert (x == y).all()


def test_definitional_equals_indexed_tiny_workload(tiny):
    R, KP, frames, idx = tiny
    prev, _, _ = oracle.exact_nn(frames[0], R)
    for t in (1, 2):
        o1 = oracle.riann_frame(idx, frames[t], prev, mode="definitional")
        o2 = oracle.riann_frame(idx, frames[t], prev, mode="indexed")
        for x, y in zip(o1, o2):
            assert (x == y).all()
        prev = o2[0]


def test_ring_limit_zero_sends_nonempty_rings_to_brute_force(tiny):
    R, KP, frames, idx = tiny
    prev, _, _ = oracle.exact_nn(frames[0], R)
    a, d, c, ns = oracle.riann_frame(idx, frames[1], prev, ring_limit=0)
    ei, ed = np_exact_nn(frames[1], R)
    wide = ns.ravel() > 0
    assert wide.any()
    assert (a.ravel()[wide] == ei[wide]).all() and (c.ravel()[wide] == len(R)).all()


def test_sampled_queries_match_full(tiny):
    R, KP, frames, idx = tiny
    prev, _, _ = oracle.exact_nn(frames[0], R)
    full = oracle.riann_frame(idx, frames[1], prev)
    qs = np.random.default_rng(14).choice(full[0].size, 500, replace=False)
    samp = oracle.riann_frame(idx, frames[1], prev, qidx=qs)
    for x, y in zip(full, samp):
        assert (x.ravel()[qs] == y).all()
