"""Pins of the oracle's Alg. 1 with random anchors (the paper's own loop:
first ring around the previous match, then rings around random members of
the candidate set until fewer than L remain)."""
import os

import numpy as np
import pytest

import oracle
import synth

HERE = os.path.dirname(os.path.abspath(__file__))
M32 = 0xFFFFFFFF


def test_philox_known_answers():
    for line in open(os.path.join(HERE, "golden", "philox4x32_10_kat.txt")):
        if line.startswith("#") or not line.strip():
            continue
        v = [int(t, 16) for t in line.split()]
        assert oracle.philox4x32_10(v[0:4], v[4:6]) == v[6:10]


def philox_py(ctr, key):
    """Philox4x32-10 from its published definition, in Python integers."""
    c0, c1, c2, c3 = ctr
    k0, k1 = key
    for _ in range(10):
        p0, p1 = 0xD2511F53 * c0, 0xCD9E8D57 * c2
        c0, c1, c2, c3 = ((p1 >> 32) ^ c1 ^ k0) & M32, p1 & M32, ((p0 >> 32) ^ c3 ^ k1) & M32, p0 & M32
        k0, k1 = (k0 + 0x9E3779B9) & M32, (k1 + 0xBB67AE85) & M32
    return [c0, c1, c2, c3]


def test_python_philox_agrees():
    rng = np.random.default_rng(0)
    for _ in range(50):
        c = [int(x) for x in rng.integers(0, 1 << 32, 4)]
        k = [int(x) for x in rng.integers(0, 1 << 32, 2)]
        assert oracle.philox4x32_10(c, k) == philox_py(c, k)


def test_full_tables_are_sorted_distance_rows():
    R = np.random.default_rng(1).integers(0, 256, (300, 64), dtype=np.uint8)
    fi = oracle.FullIndex(R)
    Ri = R.astype(np.int64)
    A = ((Ri[:, None, :] - Ri[None]) ** 2).sum(-1)
    for i in range(300):
        order = np.lexsort((np.arange(300), A[i]))
        assert np.array_equal(fi.T[i] & M32, order)
        assert np.array_equal(fi.T[i] >> np.uint64(32), A[i][order])


def ring(A, B, p, q):
    """anchor ring in integers: (q-p)^2 B <= q^2 A <= (q+p)^2 B (lower side only when p < q)"""
    lo = (q - p) ** 2 * B <= q * q * A if p < q else np.ones_like(A, bool)
    return lo & (q * q * A <= (q + p) ** 2 * B)


def patches(f):
    H, W, C = f.shape
    return np.stack([f[y:y + 8, x:x + 8].reshape(-1) for y in range(H - 7) for x in range(W - 7)]).astype(np.int64)


def anchor_py(R, frame, prev, alpha, L, max_rings, seed, frame_id):
    """Independent implementation of the loop (numpy sets, Python Philox)."""
    p, q = alpha
    Ri = R.reshape(R.shape[0], -1).astype(np.int64)
    Qs = patches(frame if frame.ndim == 3 else frame[:, :, None])
    out = []
    for qi, qv in enumerate(Qs):
        ri = int(prev.reshape(-1)[qi])
        dq = ((Ri - qv) ** 2).sum(1)
        Ari = ((Ri - Ri[ri]) ** 2).sum(1)
        order = np.lexsort((np.arange(len(Ri)), Ari))          # row r_i of the sorted matrix
        S = [j for j in order if ring(Ari[j], dq[ri], p, q)]
        seen = [ri]
        t = 0
        while len(S) >= L and t < max_rings:
            x = philox_py([qi, t, frame_id, 0], [seed & M32, seed >> 32])[0]
            a = S[(x * len(S)) >> 32]
            seen.append(a)
            Aa = ((Ri - Ri[a]) ** 2).sum(1)
            S = [j for j in S if ring(Aa[j], dq[a], p, q)]
            t += 1
        cand = sorted(set(S) | set(seen))
        best = min(cand, key=lambda j: (dq[j], j))
        out.append((best, dq[best], len(S), t))
    return [np.array(v).reshape(prev.shape) for v in zip(*out)]


@pytest.mark.parametrize("alpha,L", [((1, 4), 20), ((1, 4), 3), ((1, 2), 5), ((3, 1), 4), ((1, 8), 1)])
def test_matches_independent_implementation(alpha, L):
    R, _, frame, prev = synth.random_case(20 + L, 120, 1, 1, 12, 14)
    frame = (frame // 32).astype(np.uint8) * 32          # coarse values: many ties and shared distances
    R = (R // 32).astype(np.uint8) * 32
    fi = oracle.FullIndex(R)
    got = oracle.riann_anchor_frame(fi, frame, prev, alpha=alpha, L=L, max_rings=16, seed=0x1234ABCD5678, frame_id=7)
    want = anchor_py(R, frame, prev, alpha, L, 16, 0x1234ABCD5678, 7)
    for g, w in zip(got, want):
        assert np.array_equal(g.astype(np.int64), w.astype(np.int64))


def test_alpha_one_is_exact_nn():
    # triangle inequality: |d(a, r*) - d(a, q)| <= d(q, r*) <= d(q, a) for the exact NN r*
    # and any anchor a at least as far, so r* stays in every ring
    w = synth.WORKLOADS["tiny"]
    R = synth.workload_reference(w)[:700]
    frames = synth.Video(w.video).frames(0, 3)[:, :40, :56]
    fi = oracle.FullIndex(R)
    prev, _, _ = oracle.exact_nn(frames[0], R)
    for t in (1, 2):
        a, d, c, k = oracle.riann_anchor_frame(fi, frames[t], prev, alpha=(1, 1), L=4, seed=9, frame_id=t)
        ea, ed, _ = oracle.exact_nn(frames[t], R)
        assert np.array_equal(a, ea) and np.array_equal(d, ed)
        prev = a


def test_no_loop_is_first_ring_argmin():
    R, _, frame, prev = synth.random_case(31, 200, 1, 1, 10, 11)
    fi = oracle.FullIndex(R)
    a, d, c, k = oracle.riann_anchor_frame(fi, frame, prev, alpha=(1, 4), L=10 ** 6)
    Ri = R.reshape(200, -1).astype(np.int64)
    for qi, qv in enumerate(patches(frame)):
        ri = prev.reshape(-1)[qi]
        dq = ((Ri - qv) ** 2).sum(1)
        S0 = np.nonzero(ring(((Ri - Ri[ri]) ** 2).sum(1), dq[ri], 1, 4))[0]
        cand = np.union1d(S0, [ri])
        best = cand[np.lexsort((cand, dq[cand]))[0]]
        assert a.reshape(-1)[qi] == best and c.reshape(-1)[qi] == len(S0) and k.reshape(-1)[qi] == 0
        assert d.reshape(-1)[qi] <= dq[ri]


@pytest.mark.parametrize("alpha,L", [((1, 4), 20), ((1, 4), 2), ((1, 2), 10 ** 6)])
def test_exact_previous_match_is_kept(alpha, L):
    # Alg. 1 keeps r_i among the candidates of the final argmin, so a query
    # whose previous match is already its exact NN (lowest index among equal
    # distances) returns it, whatever the rings and anchors hold
    w = synth.WORKLOADS["tiny"]
    R = synth.workload_reference(w)[:900]
    frame = synth.Video(w.video).frames(0, 2)[1][:36, :44]
    fi = oracle.FullIndex(R)
    ea, ed, _ = oracle.exact_nn(frame, R)
    a, d, c, k = oracle.riann_anchor_frame(fi, frame, ea, alpha=alpha, L=L, seed=5, frame_id=1)
    assert np.array_equal(a, ea) and np.array_equal(d, ed)


def test_ties_at_the_minimum_go_to_the_lowest_index():
    # every reference is the query (128 everywhere) with one pixel raised by
    # 10, so all lie at squared distance 100 from it and 200 from each other;
    # r_i = 0.  Rings (alpha = 1/2) around any of them hold every other one,
    # so anchors are drawn until fewer than L remain, each tying with r_i.
    # The answer is r_i = 0, the lowest index at the minimum.
    n = 40
    R = np.full((n, 64), 128, np.uint8)
    R[np.arange(n), np.arange(n)] = 138
    R = R.reshape(n, 8, 8, 1)
    frame = np.full((8, 8, 1), 128, np.uint8)
    prev = np.zeros((1, 1), np.int32)
    fi = oracle.FullIndex(R)
    for seed in (1, 2, 3):
        a, d, c, k = oracle.riann_anchor_frame(fi, frame, prev, alpha=(1, 2), L=4, seed=seed)
        assert (a.item(), d.item(), c.item(), k.item()) == (0, 100, 3, 36)


def test_identical_references_stop_at_the_ring_cap():
    # every reference equals the query: each anchor's ring keeps all of S, so
    # only the cap ends the loop; the answer is the lowest index at distance 0
    R = np.full((40, 8, 8, 1), 100, np.uint8)
    frame = np.full((9, 9, 1), 100, np.uint8)
    prev = np.full((2, 2), 17, np.int32)
    fi = oracle.FullIndex(R)
    a, d, c, k = oracle.riann_anchor_frame(fi, frame, prev, L=20, max_rings=5)
    assert (a == 0).all() and (d == 0).all() and (c == 40).all() and (k == 5).all()


def test_golden_candidate_set_of_exactly_L():
    d = {}
    for line in open(os.path.join(HERE, "golden", "anchor_loop_at_L.txt")):
        line = line.strip()
        if line and not line.startswith("#"):
            k, v = line.split(":", 1)
            d[k.strip()] = [int(t) for t in v.split()]
    R = np.stack([np.full((8, 8, 1), v, np.uint8) for v in d["ref_values"]])
    frame = np.full((d["H"][0], d["W"][0], 1), d["query_value"][0], np.uint8)
    prev = np.full((d["H"][0] - 7, d["W"][0] - 7), d["prev"][0], np.int32)
    fi = oracle.FullIndex(R)
    for seed in (0, 1, 2, 3, 12345):          # the outcome does not depend on the anchor drawn
        a, dist, c, k = oracle.riann_anchor_frame(fi, frame, prev, alpha=tuple(d["alpha"]), L=d["L"][0], seed=seed)
        assert (int(a[0, 0]), int(dist[0, 0]), int(c[0, 0]), int(k[0, 0])) == (
            d["expect_annf"][0], d["expect_dist"][0], d["expect_count"][0], d["expect_rings"][0])


def test_random_field_definition_and_range():
    H, W, n, seed, fid = 20, 31, 777, 0xABCDEF0123, 5
    f = oracle.random_field(H, W, n, seed, fid)
    want = [(philox_py([q, 0, fid, 1], [seed & M32, seed >> 32])[0] * n) >> 32 for q in range((H - 7) * (W - 7))]
    assert np.array_equal(f.reshape(-1), np.array(want))
    big = oracle.random_field(300, 300, 10, 1)          # roughly uniform over [0, n)
    counts = np.bincount(big.reshape(-1), minlength=10)
    assert counts.min() > 0.9 * big.size / 10 and counts.max() < 1.1 * big.size / 10
