"""Pins of the oracle's unit-normalised float variant (Sec. 3.4 / Alg. 1:
unit-length patches), against float64 arithmetic, exactly representable ring
cases, and the scale invariance that normalisation implies (doubling every
byte changes no normalised vector, so every output is bit-identical)."""
import numpy as np
import pytest

import oracle
import synth
from conftest import read_fixture


def f64_unit(X):
    X = X.reshape(X.shape[0], -1).astype(np.float64)
    nrm = np.sqrt((X * X).sum(1, keepdims=True))
    return np.divide(X, nrm, out=np.zeros_like(X), where=nrm > 0)


def f64_patches(frame):
    f = frame if frame.ndim == 3 else frame[:, :, None]
    C = f.shape[2]
    return np.lib.stride_tricks.sliding_window_view(f, (8, 8, C)).reshape(-1, 64 * C)


def lowest_duplicate_ok(R, idx):
    """True when no reference with a lower index has the same bytes as R[idx]."""
    flat = R.reshape(R.shape[0], -1)
    first = {}
    for i, row in enumerate(flat):
        first.setdefault(row.tobytes(), i)
    return all(first[flat[i].tobytes()] == i for i in np.ravel(idx))


def test_normalisation_matches_float64():
    rng = np.random.default_rng(1)
    X = rng.integers(0, 256, size=(200, 192), dtype=np.uint8)
    X[3] = 0
    X[4] = 0
    X[4, 17] = 9
    got = oracle.unit_normalize(X)
    ref = f64_unit(X)
    assert np.abs(got - ref).max() <= 1.2e-7
    assert (got[3] == 0).all() and got[4, 17] == 1.0
    n2 = (got.astype(np.float64) ** 2).sum(1)
    assert np.abs(n2[np.arange(200) != 3] - 1).max() < 2e-6


@pytest.mark.parametrize("D", [64, 192])
def test_distance_matches_float64(D):
    rng = np.random.default_rng(D)
    A = oracle.unit_normalize(rng.integers(0, 256, size=(50, D), dtype=np.uint8))
    B = oracle.unit_normalize(rng.integers(0, 256, size=(50, D), dtype=np.uint8))
    for a, b in zip(A, B):
        d = oracle.unit_dist(a, b)
        ref = float(np.sqrt(((a.astype(np.float64) - b) ** 2).sum()))
        assert abs(d - ref) <= 2e-5 * ref + 1e-6
    assert oracle.unit_dist(A[0], A[0]) == 0.0


def test_ring_predicate_on_exact_values():
    # powers of two: every quantity and T = (p C) / q are exact
    assert oracle.unit_ring_member(0.75, 0.5, 1.0, 1, 4)          # |0.25| <= 0.25
    assert oracle.unit_ring_member(0.25, 0.5, 1.0, 1, 4)          # lower side, equality
    assert not oracle.unit_ring_member(1.0, 0.5, 1.0, 1, 4)
    assert not oracle.unit_ring_member(0.125, 0.5, 1.0, 1, 4)
    assert oracle.unit_ring_member(1.5, 0.5, 0.5, 2, 1)           # alpha = 2: T = 1
    assert not oracle.unit_ring_member(1.5, 0.5, 0.25, 2, 1)
    assert oracle.unit_ring_member(0.5, 0.5, 0.0, 1, 4)           # C = 0: only A = B


@pytest.mark.parametrize("alpha,limit", [((1, 4), -1), ((1, 2), 30), ((1, 1), -1)])
def test_scale_invariance_bit_exact(alpha, limit):
    R, KP, frame, prev = synth.random_case(71, 300, 6, 1, 14, 20)
    R //= 2
    KP //= 2
    frame //= 2
    a1 = oracle.riann_unit_frame(R, KP, frame, prev, alpha, limit)
    a2 = oracle.riann_unit_frame(R * 2, KP * 2, frame * 2, prev, alpha, limit)
    for x, y in zip(a1, a2):
        assert np.array_equal(x.view(np.uint32), y.view(np.uint32))


@pytest.mark.parametrize("C", [1, 3])
def test_frame0_is_float_brute_force(C):
    R, KP, frame, _ = synth.random_case(72 + C, 400, 4, C, 16, 22)
    R[200:] = R[:200]
    frame[:8, :8] = R[250]
    annf, dist, count = oracle.riann_unit_frame(R, KP, frame, None)
    Qn = f64_unit(f64_patches(frame))
    Rn = f64_unit(R)
    d64 = np.sqrt(((Qn[:, None, :] - Rn[None, :, :]) ** 2).sum(-1))
    best = d64.min(1)
    got = d64[np.arange(len(Qn)), annf.ravel()]
    assert (got - best).max() <= 2e-6                                # the answer is (near-)nearest
    assert (annf.ravel() == d64.argmin(1)).mean() > 0.98
    assert np.abs(dist.ravel() - got).max() <= 2e-6
    assert lowest_duplicate_ok(R, annf) and annf[0, 0] == 50          # R[250] == R[50]: lower index
    assert (count == 400).all()


@pytest.mark.parametrize("alpha,limit", [((1, 4), -1), ((1, 2), 50), ((1, 16), -1)])
def test_exact_previous_match_is_kept(alpha, limit):
    # r_p is always a candidate of the final argmin (Alg. 1 verifies it), so a
    # field that is already the float exact NN (lowest index among equal
    # distances; pinned above) comes back unchanged, with the same distances
    R, KP, frame, _ = synth.random_case(91, 500, 6, 1, 18, 25)
    R[300:] = R[:200]
    e_annf, e_dist, _ = oracle.riann_unit_frame(R, KP, frame, None)
    annf, dist, _ = oracle.riann_unit_frame(R, KP, frame, e_annf, alpha=alpha, ring_limit=limit)
    assert np.array_equal(annf, e_annf)
    assert np.array_equal(dist.view(np.uint32), e_dist.view(np.uint32))


def test_ring_limit_zero_routes_every_nonempty_ring():
    # ring_limit = 0: a query goes to brute force unless some ring is empty;
    # with alpha = 1 every ring holds the exact NN (triangle inequality, up
    # to rounding), so nearly every query is routed and answered as frame 0
    R, KP, frame, prev = synth.random_case(93, 300, 4, 1, 14, 19)
    a, d, c = oracle.riann_unit_frame(R, KP, frame, prev, (1, 1), 0)
    a0, d0, _ = oracle.riann_unit_frame(R, KP, frame, None)
    routed = c == 300
    assert routed.mean() > 0.9
    assert np.array_equal(a[routed], a0[routed])
    assert np.array_equal(d[routed].view(np.uint32), d0[routed].view(np.uint32))


def test_wide_rings_reduce_to_brute_force():
    # alpha = 8: T = 8 C exceeds every |A - B| <= 2 once C > 1/4, so S = R
    R, KP, frame, prev = synth.random_case(74, 300, 5, 1, 12, 18)
    R[150:] = R[:150]
    a, d, c = oracle.riann_unit_frame(R, KP, frame, prev, (8, 1), -1)
    a0, d0, _ = oracle.riann_unit_frame(R, KP, frame, None)
    Cd = np.array([oracle.unit_dist(*oracle.unit_normalize(np.stack([f64_patches(frame)[i].astype(np.uint8),
                                                                        R.reshape(300, -1)[prev.ravel()[i]]])))
                   for i in range(prev.size)])
    wide = Cd > 0.25
    assert wide.mean() > 0.9
    assert np.array_equal(a.ravel()[wide], a0.ravel()[wide]) and (c.ravel()[wide] == 300).all()
    assert lowest_duplicate_ok(R, a)


def test_alpha_one_is_near_exact_nn():
    R, KP, frame, prev = synth.random_case(75, 500, 8, 1, 13, 17)
    a, d, _ = oracle.riann_unit_frame(R, KP, frame, prev, (1, 1), -1)
    Qn = f64_unit(f64_patches(frame))
    Rn = f64_unit(R)
    d64 = np.sqrt(((Qn[:, None, :] - Rn[None, :, :]) ** 2).sum(-1))
    got = d64[np.arange(len(Qn)), a.ravel()]
    assert (got - d64.min(1)).max() <= 1e-5                          # triangle inequality, up to rounding


def _set_patch(spec):
    """8x8x1 gray patch, 200 on the listed pixels (row-major; ranges inclusive), 0 elsewhere."""
    p = np.zeros(64, np.uint8)
    for part in spec.split(","):
        lo, _, hi = part.strip().partition("-")
        p[int(lo): int(hi or lo) + 1] = 200
    return p.reshape(8, 8, 1)


def _f32_sqrt(num, den):
    # float64 sqrt then rounding to float32 is the correctly rounded float32
    # sqrt (53 >= 2 * 24 + 2 bits; no double-rounding error for sqrt)
    return np.float32(np.sqrt(np.float64(num) / np.float64(den)))


@pytest.mark.parametrize("case", ["limit_-1", "limit_5", "limit_6", "zero_query_limit_-1"])
def test_golden_16_pixel_sets(case):
    """Hand-worked unit-length step on exactly representable patches
    (tests/golden/unit_16_pixel_sets.txt)."""
    fx = read_fixture("unit_16_pixel_sets.txt")
    R = np.stack([_set_patch(s) for s in fx["refs"].split(";")])
    KP = np.stack([_set_patch(s) for s in fx["keys"].split(";")])
    zero = case.startswith("zero")
    frame = np.zeros((8, 8, 1), np.uint8) if zero else _set_patch(fx["query"])
    limit = int(case.rsplit("_", 1)[1])
    prev = np.array([[int(fx["prev"])]], np.int32)
    alpha = tuple(int(x) for x in fx["alpha"].split())
    annf, dist, count = oracle.riann_unit_frame(R, KP, frame, prev, alpha=alpha, ring_limit=limit)
    e_annf, e_d2, e_count = fx["expect_" + case].split()
    num, _, den = e_d2.partition("/")
    assert annf.ravel().tolist() == [int(e_annf)]
    assert dist.ravel()[0].view(np.uint32) == _f32_sqrt(int(num), int(den or 1)).view(np.uint32)
    assert count.ravel().tolist() == [int(e_count)]
