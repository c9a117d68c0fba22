"""Pins of the oracle's reference-set construction (Sec. 3.4: regression-tree
clusters represented by their medians).

Each check derives the expected clusters without the oracle's code: numpy
medians of the reported members, constructed inputs whose tree is fixed by
hand (a single varying coordinate, two separated groups, a dominant
coordinate, tied variances), and the partition invariants.
"""
import numpy as np
import pytest

import oracle
from conftest import read_fixture


def _members(assign, m):
    return [np.nonzero(assign == c)[0] for c in range(m)]


@pytest.mark.parametrize("n,D,leaf,seed", [(1000, 64, 16, 0), (777, 192, 5, 1), (64, 64, 64, 2), (300, 64, 1, 3)])
def test_partition_sizes_and_medians(n, D, leaf, seed):
    rng = np.random.default_rng(seed)
    X = rng.integers(0, 256, size=(n, D), dtype=np.uint8)
    X[n // 2: n // 2 + 20] = X[:20]                       # duplicates
    reps, assign = oracle.cluster_references(X, leaf)
    m = len(reps)
    assert assign.shape == (n,) and assign.min() == 0 and assign.max() == m - 1
    for c, mem in enumerate(_members(assign, m)):
        assert len(mem) >= 1
        assert len(mem) <= leaf or (X[mem] == X[mem[0]]).all()
        srt = np.sort(X[mem], axis=0)
        assert np.array_equal(reps[c], srt[(len(mem) - 1) // 2]), c      # per-coordinate lower median


def test_few_patches_one_cluster():
    rng = np.random.default_rng(4)
    X = rng.integers(0, 256, size=(9, 64), dtype=np.uint8)
    reps, assign = oracle.cluster_references(X, 9)
    assert len(reps) == 1 and (assign == 0).all()
    assert np.array_equal(reps[0], np.sort(X, axis=0)[4])


def test_identical_patches_do_not_split():
    X = np.tile(np.arange(64, dtype=np.uint8), (100, 1))
    reps, assign = oracle.cluster_references(X, 4)
    assert len(reps) == 1 and np.array_equal(reps[0], X[0])


def test_two_separated_groups():
    X = np.concatenate([np.zeros((50, 64), np.uint8), np.full((50, 64), 255, np.uint8)])
    perm = np.random.default_rng(5).permutation(100)
    reps, assign = oracle.cluster_references(X[perm], 50)
    assert len(reps) == 2
    # lower median 0: the zeros go left and come first
    assert (reps[0] == 0).all() and (reps[1] == 255).all()
    assert np.array_equal(assign, (X[perm][:, 0] == 255).astype(np.int32))


def test_single_varying_coordinate_gives_value_ranges():
    vals = np.random.default_rng(6).permutation(256).astype(np.uint8)
    X = np.full((256, 64), 77, np.uint8)
    X[:, 5] = vals
    reps, assign = oracle.cluster_references(X, 16)
    assert len(reps) == 16
    for c in range(16):
        mem = np.nonzero(assign == c)[0]
        assert sorted(vals[mem].tolist()) == list(range(16 * c, 16 * c + 16))   # left <= median, left first
        assert reps[c][5] == 16 * c + 7 and (np.delete(reps[c], 5) == 77).all()


def test_split_on_largest_variance():
    X = np.zeros((4, 64), np.uint8)
    X[:, 2] = [0, 0, 200, 200]
    X[:, 7] = [0, 10, 0, 10]
    reps, assign = oracle.cluster_references(X, 2)
    assert len(reps) == 2 and list(assign) == [0, 0, 1, 1]
    assert reps[0][2] == 0 and reps[1][2] == 200 and reps[0][7] == 0 and reps[1][7] == 0


def test_tied_variance_splits_lowest_coordinate():
    X = np.zeros((4, 64), np.uint8)
    X[:, 3] = [0, 100, 0, 100]
    X[:, 1] = [0, 0, 100, 100]
    reps, assign = oracle.cluster_references(X, 2)
    assert list(assign) == [0, 0, 1, 1]


def test_all_at_or_below_the_median_splits_strictly():
    # 6 patches with value 9 and 2 with value 3 in the only varying coordinate:
    # lower median 9 takes everything, so the values below 9 split off
    X = np.zeros((8, 64), np.uint8)
    X[:, 0] = [9, 3, 9, 9, 3, 9, 9, 9]
    reps, assign = oracle.cluster_references(X, 6)
    assert len(reps) == 2 and list(assign) == [1, 0, 1, 1, 0, 1, 1, 1]
    assert reps[0][0] == 3 and reps[1][0] == 9


GOLDEN = ["cluster_constant_patches.txt", "cluster_strict_median.txt", "cluster_largest_variance.txt",
          "cluster_tied_variance.txt", "cluster_variance_not_mean.txt"]


def _golden_patches(fx, key):
    """[m][64] uint8 patches of a fixture: constant values, or `fill` with the
    listed coordinates set per patch."""
    if "coords" not in fx:
        return np.stack([np.full(64, int(v), np.uint8) for v in fx[key].split()])
    coords = [int(c) for c in fx["coords"].split()]
    out = []
    for t in fx[key].split():
        p = np.full(64, int(fx["fill"]), np.uint8)
        p[coords] = [int(v) for v in t.split(",")]
        out.append(p)
    return np.stack(out)


@pytest.mark.parametrize("name", GOLDEN)
def test_golden_fixture(name):
    """Hand-worked trees (tests/golden/cluster_*.txt)."""
    fx = read_fixture(name)
    X = _golden_patches(fx, "values" if "values" in fx else "patches")
    reps, assign = oracle.cluster_references(X.reshape(-1, 8, 8), int(fx["leaf"]))
    want = _golden_patches(fx, "expect_reps")
    assert reps.shape == (len(want), 8, 8)
    assert np.array_equal(reps.reshape(len(want), 64), want)
    assert assign.tolist() == [int(x) for x in fx["expect_assign"].split()]
