"""Reference-set construction (Sec. 3.4) on the GPU vs the oracle (bit-exact):
the same clusters, numbered alike, with the same median representatives."""
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


def _check(rt, X, leaf):
    import torch
    reps, assign = rt.riann_cluster_references(torch.from_numpy(np.ascontiguousarray(X)).cuda(), leaf)
    oreps, oassign = oracle.cluster_references(X, leaf)
    assert reps.shape[0] == oreps.shape[0], (reps.shape, oreps.shape)
    assert np.array_equal(reps.cpu().numpy(), oreps)
    assert np.array_equal(assign.cpu().numpy(), oassign)
    return len(oreps)


@pytest.mark.parametrize("n,C,leaf,seed", [(1, 1, 1, 0), (2, 1, 1, 1), (1000, 1, 16, 2), (777, 3, 5, 3),
                                           (300, 1, 1, 4), (5000, 1, 300, 5), (4096, 3, 8, 6)])
def test_random_patches(rt, n, C, leaf, seed):
    rng = np.random.default_rng(seed)
    X = rng.integers(0, 256, size=(n, 8, 8, C), dtype=np.uint8)
    if n > 40:
        X[n // 2: n // 2 + 20] = X[:20]                        # duplicates
    _check(rt, X, leaf)


def test_identical_and_two_valued(rt):
    X = np.tile(np.arange(64, dtype=np.uint8).reshape(1, 8, 8, 1), (500, 1, 1, 1))
    assert _check(rt, X, 3) == 1
    Y = np.zeros((600, 8, 8, 1), np.uint8)
    Y[::3, 2, 5, 0] = 200                                      # one coordinate, two values, lopsided
    _check(rt, Y, 7)


def test_synthetic_cuts_large(rt):
    # 262144 cuts of synthetic scenes, clustered to leaves of at most 4
    X = synth.reference_set(16, 262144, 32, 480, 640, 1)
    m = _check(rt, X, 4)
    assert 65536 <= m <= 262144
