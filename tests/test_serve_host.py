"""Host-side logic of the served form (no GPU): the arrival trace and the
latency percentiles."""
import numpy as np

import pytest


def _serve():
    from paper_1508_07953_gb300 import serve
    return serve

def test_arrival_trace_is_poisson_with_uniform_lives():
    s = _serve()
    spec = s.ServeSpec(rate=4.0, duration=400.0, seed=3)
    tr = s.arrival_trace(spec, pool_len=16)
    n = len(tr)
    assert abs(n - 1600) < 4 * np.sqrt(1600)          # Poisson count, 4 sigma
    gaps = np.diff([a.t for a in tr])
    assert abs(gaps.mean() - 0.25) < 0.02 and (gaps > 0).all()
    lives = np.array([a.life for a in tr])
    assert lives.min() >= 5.0 and lives.max() <= 20.0 and abs(lives.mean() - 12.5) < 0.5
    fmts = {a.fmt for a in tr}
    assert fmts == set(spec.mix)
    assert all(0 <= a.pool_offset < 16 for a in tr)
    # deterministic in the seed
    assert [(a.t, a.fmt) for a in s.arrival_trace(spec, 16)] == [(a.t, a.fmt) for a in tr]


def test_percentile():
    s = _serve()
    v = list(range(1, 101))
    assert s.percentile(v, 50) == pytest.approx(50.5)
    assert s.percentile(v, 99) == pytest.approx(99.01)
    assert np.isnan(s.percentile([], 50))
