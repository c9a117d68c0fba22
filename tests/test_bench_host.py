"""Host logic of bench.py that decides what it reports (no GPU): the captured
ring-kernel DRAM traffic is reported only while the kernel sources hash to
the captured digests and the launch variant is the captured one."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _current_digests():
    import hashlib
    out = {}
    for rel in bench.RING_TRAFFIC["sha256"]:
        with open(os.path.join(ROOT, rel), "rb") as f:
            out[rel] = hashlib.sha256(f.read()).hexdigest()
    return out


def test_traffic_reported_for_the_captured_variant(monkeypatch):
    # the logic, with the digests taken from the files as they are now
    monkeypatch.setitem(bench.RING_TRAFFIC, "sha256", _current_digests())
    t = bench.RING_TRAFFIC
    got = bench.ring_traffic({"tile_shape": t["tile_shape"], "depth": t["depth"]})
    assert got == t["bytes"]
    assert bench.ring_traffic(None) == t["bytes"]


def test_traffic_withheld_for_another_variant(monkeypatch):
    monkeypatch.setitem(bench.RING_TRAFFIC, "sha256", _current_digests())
    t = bench.RING_TRAFFIC
    assert bench.ring_traffic({"tile_shape": t["tile_shape"], "depth": t["depth"] + 1}) is None
    assert bench.ring_traffic({"tile_shape": 1 - t["tile_shape"], "depth": t["depth"]}) is None


def test_traffic_withheld_when_a_source_changes(monkeypatch):
    digests = dict(bench.RING_TRAFFIC["sha256"])
    first = next(iter(digests))
    digests[first] = "0" * 64
    monkeypatch.setitem(bench.RING_TRAFFIC, "sha256", digests)
    assert bench.ring_traffic(None) is None


def test_ring_kernel_bytes_model():
    # frame + field + outputs, r_p rows, the two binary searches per ring,
    # 8 bytes per seed entry and D per candidate
    st = {"ring_queries": 10, "sum_seed": 100, "sum_candidates": 7}
    H, W, n, K = 16, 20, 1023, 4
    Q = (H - 7) * (W - 7)
    exp = H * W + 16 * Q + 10 * 64 + 10 * 2 * K * 10 * 4 + 8 * 100 + 64 * 7
    assert bench.ring_kernel_bytes(st, H, W, 1, n, K) == exp
