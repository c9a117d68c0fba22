"""Host logic of bench.py that decides what it reports (no GPU): the captured
ring-kernel DRAM and L2 traffic is reported only while the kernel sources
hash to the captured digests and the launch variant is the captured one, and
the byte counts follow their stated terms."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

SOURCES = ["paper_1508_07953_gb300/csrc/sparse_query.cu", "paper_1508_07953_gb300/csrc/common.cuh"]


def _current_digests():
    import hashlib
    out = {}
    for rel in SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as f:
            out[rel] = hashlib.sha256(f.read()).hexdigest()
    return out


def _captured(monkeypatch, digests):
    monkeypatch.setitem(bench.RING_CAPTURE, "sha256", digests)
    monkeypatch.setitem(bench.RING_CAPTURE, "dram_bytes", 1.5e9)
    monkeypatch.setitem(bench.RING_CAPTURE, "l2_bytes", 4.0e10)


def test_traffic_reported_for_the_captured_variant(monkeypatch):
    _captured(monkeypatch, _current_digests())
    t = bench.RING_CAPTURE
    assert bench.ring_traffic({"tile_shape": t["tile_shape"], "depth": t["depth"]}) == 1.5e9
    assert bench.ring_traffic(None) == 1.5e9
    assert bench.ring_l2_bytes(None) == 4.0e10


def test_traffic_withheld_for_another_variant(monkeypatch):
    _captured(monkeypatch, _current_digests())
    t = bench.RING_CAPTURE
    assert bench.ring_traffic({"tile_shape": t["tile_shape"], "depth": t["depth"] - 1}) is None
    assert bench.ring_traffic({"tile_shape": 1 - t["tile_shape"], "depth": t["depth"]}) is None
    assert bench.ring_l2_bytes({"tile_shape": 1 - t["tile_shape"], "depth": t["depth"]}) is None


def test_traffic_withheld_when_a_source_changes(monkeypatch):
    digests = _current_digests()
    digests[SOURCES[0]] = "0" * 64
    _captured(monkeypatch, digests)
    assert bench.ring_traffic(None) is None and bench.ring_l2_bytes(None) is None


def test_traffic_withheld_without_a_capture(monkeypatch):
    monkeypatch.setitem(bench.RING_CAPTURE, "sha256", {})
    assert bench.ring_traffic(None) is None


def test_ring_kernel_bytes_model():
    # frame + field + outputs, one row per member of S u {r_p}, the two
    # binary searches per ring for every query
    st = {"ring_queries": 10, "sum_seed": 100, "sum_candidates": 7}
    H, W, n, K = 16, 20, 1023, 4
    Q = (H - 7) * (W - 7)
    exp = H * W + 16 * Q + 64 * (7 + 10) + Q * 2 * K * 10 * 4
    assert bench.ring_kernel_bytes(st, H, W, 1, n, K) == exp
    assert bench.ring_verification_bytes(st, 1) == 64 * 17
    assert bench.ring_verification_bytes(st, 3) == 192 * 17


def test_ring_traffic_model():
    st = {"ring_queries": 10, "sum_seed": 100, "sum_candidates": 7, "sum_filtered": 30, "sum_exact": 9}
    H, W, K = 16, 20, 20
    Q = (H - 7) * (W - 7)
    exp = H * W + 16 * Q + 64 * 10 + 4 * 3 * 100 + (4 + 32) * 30 + 64 * 9
    assert bench.ring_traffic_model(st, H, W, 1, K, 3) == exp
