"""Real-time front end of the served form (continuous batching of video streams).

Streams arrive as a Poisson process, live for a uniformly drawn time and send
frames at a fixed rate; each frame's arrival time is its nominal capture time.
The server (C++ core, ``riann_server_*``) admits streams while their resident
state fits its device-memory budget and, when it has a load limit, while the
GPU time they claim at their frame rate fits it (a rejected stream retries
until its lifetime would have ended); every step completes the tick in flight
and batches every stream's newest pending frame into the next one.  Frames
that a stream sends faster than the GPU finishes them are replaced by newer
ones (counted as dropped), as a live pipeline would do.  Frame latency =
completion of its tick - its capture time.

The same arrival trace can be replayed through the per-frame path
(``plain=True``) for comparison.
"""
from __future__ import annotations

import dataclasses
from typing import Dict, List, Sequence, Tuple

import numpy as np


@dataclasses.dataclass
class ServeSpec:
    rate: float = 4.0                       # new streams per second (Poisson)
    life: Tuple[float, float] = (5.0, 20.0)  # stream lifetime, uniform (s)
    fps: float = 30.0
    duration: float = 15.0                  # arrivals and frames stop after this (s)
    mix: Sequence[Tuple[int, int, int]] = ((480, 640, 1), (720, 1280, 1), (1080, 1920, 1),
                                          (480, 640, 3), (720, 1280, 3), (1080, 1920, 3))
    seed: int = 7


@dataclasses.dataclass
class Arrival:
    t: float
    fmt: Tuple[int, int, int]
    life: float
    pool_offset: int


def arrival_trace(spec: ServeSpec, pool_len: int = 16) -> List[Arrival]:
    """Poisson arrivals over [0, duration) with uniform lifetimes and formats."""
    rng = np.random.default_rng(spec.seed)
    out, t = [], 0.0
    while True:
        t += float(rng.exponential(1.0 / spec.rate))
        if t >= spec.duration:
            return out
        fmt = tuple(spec.mix[int(rng.integers(len(spec.mix)))])
        out.append(Arrival(t, fmt, float(rng.uniform(*spec.life)), int(rng.integers(pool_len))))


def percentile(values, q: float) -> float:
    if not values:
        return float("nan")
    return float(np.percentile(np.asarray(values, dtype=np.float64), q))


def run(server, pools: Dict[Tuple[int, int, int], list], spec: ServeSpec, trace: List[Arrival] = None) -> dict:
    """Drive `server` (a ``riann.RiannServer``) in real time with the trace;
    return latency/throughput figures.

    pools[(H, W, C)] is a list of consecutive frames (contiguous uint8 CPU
    tensors or arrays) that a stream of that format cycles through."""
    from . import riann
    clock = riann.riann_server_clock
    trace = trace if trace is not None else arrival_trace(spec, min(len(p) for p in pools.values()))
    t0 = clock()
    ai = 0
    waiting: List[Arrival] = []
    active: Dict[int, dict] = {}
    lat: List[float] = []
    per_fmt_lat: Dict[str, List[float]] = {}
    admitted = rejected_final = skipped = 0
    stream_seconds = 0.0
    fmt_of: Dict[int, str] = {}
    while True:
        now = clock() - t0
        while ai < len(trace) and trace[ai].t <= now:
            waiting.append(trace[ai])
            ai += 1
        keep = []
        for a in waiting:
            sid = server.open(*a.fmt, fps=spec.fps)
            if sid is None:
                if now < a.t + a.life:
                    keep.append(a)          # retry while the stream would still be alive
                else:
                    rejected_final += 1
                continue
            admitted += 1
            active[sid] = {"fmt": a.fmt, "start": now, "end": now + a.life, "next": 0, "off": a.pool_offset}
            fmt_of[sid] = f"{a.fmt[0]}p{'rgb' if a.fmt[2] == 3 else ''}"
        waiting = keep
        for sid in [s for s, st in active.items() if now >= st["end"] or now >= spec.duration]:
            st = active.pop(sid)
            stream_seconds += min(now, st["end"]) - st["start"]
            server.close_stream(sid)
        for sid, st in active.items():
            k = int((now - st["start"]) * spec.fps)
            if k >= st["next"]:
                pool = pools[st["fmt"]]
                server.submit(sid, pool[(k + st["off"]) % len(pool)], k, t0 + st["start"] + k / spec.fps)
                skipped += k - st["next"]
                st["next"] = k + 1
        server.step(wait=False)
        for sid, fid, ta, td in server.poll():
            lat.append(td - ta)
            per_fmt_lat.setdefault(fmt_of.get(sid, "?"), []).append(td - ta)
        if now >= spec.duration and not active:
            break
    server.step(wait=True)
    for sid, fid, ta, td in server.poll():
        lat.append(td - ta)
    wall = clock() - t0
    info = server.info()
    frames = len(lat)
    return {
        "streams_admitted": admitted, "streams_rejected": rejected_final + len(waiting),
        "frames_completed": frames, "frames_skipped_before_submit": skipped,
        "frames_replaced_in_queue": info["dropped"],
        "latency_ms_p50": 1e3 * percentile(lat, 50), "latency_ms_p99": 1e3 * percentile(lat, 99),
        "latency_ms_p50_by_format": {k: 1e3 * percentile(v, 50) for k, v in sorted(per_fmt_lat.items())},
        "latency_ms_p99_by_format": {k: 1e3 * percentile(v, 99) for k, v in sorted(per_fmt_lat.items())},
        "frames_by_format": {k: len(v) for k, v in sorted(per_fmt_lat.items())},
        "queries_per_s": info["queries_done"] / max(wall, 1e-9), "wall_s": wall,
        "ns_per_query_measured": info["ns_per_query"],
        "ticks": info["ticks"], "stream_seconds": stream_seconds,
        "fps_per_stream": frames / max(stream_seconds, 1e-9),
    }
