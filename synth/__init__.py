"""Seeded synthetic inputs shaped like the workloads of the RIANN paper (Sec. 4).

The paper evaluates on Hollywood2 video at VGA/SVGA/XGA with 8x8 patches and a
reference set of patches cut from natural images (Sec. 3.4, "Building a
reference model"; Sec. 4).  Neither the videos nor the images are available, so
this module draws stand-ins:

* a *scene* is a periodic float texture: a sum of 8 sinusoids of random
  orientation plus Gaussian blobs, per channel;
* a *reference set* is n random 8x8 cuts of a few scenes, quantised to uint8;
* a *video* samples a scene through a per-frame displacement field (global
  sub-pixel drift, or per-64x64-region affine motion), adds N(0, sigma^2) noise
  and quantises to uint8; an optional scene cut swaps in a fresh scene;
* *key points* are reference members picked by k-means++ D^2 seeding.

This module holds none of the matching method's arithmetic: it only makes the
bytes that both the CPU oracle and the CUDA path consume.  Every draw comes from
``numpy.random.default_rng(seed)`` so the same seed gives the same bytes.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional, Sequence

import numpy as np

PATCH = 8  # patch side (Sec. 4 uses 8x8 patches)


# ----------------------------------------------------------------------------
# scenes
# ----------------------------------------------------------------------------
def render_scene(rng: np.random.Generator, H: int, W: int, C: int,
                 n_sin: int = 8, blobs_per_64k: float = 3.0) -> np.ndarray:
    """Return a periodic float32 texture [H][W][C] with values roughly in [0, 255].

    Sinusoids use an integer number of cycles across the texture so the texture
    tiles seamlessly (any displacement can be sampled by wrapping).  Blobs use
    wrapped distances for the same reason.
    """
    yy = np.arange(H, dtype=np.float32)[:, None]
    xx = np.arange(W, dtype=np.float32)[None, :]
    img = np.zeros((H, W, C), dtype=np.float32)
    for _ in range(n_sin):
        lam = rng.uniform(6.0, 48.0)            # wavelength in pixels
        th = rng.uniform(0.0, math.pi)
        kx = max(1, int(round(W * abs(math.cos(th)) / lam))) * (1 if math.cos(th) >= 0 else -1)
        ky = max(1, int(round(H * abs(math.sin(th)) / lam)))
        ph = rng.uniform(0.0, 2 * math.pi)
        amp = rng.uniform(8.0, 28.0)
        col = rng.uniform(0.5, 1.5, size=C).astype(np.float32) if C > 1 else np.ones(1, np.float32)
        wave = np.sin(2 * math.pi * (kx * xx / W + ky * yy / H) + ph).astype(np.float32)
        img += (amp * wave)[:, :, None] * col[None, None, :]
    n_blob = max(6, int(round(blobs_per_64k * H * W / 65536.0)))
    for _ in range(n_blob):
        cy, cx = rng.uniform(0, H), rng.uniform(0, W)
        sig = rng.uniform(3.0, 24.0)
        amp = rng.uniform(-70.0, 70.0)
        col = rng.uniform(0.5, 1.5, size=C).astype(np.float32) if C > 1 else np.ones(1, np.float32)
        r = int(math.ceil(3.5 * sig))
        ys = (np.arange(int(cy) - r, int(cy) + r + 1) % H)
        xs = (np.arange(int(cx) - r, int(cx) + r + 1) % W)
        dy = (np.arange(int(cy) - r, int(cy) + r + 1) - cy).astype(np.float32)
        dx = (np.arange(int(cx) - r, int(cx) + r + 1) - cx).astype(np.float32)
        g = np.exp(-(dy[:, None] ** 2 + dx[None, :] ** 2) / (2 * sig * sig)).astype(np.float32)
        img[np.ix_(ys, xs)] += (amp * g)[:, :, None] * col[None, None, :]
    img += 128.0
    return img


def quantise(x: np.ndarray) -> np.ndarray:
    """Round to nearest and clip to uint8."""
    return np.clip(np.rint(x), 0, 255).astype(np.uint8)


def bilinear_wrap(tex: np.ndarray, Y: np.ndarray, X: np.ndarray) -> np.ndarray:
    """Sample the periodic texture at float coordinates (Y, X) with bilinear weights."""
    H, W, _ = tex.shape
    y0 = np.floor(Y)
    x0 = np.floor(X)
    fy = (Y - y0).astype(np.float32)[..., None]
    fx = (X - x0).astype(np.float32)[..., None]
    y0 = y0.astype(np.int64) % H
    x0 = x0.astype(np.int64) % W
    y1 = (y0 + 1) % H
    x1 = (x0 + 1) % W
    top = tex[y0, x0] * (1 - fx) + tex[y0, x1] * fx
    bot = tex[y1, x0] * (1 - fx) + tex[y1, x1] * fx
    return top * (1 - fy) + bot * fy


# ----------------------------------------------------------------------------
# reference sets and key points
# ----------------------------------------------------------------------------
def reference_set(seed: int, n: int, n_images: int, H: int, W: int, C: int) -> np.ndarray:
    """n random 8x8 cuts from n_images synthetic scenes: uint8 [n][8][8][C] (dy, dx, c order)."""
    rng = np.random.default_rng(seed)
    imgs = [quantise(render_scene(rng, H, W, C)) for _ in range(n_images)]
    which = rng.integers(0, n_images, size=n)
    ys = rng.integers(0, H - PATCH + 1, size=n)
    xs = rng.integers(0, W - PATCH + 1, size=n)
    out = np.empty((n, PATCH, PATCH, C), dtype=np.uint8)
    for i in range(n):
        out[i] = imgs[which[i]][ys[i]:ys[i] + PATCH, xs[i]:xs[i] + PATCH]
    return out


def reference_volumes(seed: int, n: int, n_videos: int, H: int, W: int, T: int = 3) -> np.ndarray:
    """n random 8x8xT spatio-temporal cuts (T consecutive frames) of n_videos
    synthetic gray videos: uint8 [n][8][8][T], (dy, dx, tau) order, tau = 0
    the oldest frame.  Each video has 8 frames of region motion."""
    rng = np.random.default_rng(seed)
    vids = []
    for _ in range(n_videos):
        spec = VideoSpec(H, W, 1, int(rng.integers(1 << 30)), speeds=(0.0, 0.5, 2.0, 6.0), noise_sigma=2.0)
        vids.append(Video(spec).frames(0, 8)[..., 0])            # [8][H][W]
    which = rng.integers(0, n_videos, size=n)
    ts = rng.integers(0, 8 - T + 1, size=n)
    ys = rng.integers(0, H - PATCH + 1, size=n)
    xs = rng.integers(0, W - PATCH + 1, size=n)
    out = np.empty((n, PATCH, PATCH, T), dtype=np.uint8)
    for i in range(n):
        v = vids[which[i]][ts[i]:ts[i] + T, ys[i]:ys[i] + PATCH, xs[i]:xs[i] + PATCH]   # [T][8][8]
        out[i] = np.moveaxis(v, 0, -1)
    return out


def keypoints_kmeanspp(R: np.ndarray, K: int, seed: int) -> tuple[np.ndarray, np.ndarray]:
    """k-means++ D^2 seeding over the reference set; returns (indices, patches).

    The first centre is uniform; each next one is drawn with probability
    proportional to its squared distance to the nearest centre chosen so far.
    Key points are reference members, so their bytes are those of R.
    """
    rng = np.random.default_rng(seed)
    n = R.shape[0]
    X = R.reshape(n, -1).astype(np.int64)
    first = int(rng.integers(0, n))
    idx = [first]
    d2 = ((X - X[first]) ** 2).sum(1)
    for _ in range(1, K):
        tot = float(d2.sum())
        if tot <= 0:
            nxt = int(rng.integers(0, n))
        else:
            nxt = int(rng.choice(n, p=d2.astype(np.float64) / tot))
        idx.append(nxt)
        d2 = np.minimum(d2, ((X - X[nxt]) ** 2).sum(1))
    idx = np.asarray(idx, dtype=np.int64)
    return idx, np.ascontiguousarray(R[idx])


# ----------------------------------------------------------------------------
# video
# ----------------------------------------------------------------------------
@dataclasses.dataclass
class VideoSpec:
    H: int
    W: int
    C: int
    seed: int
    motion: str = "region"              # "global" (sub-pixel drift <= max_shift) or "region"
    speeds: Sequence[float] = (0.0, 0.5, 2.0, 6.0)
    max_shift: float = 1.0
    noise_sigma: float = 2.0
    cut_every: Optional[int] = None     # scene cut period in frames
    region: int = 64
    affine: float = 0.002               # max |entry| of the per-region affine rate (1/frame)


class Video:
    """Deterministic synthetic video; ``frame(t)`` returns uint8 [H][W][C].

    Frames are generated independently from (seed, t), so any frame can be
    drawn without its predecessors.
    """

    def __init__(self, spec: VideoSpec):
        self.spec = spec
        self._scenes: dict[int, tuple] = {}

    def _scene(self, shot: int):
        if shot not in self._scenes:
            s = self.spec
            rng = np.random.default_rng([s.seed, shot, 7])
            tex = render_scene(rng, s.H, s.W, s.C)
            ry = (s.H + s.region - 1) // s.region
            rx = (s.W + s.region - 1) // s.region
            sp = rng.choice(np.asarray(s.speeds, dtype=np.float64), size=(ry, rx))
            th = rng.uniform(0, 2 * math.pi, size=(ry, rx))
            vel = np.stack([sp * np.sin(th), sp * np.cos(th)], -1)        # (vy, vx) px/frame
            aff = rng.uniform(-s.affine, s.affine, size=(ry, rx, 2, 2))
            self._scenes[shot] = (tex, vel, aff)
            if len(self._scenes) > 4:
                self._scenes.pop(min(self._scenes))
        return self._scenes[shot]

    def _drift(self, shot: int, t: int) -> tuple[float, float]:
        """Cumulative global displacement after t frames (each step within max_shift)."""
        rng = np.random.default_rng([self.spec.seed, shot, 11])
        r = self.spec.max_shift * np.sqrt(rng.uniform(0, 1, size=t))
        a = rng.uniform(0, 2 * math.pi, size=t)
        return float((r * np.sin(a)).sum()), float((r * np.cos(a)).sum())

    def frame(self, t: int) -> np.ndarray:
        s = self.spec
        shot, tt = (t // s.cut_every, t % s.cut_every) if s.cut_every else (0, t)
        tex, vel, aff = self._scene(shot)
        Y = np.arange(s.H, dtype=np.float32)[:, None]
        X = np.arange(s.W, dtype=np.float32)[None, :]
        if s.motion == "global":
            dy, dx = self._drift(shot, tt)
            Ys, Xs = Y - np.float32(dy), X - np.float32(dx)
        else:
            ry = np.arange(s.H) // s.region
            rx = np.arange(s.W) // s.region
            cy = ((ry + 0.5) * s.region).astype(np.float32)[:, None]
            cx = ((rx + 0.5) * s.region).astype(np.float32)[None, :]
            v = vel.astype(np.float32)[ry][:, rx]            # [H][W][2]
            A = aff.astype(np.float32)[ry][:, rx]            # [H][W][2][2]
            py, px = Y - cy, X - cx
            f = np.float32(tt)
            dy = f * (v[..., 0] + A[..., 0, 0] * py + A[..., 0, 1] * px)
            dx = f * (v[..., 1] + A[..., 1, 0] * py + A[..., 1, 1] * px)
            Ys, Xs = Y - dy, X - dx
        img = bilinear_wrap(tex, np.broadcast_to(Ys, (s.H, s.W)), np.broadcast_to(Xs, (s.H, s.W)))
        noise = np.random.default_rng([s.seed, t, 13]).standard_normal(size=img.shape, dtype=np.float32)
        return quantise(img + np.float32(s.noise_sigma) * noise)

    def frames(self, t0: int, t1: int) -> np.ndarray:
        return np.stack([self.frame(t) for t in range(t0, t1)])


# ----------------------------------------------------------------------------
# the workloads (sizes, seeds, distributions)
# ----------------------------------------------------------------------------
@dataclasses.dataclass
class Workload:
    name: str
    n: int
    K: int
    C: int
    ref_images: int
    ref_hw: tuple
    ref_seed: int
    video: VideoSpec
    frames: int
    kp_seed: int = 11
    volumes: bool = False     # references are 8x8xC spatio-temporal cuts of gray videos (C frames)


WORKLOADS = {
    # 4096 gray refs from 16 128x128 images (seed 1); 16 key points; 8 frames of
    # 128x128 (seed 2) with sub-pixel global drift <= 1 px/frame and N(0, 2^2) noise.
    "tiny": Workload("tiny", 4096, 16, 1, 16, (128, 128), 1,
                     VideoSpec(128, 128, 1, 2, motion="global", noise_sigma=2.0), 8),
    # 16384 RGB refs from 64 1280x720 images; 32 key points; 60 frames of 720p RGB,
    # per-64x64-region affine motion at speeds {0, 0.5, 2, 6} px/frame, N(0, 3^2).
    "720p_rgb": Workload("720p_rgb", 16384, 32, 3, 64, (720, 1280), 3,
                         VideoSpec(720, 1280, 3, 4, speeds=(0.0, 0.5, 2.0, 6.0), noise_sigma=3.0), 60),
    # 65536 gray refs, 64 key points; 120 frames of 1080p gray with region motion
    # and a scene cut every 40 frames.
    "1080p": Workload("1080p", 65536, 64, 1, 64, (1080, 1920), 5,
                      VideoSpec(1080, 1920, 1, 6, speeds=(0.0, 0.5, 2.0, 6.0), noise_sigma=2.0,
                                cut_every=40), 120),
}

# 3-D spatio-temporal patches: 8x8x3 volumes (three consecutive gray frames) of
# the 1080p video against 65536 reference volumes cut from 16 synthetic 480x640
# gray videos (seed 14), 64 key volumes.
WORKLOADS["1080p_st"] = Workload("1080p_st", 65536, 64, 3, 16, (480, 640), 14, WORKLOADS["1080p"].video, 120,
                                 volumes=True)
WORKLOADS["tiny_st"] = Workload("tiny_st", 4096, 16, 3, 8, (128, 128), 15, WORKLOADS["tiny"].video, 8,
                                volumes=True)

# Batched form: 32 gray streams (8 at each size) sharing a 16384-patch, 32-key index;
# per-stream speeds drawn from {0.25, 1, 4} px/frame; stream s uses seed 1000 + s.
BATCH_SIZES = [(240, 320)] * 8 + [(480, 640)] * 8 + [(720, 1280)] * 8 + [(1080, 1920)] * 8
BATCH_INDEX = Workload("batch_index", 16384, 32, 1, 64, (720, 1280), 8,
                       VideoSpec(720, 1280, 1, 9), 60)


# Served form: an RGB index (65536 patches, 64 key points) beside the 1080p gray
# one; streams of 480p / 720p / 1080p, gray or RGB, region motion, N(0, 2^2).
SERVE_RGB_INDEX = Workload("serve_rgb", 65536, 64, 3, 32, (720, 1280), 12,
                           VideoSpec(720, 1280, 3, 13), 60)
SERVE_FORMATS = ((480, 640, 1), (720, 1280, 1), (1080, 1920, 1), (480, 640, 3), (720, 1280, 3), (1080, 1920, 3))


def serve_frame_pool(fmt, n_frames: int, seed: int) -> list:
    """n_frames consecutive frames of one synthetic stream of format (H, W, C)."""
    H, W, C = fmt
    v = Video(VideoSpec(H, W, C, seed, speeds=(0.0, 0.5, 2.0, 6.0), noise_sigma=2.0))
    return [v.frame(t) for t in range(n_frames)]


def batch_stream_spec(s: int) -> VideoSpec:
    H, W = BATCH_SIZES[s]
    rng = np.random.default_rng(1000 + s)
    sp = float(rng.choice([0.25, 1.0, 4.0]))
    return VideoSpec(H, W, 1, 1000 + s, speeds=(sp,), noise_sigma=2.0)


def workload_reference(w: Workload) -> np.ndarray:
    H, W = w.ref_hw
    if w.volumes:
        return reference_volumes(w.ref_seed, w.n, w.ref_images, H, W, w.C)
    return reference_set(w.ref_seed, w.n, w.ref_images, H, W, w.C)


def workload_keypoints(w: Workload, R: np.ndarray) -> np.ndarray:
    return keypoints_kmeanspp(R, w.K, w.kp_seed)[1]


def random_case(seed: int, n: int, K: int, C: int, H: int, W: int):
    """A small random (R, KP, frame, prev) case of uniform bytes, for edge-case tests."""
    rng = np.random.default_rng(seed)
    R = rng.integers(0, 256, size=(n, PATCH, PATCH, C), dtype=np.uint8)
    KP = R[rng.choice(n, size=K, replace=K > n)].copy()
    frame = rng.integers(0, 256, size=(H, W, C), dtype=np.uint8)
    prev = rng.integers(0, n, size=(H - PATCH + 1, W - PATCH + 1), dtype=np.int32)
    return R, KP, frame, prev
