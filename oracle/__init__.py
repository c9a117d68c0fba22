"""CPU oracle for RIANN's per-frame query step (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It wraps ``riann_oracle.c`` (plain C99 +
OpenMP) through ctypes and numpy; it shares no code with the CUDA library.

Every function takes numpy arrays in the layouts of ``riann_oracle.h``:
frames uint8 [H][W][C], reference patches uint8 [n][8][8][C], previous ANN
field int32 [H-7][W-7].  ``qidx`` (optional int64 list of query indices
y*(W-7)+x) restricts the work to a sample; outputs then follow the list order.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "riann_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, OpenMP) into oracle/_build/liboracle.so."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if not force and os.path.exists(_LIB_PATH) and \
            os.path.getmtime(_LIB_PATH) >= max(os.path.getmtime(_SRC),
                                                os.path.getmtime(os.path.join(_HERE, "riann_oracle.h"))):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-std=c99", "-O2", "-fopenmp", "-fPIC", "-shared", "-Wall", "-Wextra",
           "-ffp-contract=off", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            P = ctypes.c_void_p
            i32, i64, u32 = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32
            lib.oracle_ring_member.argtypes = [u32, u32, u32, i32, i32]
            lib.oracle_ring_member.restype = ctypes.c_int
            lib.oracle_key_distances.argtypes = [P, i32, i32, P, i32, P]
            lib.oracle_sort_tables.argtypes = [P, i32, i32, P, P]
            lib.oracle_exact_nn.argtypes = [P, i32, i32, i32, P, i32, P, i64, P, P, P]
            lib.oracle_riann_definitional.argtypes = [P, i32, i32, i32, P, i32, P, i32, P, P,
                                                      i32, i32, i32, P, i64, P, P, P, P]
            lib.oracle_riann_indexed.argtypes = [P, i32, i32, i32, P, i32, P, i32, P, P, P, P,
                                                 i32, i32, i32, P, i64, P, P, P, P]
            lib.oracle_riann_knn.argtypes = [P, i32, i32, i32, P, i32, P, i32, P, P,
                                             i32, i32, i32, i32, P, i64, P, P, P]
            lib.oracle_reconstruct.argtypes = [P, i32, i32, P, i32, i32, P, P, P]
            lib.oracle_cluster_references.argtypes = [P, i32, i32, i32, P, P]
            lib.oracle_unit_normalize.argtypes = [P, i32, i32, P]
            lib.oracle_unit_dist.argtypes = [P, P, i32]
            lib.oracle_unit_dist.restype = ctypes.c_float
            lib.oracle_unit_ring_member.argtypes = [ctypes.c_float, ctypes.c_float, ctypes.c_float, i32, i32]
            lib.oracle_unit_ring_member.restype = ctypes.c_int
            lib.oracle_riann_unit.argtypes = [P, i32, i32, i32, P, i32, P, i32, P, i32, i32, i32, P, i64, P, P, P]
            lib.oracle_cluster_references.restype = i32
            lib.oracle_philox4x32_10.argtypes = [P, P, P]
            lib.oracle_random_field.argtypes = [i32, i32, i32, ctypes.c_uint64, u32, P]
            lib.oracle_full_tables.argtypes = [P, i32, i32, P]
            lib.oracle_riann_anchor.argtypes = [P, i32, i32, i32, P, i32, P, P, i32, i32, i32, i32,
                                                ctypes.c_uint64, u32, P, i64, P, P, P, P]
            lib.oracle_num_threads.restype = ctypes.c_int
            lib.oracle_set_num_threads.argtypes = [ctypes.c_int]
            _lib = lib
    return _lib


class use_library:
    """Context manager that routes this module's calls to another build of
    riann_oracle.c (the mutation tests compile deliberately broken copies)."""

    def __init__(self, path: str):
        self.path = path

    def __enter__(self):
        global _lib
        _load()
        self._saved = _lib
        lib = ctypes.CDLL(self.path)
        for name in ("oracle_ring_member", "oracle_key_distances", "oracle_sort_tables", "oracle_exact_nn",
                     "oracle_riann_definitional", "oracle_riann_indexed", "oracle_riann_knn", "oracle_reconstruct", "oracle_cluster_references",
                     "oracle_unit_normalize", "oracle_unit_dist", "oracle_unit_ring_member", "oracle_riann_unit",
                     "oracle_philox4x32_10", "oracle_full_tables", "oracle_riann_anchor", "oracle_random_field",
                     "oracle_num_threads",
                     "oracle_set_num_threads"):
            f, g = getattr(self._saved, name), getattr(lib, name)
            g.argtypes, g.restype = f.argtypes, f.restype
        _lib = lib
        return self

    def __exit__(self, *exc):
        global _lib
        _lib = self._saved


def _ptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def num_threads() -> int:
    return int(_load().oracle_num_threads())


def set_num_threads(n: int) -> None:
    _load().oracle_set_num_threads(int(n))


def ring_member(A: int, B: int, C: int, p: int, q: int) -> bool:
    """Exact |sqrt(A) - sqrt(B)| <= (p/q) sqrt(C)."""
    return bool(_load().oracle_ring_member(A, B, C, p, q))


class Index:
    """Oracle-side pre-processing: key-point distances and sorted per-key lists."""

    def __init__(self, R: np.ndarray, KP: np.ndarray):
        lib = _load()
        self.R = _c(R, np.uint8)
        self.KP = _c(KP, np.uint8)
        self.n = self.R.shape[0]
        self.C = self.R.shape[-1]
        self.D = 64 * self.C
        self.K = self.KP.shape[0]
        assert self.R.shape[1:] == (8, 8, self.C) and self.KP.shape[1:] == (8, 8, self.C)
        self.P = np.empty((self.n, self.K), np.uint32)
        lib.oracle_key_distances(_ptr(self.R), self.n, self.D, _ptr(self.KP), self.K, _ptr(self.P))
        self.TA = np.empty((self.K, self.n), np.uint32)
        self.Tid = np.empty((self.K, self.n), np.int32)
        lib.oracle_sort_tables(_ptr(self.P), self.n, self.K, _ptr(self.TA), _ptr(self.Tid))


def _outputs(frame: np.ndarray, qidx):
    H, W = frame.shape[:2]
    shape = (len(qidx),) if qidx is not None else (H - 7, W - 7)
    return (np.empty(shape, np.int32), np.empty(shape, np.uint32),
            np.empty(shape, np.uint32), np.empty(shape, np.uint32))


def _frame3(frame):
    f = _c(frame, np.uint8)
    return f if f.ndim == 3 else f[:, :, None]


def exact_nn(frame: np.ndarray, R: np.ndarray, qidx=None):
    """Brute-force exact NN field: (annf, dist, count)."""
    lib = _load()
    f = _frame3(frame)
    H, W, C = f.shape
    R = _c(R, np.uint8)
    q = None if qidx is None else _c(qidx, np.int64)
    annf, dist, count, _ = _outputs(f, q)
    lib.oracle_exact_nn(_ptr(f), H, W, C, _ptr(R), R.shape[0], _ptr(q),
                        0 if q is None else len(q), _ptr(annf), _ptr(dist), _ptr(count))
    return annf, dist, count


def riann_frame(index: Index, frame: np.ndarray, prev: Optional[np.ndarray],
                alpha=(1, 4), ring_limit: int = -1, qidx=None, mode: str = "indexed"):
    """One RIANN query step: (annf, dist, count, nseed).

    prev None means frame 0 (brute force).  alpha is (num, den).  ring_limit < 0
    never falls back to brute force.  mode is "indexed" or "definitional".
    """
    lib = _load()
    f = _frame3(frame)
    H, W, C = f.shape
    assert C == index.C
    q = None if qidx is None else _c(qidx, np.int64)
    pv = None if prev is None else _c(prev, np.int32)
    if pv is not None:
        assert pv.shape == (H - 7, W - 7)
    annf, dist, count, nseed = _outputs(f, q)
    nq = 0 if q is None else len(q)
    if mode == "definitional":
        lib.oracle_riann_definitional(_ptr(f), H, W, C, _ptr(index.R), index.n, _ptr(index.KP),
                                      index.K, _ptr(index.P), _ptr(pv), alpha[0], alpha[1],
                                      ring_limit, _ptr(q), nq, _ptr(annf), _ptr(dist),
                                      _ptr(count), _ptr(nseed))
    elif mode == "indexed":
        lib.oracle_riann_indexed(_ptr(f), H, W, C, _ptr(index.R), index.n, _ptr(index.KP),
                                 index.K, _ptr(index.P), _ptr(index.TA), _ptr(index.Tid),
                                 _ptr(pv), alpha[0], alpha[1], ring_limit, _ptr(q), nq,
                                 _ptr(annf), _ptr(dist), _ptr(count), _ptr(nseed))
    else:
        raise ValueError(mode)
    return annf, dist, count, nseed


def cluster_references(X: np.ndarray, leaf: int):
    """Sec. 3.4 reference-set construction: (reps uint8 [m][...patch shape],
    assign int32 [n]) of the regression-tree clustering of the n patches X."""
    lib = _load()
    Xc = _c(X, np.uint8)
    n = Xc.shape[0]
    D = int(np.prod(Xc.shape[1:])) if n else int(np.prod(X.shape[1:]))
    reps = np.empty((max(n, 1), D), np.uint8)
    assign = np.empty(max(n, 1), np.int32)
    m = lib.oracle_cluster_references(_ptr(Xc), n, D, leaf, _ptr(reps), _ptr(assign))
    return reps[:m].reshape((m,) + tuple(X.shape[1:])), assign[:n]


def unit_normalize(X: np.ndarray) -> np.ndarray:
    """Unit-variant normalisation of n patches: float32 [n][D]."""
    lib = _load()
    Xc = _c(X, np.uint8)
    n = Xc.shape[0]
    D = Xc.size // max(n, 1)
    out = np.empty((n, D), np.float32)
    lib.oracle_unit_normalize(_ptr(Xc), n, D, _ptr(out))
    return out


def unit_dist(a: np.ndarray, b: np.ndarray) -> float:
    lib = _load()
    a32, b32 = _c(a, np.float32), _c(b, np.float32)
    return float(lib.oracle_unit_dist(_ptr(a32), _ptr(b32), a32.size))


def unit_ring_member(A: float, B: float, C: float, p: int, q: int) -> bool:
    return bool(_load().oracle_unit_ring_member(A, B, C, p, q))


def riann_unit_frame(R: np.ndarray, KP: np.ndarray, frame: np.ndarray, prev: Optional[np.ndarray],
                     alpha=(1, 4), ring_limit: int = -1, qidx=None):
    """Unit-normalised float variant of one query step: (annf int32, dist float32, count uint32)."""
    lib = _load()
    f = _frame3(frame)
    H, W, C = f.shape
    Rc, Kc = _c(R, np.uint8), _c(KP, np.uint8)
    assert Rc.shape[-1] == C
    q = None if qidx is None else _c(qidx, np.int64)
    pv = None if prev is None else _c(prev, np.int32)
    shape = (len(q),) if q is not None else (H - 7, W - 7)
    annf = np.empty(shape, np.int32)
    dist = np.empty(shape, np.float32)
    count = np.empty(shape, np.uint32)
    lib.oracle_riann_unit(_ptr(f), H, W, C, _ptr(Rc), Rc.shape[0], _ptr(Kc), Kc.shape[0], _ptr(pv),
                          alpha[0], alpha[1], ring_limit, _ptr(q), 0 if q is None else len(q),
                          _ptr(annf), _ptr(dist), _ptr(count))
    return annf, dist, count


def stack_frames(f0: np.ndarray, f1: np.ndarray, f2: np.ndarray) -> np.ndarray:
    """3-D spatio-temporal patches: out[y][x][tau] = f_tau[y][x] (tau = 0 the
    oldest frame), so that the (dy, dx, c) patch of the result at (y, x) is the
    8x8x3 volume of the three frames in (dy, dx, tau) order."""
    fs = [np.asarray(f, np.uint8).reshape(f.shape[0], f.shape[1]) for f in (f0, f1, f2)]
    out = np.empty(fs[0].shape + (3,), np.uint8)
    for tau, f in enumerate(fs):
        out[:, :, tau] = f
    return out


def riann_knn(index: Index, frame: np.ndarray, prev: Optional[np.ndarray], k: int,
              alpha=(1, 4), ring_limit: int = -1, qidx=None):
    """k-NN output of one RIANN query step: (knn [.., k] int32, knn_dist [.., k]
    uint32, count), the k best of the argmin's candidate set (Sec. 7)."""
    lib = _load()
    f = _frame3(frame)
    H, W, C = f.shape
    assert C == index.C and k >= 1
    q = None if qidx is None else _c(qidx, np.int64)
    pv = None if prev is None else _c(prev, np.int32)
    if pv is not None:
        assert pv.shape == (H - 7, W - 7)
    shape = (len(q),) if q is not None else (H - 7, W - 7)
    knn = np.empty(shape + (k,), np.int32)
    kd = np.empty(shape + (k,), np.uint32)
    count = np.empty(shape, np.uint32)
    lib.oracle_riann_knn(_ptr(f), H, W, C, _ptr(index.R), index.n, _ptr(index.KP), index.K,
                         _ptr(index.P), _ptr(pv), alpha[0], alpha[1], ring_limit, k, _ptr(q),
                         0 if q is None else len(q), _ptr(knn), _ptr(kd), _ptr(count))
    return knn, kd, count


def reconstruct(R: np.ndarray, annf: np.ndarray, frame: Optional[np.ndarray] = None):
    """Sec. 4 reconstruction of a frame from its field: (out uint8 [H][W][C],
    err2 = (sum (f_GT - f_R)^2, sum f_GT^2) or None).  R: [n][8][8][C] or
    [n][D]; annf: [H-7][W-7]; frame: [H][W] or [H][W][C] (its shape gives H, W)."""
    lib = _load()
    Rr = _c(R, np.uint8).reshape(R.shape[0], -1)
    n, D = Rr.shape
    C = D // 64
    a = _c(annf, np.int32)
    H, W = a.shape[0] + 7, a.shape[1] + 7
    f = None if frame is None else _frame3(frame)
    if f is not None:
        assert f.shape == (H, W, C)
    out = np.empty((H, W, C), np.uint8)
    err2 = np.zeros(2, np.uint64) if f is not None else None
    lib.oracle_reconstruct(_ptr(Rr), n, C, _ptr(a), H, W, _ptr(f), _ptr(out), _ptr(err2))
    return out, (None if err2 is None else (int(err2[0]), int(err2[1])))


# ---- Alg. 1 with random anchors --------------------------------------------
def philox4x32_10(ctr, key):
    """Philox4x32-10 of a 4-word counter and a 2-word key -> 4 words."""
    lib = _load()
    c = np.asarray(ctr, np.uint32).copy()
    k = np.asarray(key, np.uint32).copy()
    out = np.zeros(4, np.uint32)
    lib.oracle_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return [int(v) for v in out]


class FullIndex:
    """Reference set with the sorted distance matrix of Sec. 3.4:
    T[i][j] = (||r_i - r_id||^2 << 32) | id, each row ascending."""

    def __init__(self, R: np.ndarray):
        lib = _load()
        self.R = _c(R, np.uint8).reshape(R.shape[0], -1)
        self.n, self.D = self.R.shape
        self.C = self.D // 64
        self.T = np.empty((self.n, self.n), np.uint64)
        lib.oracle_full_tables(_ptr(self.R), self.n, self.D, _ptr(self.T))


def riann_anchor_frame(index: FullIndex, frame: np.ndarray, prev: Optional[np.ndarray], alpha=(1, 4),
                       L: int = 20, max_rings: int = 64, seed: int = 0, frame_id: int = 0, qidx=None):
    """Alg. 1 with random anchors: (annf, dist, count, rings); see riann_oracle.h
    for the readings (anchor draw, ring test, final argmin)."""
    lib = _load()
    f = _frame3(frame)
    H, W, C = f.shape
    assert C == index.C
    q = None if qidx is None else _c(qidx, np.int64)
    pv = None if prev is None else _c(prev, np.int32)
    annf, dist, count, rings = _outputs(f, q)
    nq = 0 if q is None else len(q)
    lib.oracle_riann_anchor(_ptr(f), H, W, C, _ptr(index.R), index.n, _ptr(index.T), _ptr(pv),
                            alpha[0], alpha[1], L, max_rings, seed & ((1 << 64) - 1), frame_id & 0xffffffff,
                            _ptr(q), nq, _ptr(annf), _ptr(dist), _ptr(count), _ptr(rings))
    return annf, dist, count, rings


def random_field(H: int, W: int, n: int, seed: int = 0, frame_id: int = 0) -> np.ndarray:
    """Alg. 1's random initial field, 0-based: int32 [H-7][W-7]."""
    lib = _load()
    out = np.empty((H - 7, W - 7), np.int32)
    lib.oracle_random_field(H, W, n, seed & ((1 << 64) - 1), frame_id & 0xffffffff, _ptr(out))
    return out

