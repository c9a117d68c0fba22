"""Thin Python binding of the RIANN C ABI (include/riann.h).

Argument marshalling only: torch tensors are passed as raw device pointers and
``torch.cuda.Stream`` objects as ``cudaStream_t`` handles.  Every step of the
query path runs in the CUDA library; there is no CPU fallback -- importing this
module raises if ``libriann.so`` has not been built.

Function names match the C entry points.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import torch

# RIANN_LIBRARY=checked selects the checked build (every gathered table index
# tested before the access, RIANN_DEV_BOUNDS on a failure)
_LIB_NAME = "libriann_checked.so" if os.environ.get("RIANN_LIBRARY") == "checked" else "libriann.so"
_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_lib", _LIB_NAME)
if not os.path.exists(_LIB_PATH):
    raise ImportError(
        f"RIANN CUDA library not found at {_LIB_PATH}; build it with "
        "`python -c 'import __graft_entry__ as g; g.build()'`")
_lib = ctypes.CDLL(_LIB_PATH)

RIANN_OK = 0
RIANN_ERR_INVALID_ARG = 1
RIANN_ERR_OOM = 2
RIANN_ERR_UNSUPPORTED = 3
RIANN_ERR_CUDA = 4
RIANN_ERR_TIMEOUT = 5
RIANN_ERR_ADMISSION = 6
RIANN_ERR_DEVICE = 7
RIANN_ERR_TOO_LARGE = 8
RIANN_DEV_BAD_PREV = 0x1
RIANN_DEV_BOUNDS = 0x2
RIANN_DEV_TIMEOUT = 0x4
RIANN_SCAN_AUTO = 0
RIANN_SCAN_PAIRS = 1
RIANN_SCAN_SINGLE = 2


class riann_params(ctypes.Structure):
    _fields_ = [("alpha_num", ctypes.c_int32), ("alpha_den", ctypes.c_int32),
                ("ring_limit", ctypes.c_int32), ("cap", ctypes.c_int32)]

    def __repr__(self):
        return (f"riann_params(alpha={self.alpha_num}/{self.alpha_den}, "
                f"ring_limit={self.ring_limit}, cap={self.cap})")


class riann_index_info_t(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("K", ctypes.c_int32), ("channels", ctypes.c_int32),
                ("dim", ctypes.c_int32), ("device_bytes", ctypes.c_size_t), ("unit", ctypes.c_int32)]


class riann_frame_stats_t(ctypes.Structure):
    _fields_ = [("ring_queries", ctypes.c_uint64), ("dense_queries", ctypes.c_uint64),
                ("sum_seed", ctypes.c_uint64), ("sum_candidates", ctypes.c_uint64),
                ("sum_filtered", ctypes.c_uint64), ("sum_exact", ctypes.c_uint64)]

    def as_dict(self):
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


class riann_session_info_t(ctypes.Structure):
    _fields_ = [("H", ctypes.c_int32), ("W", ctypes.c_int32), ("frames", ctypes.c_int64),
                ("has_field", ctypes.c_int32), ("device_bytes", ctypes.c_size_t)]


class riann_batch_info_t(ctypes.Structure):
    _fields_ = [("max_items", ctypes.c_int32), ("max_queries", ctypes.c_int64),
                ("uses_graph", ctypes.c_int32), ("runs", ctypes.c_int64),
                ("graph_builds", ctypes.c_int64), ("device_bytes", ctypes.c_size_t)]


class riann_tuning_t(ctypes.Structure):
    _fields_ = [("tile_shape", ctypes.c_int32), ("depth", ctypes.c_int32), ("ms", ctypes.c_float)]

    def as_dict(self):
        return {"tile_shape": int(self.tile_shape), "depth": int(self.depth), "ms": float(self.ms)}


_P = ctypes.c_void_p
_i32 = ctypes.c_int32
_i64 = ctypes.c_int64
_lib.riann_default_params.argtypes = [_i32]
_lib.riann_default_params.restype = riann_params
_lib.riann_strerror.argtypes = [ctypes.c_int]
_lib.riann_strerror.restype = ctypes.c_char_p
_lib.riann_build_reference_index.argtypes = [_P, _i32, _i32, _P, _i32, _P, ctypes.POINTER(_P)]
_lib.riann_build_unit_index.argtypes = [_P, _i32, _i32, _P, _i32, _P, ctypes.POINTER(_P)]
_lib.riann_build_reference_index_ex.argtypes = [_P, _i32, _i32, _P, _i32, _i32, _P, ctypes.POINTER(_P)]
_lib.riann_index_destroy.argtypes = [_P]
_lib.riann_index_destroy.restype = None
_lib.riann_index_info.argtypes = [_P, ctypes.POINTER(riann_index_info_t)]
_lib.riann_index_tables.argtypes = [_P, _P, _P, _P, _P]
_lib.riann_annf_frame.argtypes = [_P, ctypes.POINTER(riann_params), _P, _P, _i32, _i32, _P, _P, _P, _P]
_lib.riann_knn_frame.argtypes = [_P, ctypes.POINTER(riann_params), _P, _P, _i32, _i32, _P, _i32, _P, _P, _P, _P]
_lib.riann_exact_nn.argtypes = [_P, _P, _P, _i32, _i32, _P, _P]
_lib.riann_stack_frames.argtypes = [_P, _P, _P, _P, _i32, _i32, _P]
_lib.riann_cluster_references.argtypes = [_P, _P, _i32, _i32, _i32, _P, _P, ctypes.POINTER(_i32)]
_lib.riann_frame_stats.argtypes = [_P, _P, ctypes.POINTER(riann_frame_stats_t)]
_lib.riann_profile_enable.argtypes = [_P, ctypes.c_int]
_lib.riann_profile_read.argtypes = [_P, _P, ctypes.POINTER(ctypes.c_float), _i32]
_lib.riann_exact_nn_noalloc.argtypes = [_P, _P, _P, _i32, _i32, _P, _P]
_lib.riann_test_wait_expiry.argtypes = [_P, _P, _P, _i32, _i32, _P, _i64]
_lib.riann_measure_int_peak.argtypes = [_P, ctypes.POINTER(ctypes.c_double)]
_lib.riann_test_corrupt_offsets.argtypes = [_P, _i32, _i32]
_lib.riann_exact_nn_noalloc_max_queries.argtypes = [_i32]
_lib.riann_exact_nn_noalloc_max_queries.restype = ctypes.c_int64
_lib.riann_session_create.argtypes = [_P, _i32, _i32, ctypes.POINTER(_P)]
_lib.riann_session_destroy.argtypes = [_P]
_lib.riann_session_destroy.restype = None
_lib.riann_session_reset.argtypes = [_P]
_lib.riann_session_info.argtypes = [_P, ctypes.POINTER(riann_session_info_t)]
_lib.riann_session_state_bytes.argtypes = [_P, _i32, _i32]
_lib.riann_session_state_bytes.restype = _i64
_lib.riann_session_frame.argtypes = [_P, ctypes.POINTER(riann_params), _P, _P, _P, _P, _P]
_lib.riann_session_frame_host.argtypes = [_P, ctypes.POINTER(riann_params), _P, _P, _P, _P, _P]
_lib.riann_session_field.argtypes = [_P, _P, _P]
_lib.riann_session_restore.argtypes = [_P, _P, _P]
_lib.riann_session_outputs.argtypes = [_P, ctypes.POINTER(_P), ctypes.POINTER(_P), ctypes.POINTER(_P)]
_lib.riann_session_copy_outputs.argtypes = [_P, _P, _P, _P, _P]
_lib.riann_session_frame_buffer.argtypes = [_P]
_lib.riann_session_frame_buffer.restype = _P
_lib.riann_batch_create.argtypes = [_P, _i32, _i64, _i32, ctypes.POINTER(_P)]
_lib.riann_batch_destroy.argtypes = [_P]
_lib.riann_batch_destroy.restype = None
_lib.riann_batch_run.argtypes = [_P, ctypes.POINTER(riann_params), _P, ctypes.POINTER(_P), ctypes.POINTER(_P), _i32]
_lib.riann_batch_stats.argtypes = [_P, _P, ctypes.POINTER(riann_frame_stats_t)]
_lib.riann_batch_info.argtypes = [_P, ctypes.POINTER(riann_batch_info_t)]
_lib.riann_autotune.argtypes = [_P, ctypes.POINTER(riann_params), _P, _P, _i32, _i32, _P, _i32,
                                ctypes.POINTER(riann_tuning_t), _i32, ctypes.POINTER(_i32)]
_lib.riann_set_tuning.argtypes = [_P, ctypes.POINTER(riann_tuning_t)]
_lib.riann_get_tuning.argtypes = [_P, ctypes.POINTER(riann_tuning_t)]
_lib.riann_server_clock.restype = ctypes.c_double
_lib.riann_server_create.argtypes = [_P, _P, ctypes.c_size_t, _i64, _i32, ctypes.POINTER(riann_params), _i32,
                                     ctypes.c_double, ctypes.POINTER(_P)]
_lib.riann_server_destroy.argtypes = [_P]
_lib.riann_server_destroy.restype = None
_lib.riann_server_open.argtypes = [_P, _i32, _i32, _i32, ctypes.c_double, ctypes.POINTER(_i32)]
_lib.riann_server_close.argtypes = [_P, _i32]
_lib.riann_server_submit.argtypes = [_P, _i32, _P, _i64, ctypes.c_double]
_lib.riann_server_step.argtypes = [_P, _P, _i32, ctypes.POINTER(_i32)]
_lib.riann_server_field.argtypes = [_P, _i32, _P]
_lib.riann_server_stream_counts.argtypes = [_P, _i32, ctypes.POINTER(_i64), ctypes.POINTER(_i64),
                                            ctypes.POINTER(_i64)]
_lib.riann_status.argtypes = [_P, _P, ctypes.POINTER(ctypes.c_uint32)]
_lib.riann_reconstruct.argtypes = [_P, _P, _P, _i32, _i32, _P, _P, _P]
_lib.riann_reconstruct_payload.argtypes = [_P, _P, _P, _i32, _P, _i32, _i32, _P, _P, _P]


class riann_anchor_params(ctypes.Structure):
    _fields_ = [("alpha_num", ctypes.c_int32), ("alpha_den", ctypes.c_int32), ("L", ctypes.c_int32),
                ("max_rings", ctypes.c_int32), ("seed", ctypes.c_uint64), ("frame_id", ctypes.c_uint32)]


_lib.riann_default_anchor_params.restype = riann_anchor_params
_lib.riann_default_anchor_params.argtypes = []
_lib.riann_full_create.argtypes = [_P, _P, ctypes.POINTER(_P)]
_lib.riann_full_destroy.argtypes = [_P]
_lib.riann_full_destroy.restype = None
_lib.riann_full_table.argtypes = [_P, _P, _P]
_lib.riann_anchor_frame.argtypes = [_P, ctypes.POINTER(riann_anchor_params), _P, _P, _i32, _i32, _P, _P, _P, _P, _P]
_lib.riann_anchor_work.argtypes = [_P, _P, _P]
_lib.riann_random_field.argtypes = [_P, _i32, _i32, _i32, ctypes.c_uint64, ctypes.c_uint32, _P]


class RiannError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: {_lib.riann_strerror(code).decode()} (code {code})")
        self.code = code


def _check(code: int, what: str):
    if code != RIANN_OK:
        raise RiannError(code, what)


def library_path() -> str:
    return _LIB_PATH


def _stream(stream: Optional[torch.cuda.Stream]):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dev(t: Optional[torch.Tensor], dtypes, name: str, numel: Optional[int] = None):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype not in dtypes:
        raise ValueError(f"{name} must have dtype in {dtypes}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name} must hold {numel} elements, got {t.numel()}")
    return ctypes.c_void_p(t.data_ptr())


_I32 = (torch.int32,)
_U32 = (torch.int32, torch.uint32)


def riann_default_params(n: int) -> riann_params:
    return _lib.riann_default_params(int(n))


class RiannIndex:
    """Owns a ``riann_index_t``; destroyed with the object (or ``close()``)."""

    def __init__(self, handle: int, n: int, K: int, C: int):
        self.handle = ctypes.c_void_p(handle)
        self.n, self.K, self.C = n, K, C

    def info(self) -> riann_index_info_t:
        out = riann_index_info_t()
        _check(_lib.riann_index_info(self.handle, ctypes.byref(out)), "riann_index_info")
        return out

    def close(self):
        if self.handle and self.handle.value:
            _lib.riann_index_destroy(self.handle)
            self.handle = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def riann_build_reference_index(patches: torch.Tensor, keypoints: torch.Tensor,
                                stream: Optional[torch.cuda.Stream] = None, unit: bool = False,
                                scan_order: Optional[int] = None) -> RiannIndex:
    """patches uint8 [n][8][8][C] and keypoints uint8 [K][8][8][C] on the GPU.
    unit=True builds the unit-normalised float index (riann_build_unit_index);
    scan_order (RIANN_SCAN_*) calls riann_build_reference_index_ex."""
    if patches.dim() != 4 or patches.shape[1:3] != (8, 8):
        raise ValueError("patches must be [n][8][8][C]")
    n, C = patches.shape[0], patches.shape[3]
    if keypoints.dim() != 4 or tuple(keypoints.shape[1:]) != (8, 8, C):
        raise ValueError("keypoints must be [K][8][8][C] with the patches' C")
    K = keypoints.shape[0]
    h = ctypes.c_void_p(0)
    if scan_order is not None:
        if unit:
            raise ValueError("scan_order applies to the integer index")
        _check(_lib.riann_build_reference_index_ex(_dev(patches, (torch.uint8,), "patches"), n, C,
                                                   _dev(keypoints, (torch.uint8,), "keypoints"), K, int(scan_order),
                                                   _stream(stream), ctypes.byref(h)),
               "riann_build_reference_index_ex")
        return RiannIndex(h.value, n, K, C)
    fn = _lib.riann_build_unit_index if unit else _lib.riann_build_reference_index
    _check(fn(_dev(patches, (torch.uint8,), "patches"), n, C, _dev(keypoints, (torch.uint8,), "keypoints"), K,
              _stream(stream), ctypes.byref(h)),
           "riann_build_unit_index" if unit else "riann_build_reference_index")
    return RiannIndex(h.value, n, K, C)


def riann_build_unit_index(patches: torch.Tensor, keypoints: torch.Tensor,
                           stream: Optional[torch.cuda.Stream] = None) -> RiannIndex:
    """Unit-normalised float variant of the index: out_dist of a frame holds
    float32 distances between unit-length patches (view the int32 output as
    torch.float32)."""
    return riann_build_reference_index(patches, keypoints, stream, unit=True)


def _frame_dims(frame: torch.Tensor, C: int):
    if frame.dim() == 2:
        H, W = frame.shape
        fc = 1
    else:
        H, W, fc = frame.shape
    if fc != C:
        raise ValueError(f"frame has {fc} channels, index has {C}")
    return int(H), int(W)


def riann_index_tables(index: RiannIndex, P: Optional[torch.Tensor] = None,
                       TA: Optional[torch.Tensor] = None, Tid: Optional[torch.Tensor] = None,
                       stream: Optional[torch.cuda.Stream] = None) -> None:
    """Copy P [n][K], TA [K][n] (uint32 bits in int32/uint32 tensors) and Tid [K][n] out."""
    nk = index.n * index.K

    def ptr(t, name):
        if t is None:
            return None
        if t.dtype not in _U32 or not t.is_contiguous() or t.numel() != nk:
            raise ValueError(f"{name} must be a contiguous 32-bit tensor of {nk} elements")
        return ctypes.c_void_p(t.data_ptr())

    _check(_lib.riann_index_tables(index.handle, _stream(stream), ptr(P, "P"), ptr(TA, "TA"),
                                   ptr(Tid, "Tid")), "riann_index_tables")


def riann_annf_frame(index: RiannIndex, params: riann_params, frame: torch.Tensor,
                     prev_annf: Optional[torch.Tensor], out_annf: torch.Tensor,
                     out_dist: Optional[torch.Tensor] = None,
                     out_count: Optional[torch.Tensor] = None,
                     stream: Optional[torch.cuda.Stream] = None) -> None:
    """One query step; prev_annf None means frame 0 (brute force)."""
    H, W = _frame_dims(frame, index.C)
    Q = (H - 7) * (W - 7)
    _check(_lib.riann_annf_frame(index.handle, ctypes.byref(params), _stream(stream),
                                 _dev(frame, (torch.uint8,), "frame"), H, W,
                                 _dev(prev_annf, _I32, "prev_annf", Q),
                                 _dev(out_annf, _I32, "out_annf", Q),
                                 _dev(out_dist, _U32, "out_dist", Q),
                                 _dev(out_count, _U32, "out_count", Q)),
           "riann_annf_frame")


RIANN_KNN_MAX = 8


def riann_cluster_references(patches: torch.Tensor, leaf: int, want_assign: bool = True,
                             stream: Optional[torch.cuda.Stream] = None):
    """Sec. 3.4 reference-set construction: returns (reps uint8 [m][8][8][C],
    assign int32 [n] or None), the per-cluster lower medians of the
    regression-tree leaves (at most `leaf` patches each) of the n patches."""
    if patches.dim() != 4 or tuple(patches.shape[1:3]) != (8, 8) or patches.shape[3] not in (1, 3):
        raise ValueError("patches must be uint8 [n][8][8][C], C in {1, 3}")
    n, C = int(patches.shape[0]), int(patches.shape[3])
    reps = torch.empty_like(patches)
    assign = torch.empty(n, dtype=torch.int32, device=patches.device) if want_assign else None
    m = _i32(0)
    _check(_lib.riann_cluster_references(_stream(stream), _dev(patches, (torch.uint8,), "patches", n * 64 * C), n, C,
                                         int(leaf), _dev(reps, (torch.uint8,), "reps", n * 64 * C),
                                         _dev(assign, _I32, "assign", n), ctypes.byref(m)),
           "riann_cluster_references")
    return reps[:m.value], assign


def riann_stack_frames(f0: torch.Tensor, f1: torch.Tensor, f2: torch.Tensor, out: Optional[torch.Tensor] = None,
                       stream: Optional[torch.cuda.Stream] = None) -> torch.Tensor:
    """3-D spatio-temporal patches: three consecutive gray frames [H][W] (or
    [H][W][1]), oldest first, interleaved into one uint8 [H][W][3] frame whose
    (dy, dx, c) patches are the 8x8x3 volumes in (dy, dx, tau) order."""
    H, W = int(f0.shape[0]), int(f0.shape[1])
    for f in (f0, f1, f2):
        if f.numel() != H * W:
            raise ValueError("the three frames must have the same H x W gray shape")
    if out is None:
        out = torch.empty((H, W, 3), dtype=torch.uint8, device=f0.device)
    _check(_lib.riann_stack_frames(_stream(stream), _dev(f0, (torch.uint8,), "f0", H * W),
                                   _dev(f1, (torch.uint8,), "f1", H * W), _dev(f2, (torch.uint8,), "f2", H * W),
                                   H, W, _dev(out, (torch.uint8,), "out", 3 * H * W)),
           "riann_stack_frames")
    return out


def riann_knn_frame(index: RiannIndex, params: riann_params, frame: torch.Tensor,
                    prev_annf: Optional[torch.Tensor], k: int, out_annf: torch.Tensor,
                    out_knn: torch.Tensor, out_knn_dist: Optional[torch.Tensor] = None,
                    out_count: Optional[torch.Tensor] = None,
                    stream: Optional[torch.cuda.Stream] = None) -> None:
    """k-NN query step (Sec. 7): out_knn / out_knn_dist [H-7][W-7][k], the k best
    of the argmin's candidate set in ascending (distance, index) order."""
    H, W = _frame_dims(frame, index.C)
    Q = (H - 7) * (W - 7)
    k = int(k)
    Qk = Q * k if 1 <= k <= RIANN_KNN_MAX else None    # an invalid k is the library's to reject
    _check(_lib.riann_knn_frame(index.handle, ctypes.byref(params), _stream(stream),
                                _dev(frame, (torch.uint8,), "frame"), H, W,
                                _dev(prev_annf, _I32, "prev_annf", Q), k,
                                _dev(out_annf, _I32, "out_annf", Q),
                                _dev(out_knn, _I32, "out_knn", Qk),
                                _dev(out_knn_dist, _U32, "out_knn_dist", Qk),
                                _dev(out_count, _U32, "out_count", Q)),
           "riann_knn_frame")


def riann_reconstruct(index: RiannIndex, annf: torch.Tensor, frame: Optional[torch.Tensor] = None,
                      out: Optional[torch.Tensor] = None, err2: Optional[torch.Tensor] = None,
                      stream: Optional[torch.cuda.Stream] = None) -> None:
    """Sec. 4 reconstruction of the frame from its field (asynchronous).

    annf: int32 [H-7][W-7]; frame (f_GT, optional): uint8 [H][W](C); out
    (optional): uint8 with the frame's element count; err2 (optional, needs
    frame): 2 int64/uint64 elements receiving sum (f_GT - f_R)^2 and sum f_GT^2."""
    if annf.dim() != 2:
        raise ValueError("annf must be [H-7][W-7]")
    H, W = annf.shape[0] + 7, annf.shape[1] + 7
    n = H * W * index.C
    _check(_lib.riann_reconstruct(index.handle, _stream(stream), _dev(annf, _I32, "annf", (H - 7) * (W - 7)), H, W,
                                  _dev(frame, (torch.uint8,), "frame", n), _dev(out, (torch.uint8,), "out", n),
                                  _dev(err2, (torch.int64, torch.uint64), "err2", 2)),
           "riann_reconstruct")


def riann_reconstruct_payload(index: RiannIndex, payload: torch.Tensor, annf: torch.Tensor,
                              frame: Optional[torch.Tensor] = None, out: Optional[torch.Tensor] = None,
                              err2: Optional[torch.Tensor] = None,
                              stream: Optional[torch.cuda.Stream] = None) -> None:
    """Sec. 5 effects (asynchronous): the reconstruction of riann_reconstruct
    with the matched rows taken from payload, uint8 [n][8][8][C'] on the
    device (row r = T(reference r), C' in {1, 3}); frame and out have C'
    channels."""
    if annf.dim() != 2:
        raise ValueError("annf must be [H-7][W-7]")
    if payload.dim() != 4 or tuple(payload.shape[:3]) != (index.n, 8, 8) or payload.shape[3] not in (1, 3):
        raise ValueError("payload must be uint8 [n][8][8][C'] with the index's n and C' in {1, 3}")
    C = int(payload.shape[3])
    H, W = annf.shape[0] + 7, annf.shape[1] + 7
    n = H * W * C
    _check(_lib.riann_reconstruct_payload(index.handle, _stream(stream),
                                          _dev(payload, (torch.uint8,), "payload", index.n * 64 * C), C,
                                          _dev(annf, _I32, "annf", (H - 7) * (W - 7)), H, W,
                                          _dev(frame, (torch.uint8,), "frame", n), _dev(out, (torch.uint8,), "out", n),
                                          _dev(err2, (torch.int64, torch.uint64), "err2", 2)),
           "riann_reconstruct_payload")


def reconstruct(index: RiannIndex, annf: torch.Tensor, frame: Optional[torch.Tensor] = None):
    """Convenience: (f_R uint8 [H][W][C] on the device, E or None); synchronises."""
    H, W = annf.shape[0] + 7, annf.shape[1] + 7
    out = torch.empty((H, W, index.C), dtype=torch.uint8, device=annf.device)
    err2 = torch.zeros(2, dtype=torch.int64, device=annf.device) if frame is not None else None
    riann_reconstruct(index, annf, frame, out, err2)
    if err2 is None:
        return out, None
    e, g = (int(v) for v in err2.cpu())
    return out, (e / g) ** 0.5 if g else 0.0


# ---------------------------------------------------------------------------
# Alg. 1 with random anchors over the sorted distance matrix
# ---------------------------------------------------------------------------
def riann_default_anchor_params() -> riann_anchor_params:
    return _lib.riann_default_anchor_params()


class RiannFull:
    """The sorted distance matrix of an index (n^2 8-byte keys on the device)."""

    def __init__(self, index: RiannIndex, stream: Optional[torch.cuda.Stream] = None):
        h = ctypes.c_void_p(0)
        _check(_lib.riann_full_create(index.handle, _stream(stream), ctypes.byref(h)), "riann_full_create")
        self.handle = h
        self.index = index

    def close(self):
        if self.handle:
            _lib.riann_full_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def riann_full_create(index: RiannIndex, stream=None) -> RiannFull:
    return RiannFull(index, stream)


def riann_full_table(full: RiannFull, stream=None):
    """Host copy of the matrix: numpy uint64 [n][n]."""
    import numpy as np
    n = full.index.n
    out = np.empty((n, n), np.uint64)
    _check(_lib.riann_full_table(full.handle, _stream(stream), out.ctypes.data_as(ctypes.c_void_p)), "riann_full_table")
    return out


def riann_anchor_frame(full: RiannFull, params: riann_anchor_params, frame: torch.Tensor,
                       prev: Optional[torch.Tensor], out_annf: torch.Tensor, out_dist=None, out_count=None,
                       out_rings=None, stream: Optional[torch.cuda.Stream] = None) -> None:
    H, W = _frame_dims(frame, full.index.C)
    Q = (H - 7) * (W - 7)
    _check(_lib.riann_anchor_frame(full.handle, ctypes.byref(params), _stream(stream),
                                   _dev(frame, (torch.uint8,), "frame"), H, W, _dev(prev, _I32, "prev", Q),
                                   _dev(out_annf, _I32, "out_annf", Q), _dev(out_dist, _U32, "out_dist", Q),
                                   _dev(out_count, _U32, "out_count", Q), _dev(out_rings, _U32, "out_rings", Q)),
           "riann_anchor_frame")


def riann_random_field(H: int, W: int, n: int, seed: int, frame_id: int, out: torch.Tensor,
                       stream: Optional[torch.cuda.Stream] = None) -> None:
    """Alg. 1's random initial field into out (int32 [H-7][W-7])."""
    _check(_lib.riann_random_field(_stream(stream), H, W, n, seed & ((1 << 64) - 1), frame_id & 0xffffffff,
                                   _dev(out, _I32, "out", (H - 7) * (W - 7))), "riann_random_field")


def riann_anchor_work(full: RiannFull, stream=None) -> dict:
    """Counters of the last riann_anchor_frame on this handle."""
    buf = (ctypes.c_uint64 * 3)()
    _check(_lib.riann_anchor_work(full.handle, _stream(stream), buf), "riann_anchor_work")
    return {"sum_first_ring": int(buf[0]), "ring_tests": int(buf[1]), "sum_final": int(buf[2])}


def anchor(full: RiannFull, frame: torch.Tensor, prev: Optional[torch.Tensor], params: riann_anchor_params,
           stream=None):
    """Convenience: (annf, dist, count, rings) int32 tensors [H-7][W-7]."""
    H, W = _frame_dims(frame, full.index.C)
    shp = (H - 7, W - 7)
    outs = [torch.empty(shp, dtype=torch.int32, device=frame.device) for _ in range(4)]
    riann_anchor_frame(full, params, frame, prev, *outs, stream=stream)
    return tuple(outs)


def riann_exact_nn(index: RiannIndex, frame: torch.Tensor, out_annf: torch.Tensor,
                   out_dist: Optional[torch.Tensor] = None,
                   stream: Optional[torch.cuda.Stream] = None) -> None:
    H, W = _frame_dims(frame, index.C)
    Q = (H - 7) * (W - 7)
    _check(_lib.riann_exact_nn(index.handle, _stream(stream), _dev(frame, (torch.uint8,), "frame"),
                               H, W, _dev(out_annf, _I32, "out_annf", Q),
                               _dev(out_dist, _U32, "out_dist", Q)),
           "riann_exact_nn")


def riann_test_wait_expiry(index: RiannIndex, frame: torch.Tensor, out_annf: torch.Tensor, spin_cycles: int,
                           stream: Optional[torch.cuda.Stream] = None) -> None:
    """Brute force with every reference tile withheld, so that its bounded
    wait runs out after spin_cycles (see riann.h); read the result with riann_status."""
    H, W = _frame_dims(frame, index.C)
    Q = (H - 7) * (W - 7)
    _check(_lib.riann_test_wait_expiry(index.handle, _stream(stream), _dev(frame, (torch.uint8,), "frame"),
                                       H, W, _dev(out_annf, _I32, "out_annf", Q), int(spin_cycles)),
           "riann_test_wait_expiry")


def riann_test_corrupt_offsets(index: RiannIndex, key: int, extra: int) -> None:
    """Checked-build check: push key `key`'s scan runs `extra` entries past its
    rows (see riann.h).  The index is unusable afterwards."""
    _check(_lib.riann_test_corrupt_offsets(index.handle, int(key), int(extra)), "riann_test_corrupt_offsets")


def library_name() -> str:
    return _LIB_NAME


def riann_measure_int_peak(stream: Optional[torch.cuda.Stream] = None) -> float:
    """Integer operations per second of the absolute-difference / dot-product
    pair the key-point distances use (see riann.h)."""
    v = ctypes.c_double(0.0)
    _check(_lib.riann_measure_int_peak(_stream(stream), ctypes.byref(v)), "riann_measure_int_peak")
    return float(v.value)


def riann_frame_stats(index: RiannIndex, stream: Optional[torch.cuda.Stream] = None) -> dict:
    """Counters of the last frame run on this index (synchronises the stream)."""
    out = riann_frame_stats_t()
    _check(_lib.riann_frame_stats(index.handle, _stream(stream), ctypes.byref(out)),
           "riann_frame_stats")
    return out.as_dict()


RIANN_SLOT_RING = 0
RIANN_SLOT_DENSE = 1
RIANN_SLOT_PREP = 2


def riann_profile_enable(index: RiannIndex, on: bool = True) -> None:
    _check(_lib.riann_profile_enable(index.handle, int(bool(on))), "riann_profile_enable")


def riann_profile_read(index: RiannIndex, stream: Optional[torch.cuda.Stream] = None, nslots: int = 3):
    """Per-kernel milliseconds of the most recent launches (-1: did not run)."""
    buf = (ctypes.c_float * nslots)()
    _check(_lib.riann_profile_read(index.handle, _stream(stream), buf, nslots), "riann_profile_read")
    return [float(x) for x in buf]


def riann_exact_nn_noalloc(index: RiannIndex, frame: torch.Tensor, out_annf: torch.Tensor,
                           out_dist: Optional[torch.Tensor] = None,
                           stream: Optional[torch.cuda.Stream] = None) -> None:
    """Brute force with the library's fixed scratch: allocates nothing (see riann.h)."""
    H, W = _frame_dims(frame, index.C)
    Q = (H - 7) * (W - 7)
    _check(_lib.riann_exact_nn_noalloc(index.handle, _stream(stream),
                                       _dev(frame, (torch.uint8,), "frame"), H, W,
                                       _dev(out_annf, _I32, "out_annf", Q),
                                       _dev(out_dist, _U32, "out_dist", Q)),
           "riann_exact_nn_noalloc")


def riann_exact_nn_noalloc_max_queries(channels: int) -> int:
    return int(_lib.riann_exact_nn_noalloc_max_queries(int(channels)))


def riann_status(index: RiannIndex, stream: Optional[torch.cuda.Stream] = None) -> int:
    """Synchronise and return the device status bits (0 = clean); clears them."""
    bits = ctypes.c_uint32(0)
    _lib.riann_status(index.handle, _stream(stream), ctypes.byref(bits))
    return int(bits.value)


# ---------------------------------------------------------------------------
# convenience: allocate outputs and run a frame
# ---------------------------------------------------------------------------
def annf(index: RiannIndex, frame: torch.Tensor, prev: Optional[torch.Tensor],
         params: Optional[riann_params] = None, stream=None):
    """Allocate outputs and run one frame: returns (annf int32, dist int32, count int32)."""
    H, W = _frame_dims(frame, index.C)
    shape = (H - 7, W - 7)
    dev = frame.device
    out = torch.empty(shape, dtype=torch.int32, device=dev)
    dist = torch.empty(shape, dtype=torch.int32, device=dev)
    cnt = torch.empty(shape, dtype=torch.int32, device=dev)
    riann_annf_frame(index, params if params is not None else riann_default_params(index.n),
                     frame, prev, out, dist, cnt, stream)
    return out, dist, cnt


def knn(index: RiannIndex, frame: torch.Tensor, prev: Optional[torch.Tensor], k: int,
        params: Optional[riann_params] = None, stream=None):
    """Allocate outputs and run one k-NN frame: returns (annf int32 [Hq][Wq],
    knn int32 [Hq][Wq][k], knn_dist int32 [Hq][Wq][k], count int32 [Hq][Wq])."""
    H, W = _frame_dims(frame, index.C)
    shape = (H - 7, W - 7)
    dev = frame.device
    out = torch.empty(shape, dtype=torch.int32, device=dev)
    kn = torch.empty(shape + (int(k),), dtype=torch.int32, device=dev)
    kd = torch.empty(shape + (int(k),), dtype=torch.int32, device=dev)
    cnt = torch.empty(shape, dtype=torch.int32, device=dev)
    riann_knn_frame(index, params if params is not None else riann_default_params(index.n),
                    frame, prev, k, out, kn, kd, cnt, stream)
    return out, kn, kd, cnt


# ---------------------------------------------------------------------------
# sessions (per-stream state)
# ---------------------------------------------------------------------------
RIANN_BATCH_NO_GRAPH = 0x1


class RiannSession:
    """Owns a ``riann_session_t``: one video stream's resident previous field."""

    def __init__(self, index: RiannIndex, H: int, W: int):
        h = ctypes.c_void_p(0)
        _check(_lib.riann_session_create(index.handle, int(H), int(W), ctypes.byref(h)), "riann_session_create")
        self.handle = h
        self.index = index          # keeps the index alive
        self.H, self.W = int(H), int(W)
        self.shape = (self.H - 7, self.W - 7)

    def info(self) -> riann_session_info_t:
        out = riann_session_info_t()
        _check(_lib.riann_session_info(self.handle, ctypes.byref(out)), "riann_session_info")
        return out

    def close(self):
        if self.handle and self.handle.value:
            _lib.riann_session_destroy(self.handle)
            self.handle = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def riann_session_create(index: RiannIndex, H: int, W: int) -> RiannSession:
    return RiannSession(index, H, W)


def riann_session_reset(session: RiannSession) -> None:
    _check(_lib.riann_session_reset(session.handle), "riann_session_reset")


def riann_session_state_bytes(index: RiannIndex, H: int, W: int) -> int:
    return int(_lib.riann_session_state_bytes(index.handle, int(H), int(W)))


def riann_session_frame(session: RiannSession, params: riann_params, frame: torch.Tensor,
                        out_annf: Optional[torch.Tensor] = None, out_dist: Optional[torch.Tensor] = None,
                        out_count: Optional[torch.Tensor] = None,
                        stream: Optional[torch.cuda.Stream] = None) -> None:
    Q = session.shape[0] * session.shape[1]
    _frame_dims(frame, session.index.C)
    _check(_lib.riann_session_frame(session.handle, ctypes.byref(params), _stream(stream),
                                    _dev(frame, (torch.uint8,), "frame"),
                                    _dev(out_annf, _I32, "out_annf", Q), _dev(out_dist, _U32, "out_dist", Q),
                                    _dev(out_count, _U32, "out_count", Q)), "riann_session_frame")


def _host(t: Optional[torch.Tensor], dtypes, name: str, numel: int):
    if t is None:
        return None
    if t.is_cuda or t.dtype not in dtypes or not t.is_contiguous() or t.numel() != numel:
        raise ValueError(f"{name} must be a contiguous CPU tensor of {numel} elements in {dtypes}")
    return ctypes.c_void_p(t.data_ptr())


def riann_session_frame_host(session: RiannSession, params: riann_params, frame: torch.Tensor,
                             out_annf: torch.Tensor, out_dist: Optional[torch.Tensor] = None,
                             out_count: Optional[torch.Tensor] = None,
                             stream: Optional[torch.cuda.Stream] = None) -> None:
    """Host frame in, host field out (pinned host tensors keep it asynchronous)."""
    Q = session.shape[0] * session.shape[1]
    _check(_lib.riann_session_frame_host(session.handle, ctypes.byref(params), _stream(stream),
                                         _host(frame, (torch.uint8,), "frame", session.H * session.W * session.index.C),
                                         _host(out_annf, _I32, "out_annf", Q), _host(out_dist, _U32, "out_dist", Q),
                                         _host(out_count, _U32, "out_count", Q)), "riann_session_frame_host")


def riann_session_field(session: RiannSession, out: torch.Tensor, stream=None) -> None:
    Q = session.shape[0] * session.shape[1]
    if out.dtype != torch.int32 or not out.is_contiguous() or out.numel() != Q:
        raise ValueError("out must be a contiguous int32 tensor of the field's size")
    _check(_lib.riann_session_field(session.handle, _stream(stream), ctypes.c_void_p(out.data_ptr())),
           "riann_session_field")


def riann_session_restore(session: RiannSession, field: torch.Tensor, stream=None) -> None:
    Q = session.shape[0] * session.shape[1]
    if field.dtype != torch.int32 or not field.is_contiguous() or field.numel() != Q:
        raise ValueError("field must be a contiguous int32 tensor of the field's size")
    _check(_lib.riann_session_restore(session.handle, _stream(stream), ctypes.c_void_p(field.data_ptr())),
           "riann_session_restore")


def riann_session_outputs(session: RiannSession):
    """(annf, dist, count) device pointers of the latest frame, as ints."""
    a, d, c = ctypes.c_void_p(0), ctypes.c_void_p(0), ctypes.c_void_p(0)
    _check(_lib.riann_session_outputs(session.handle, ctypes.byref(a), ctypes.byref(d), ctypes.byref(c)),
           "riann_session_outputs")
    return a.value, d.value, c.value


def session_result(session: RiannSession, stream=None):
    """Copies of the latest (annf, dist, count) as int32 CUDA tensors."""
    outs = [torch.empty(session.shape, dtype=torch.int32, device="cuda") for _ in range(3)]
    _check(_lib.riann_session_copy_outputs(session.handle, _stream(stream),
                                           *[ctypes.c_void_p(t.data_ptr()) for t in outs]),
           "riann_session_copy_outputs")
    return tuple(outs)


# ---------------------------------------------------------------------------
# batched form
# ---------------------------------------------------------------------------
class RiannBatch:
    def __init__(self, index: RiannIndex, max_items: int, max_queries: int, use_graph: bool = True):
        h = ctypes.c_void_p(0)
        flags = 0 if use_graph else RIANN_BATCH_NO_GRAPH
        _check(_lib.riann_batch_create(index.handle, int(max_items), int(max_queries), flags, ctypes.byref(h)),
               "riann_batch_create")
        self.handle = h
        self.index = index
        self.max_items = int(max_items)

    def info(self) -> riann_batch_info_t:
        out = riann_batch_info_t()
        _check(_lib.riann_batch_info(self.handle, ctypes.byref(out)), "riann_batch_info")
        return out

    def close(self):
        if self.handle and self.handle.value:
            _lib.riann_batch_destroy(self.handle)
            self.handle = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def riann_batch_create(index: RiannIndex, max_items: int, max_queries: int, use_graph: bool = True) -> RiannBatch:
    return RiannBatch(index, max_items, max_queries, use_graph)


def riann_batch_run(batch: RiannBatch, params: riann_params, sessions, frames, stream=None) -> None:
    """One batched step: frames[i] (CUDA uint8 tensor) is the next frame of sessions[i]."""
    n = len(sessions)
    if n != len(frames):
        raise ValueError("one frame per session")
    hs = (ctypes.c_void_p * n)(*[s.handle.value for s in sessions])
    fs = (ctypes.c_void_p * n)(*[_dev(f, (torch.uint8,), "frame").value for f in frames])
    for s, f in zip(sessions, frames):
        if _frame_dims(f, s.index.C) != (s.H, s.W):
            raise ValueError("frame size differs from its session's")
    _check(_lib.riann_batch_run(batch.handle, ctypes.byref(params), _stream(stream), hs, fs, n), "riann_batch_run")


def riann_batch_stats(batch: RiannBatch, stream=None) -> dict:
    out = riann_frame_stats_t()
    _check(_lib.riann_batch_stats(batch.handle, _stream(stream), ctypes.byref(out)), "riann_batch_stats")
    return out.as_dict()


# ---------------------------------------------------------------------------
# autotuner
# ---------------------------------------------------------------------------
def riann_autotune(index: RiannIndex, params: riann_params, frame: torch.Tensor, prev_annf: torch.Tensor,
                   iters: int = 3, stream=None):
    """Times every ring-kernel variant on one frame; keeps the fastest. Returns all timings."""
    H, W = _frame_dims(frame, index.C)
    res = (riann_tuning_t * 16)()
    nres = ctypes.c_int32(0)
    _check(_lib.riann_autotune(index.handle, ctypes.byref(params), _stream(stream),
                               _dev(frame, (torch.uint8,), "frame"), H, W,
                               _dev(prev_annf, _I32, "prev_annf", (H - 7) * (W - 7)), int(iters),
                               res, 16, ctypes.byref(nres)), "riann_autotune")
    return [res[i].as_dict() for i in range(nres.value)]


def riann_set_tuning(index: RiannIndex, tile_shape: int, depth: int) -> None:
    t = riann_tuning_t(int(tile_shape), int(depth), -1.0)
    _check(_lib.riann_set_tuning(index.handle, ctypes.byref(t)), "riann_set_tuning")


def riann_get_tuning(index: RiannIndex) -> dict:
    t = riann_tuning_t()
    _check(_lib.riann_get_tuning(index.handle, ctypes.byref(t)), "riann_get_tuning")
    return t.as_dict()


# ---------------------------------------------------------------------------
# served form
# ---------------------------------------------------------------------------
RIANN_SERVER_PLAIN = 0x1


class riann_server_result_t(ctypes.Structure):
    _fields_ = [("stream_id", ctypes.c_int32), ("frame_id", ctypes.c_int64),
                ("t_arrival", ctypes.c_double), ("t_done", ctypes.c_double)]


class riann_server_info_t(ctypes.Structure):
    _fields_ = [("open_streams", ctypes.c_int32), ("budget_bytes", ctypes.c_size_t),
                ("used_bytes", ctypes.c_size_t), ("ticks", ctypes.c_int64), ("frames_done", ctypes.c_int64),
                ("queries_done", ctypes.c_int64), ("rejected", ctypes.c_int64), ("submitted", ctypes.c_int64),
                ("dropped", ctypes.c_int64), ("load", ctypes.c_double), ("ns_per_query", ctypes.c_double * 2)]

    def as_dict(self):
        d = {k: int(getattr(self, k)) for k, _ in self._fields_[:9]}
        d["load"] = float(self.load)
        d["ns_per_query"] = [float(x) for x in self.ns_per_query]
        return d


_lib.riann_server_poll.argtypes = [_P, ctypes.POINTER(riann_server_result_t), _i32, ctypes.POINTER(_i32)]
_lib.riann_server_info.argtypes = [_P, ctypes.POINTER(riann_server_info_t)]


def riann_server_clock() -> float:
    return float(_lib.riann_server_clock())


class RiannServer:
    def __init__(self, gray: Optional[RiannIndex], rgb: Optional[RiannIndex], budget_bytes: int,
                 max_tick_queries: int, max_streams: int, params: riann_params, plain: bool = False,
                 load_limit: float = 0.0):
        h = ctypes.c_void_p(0)
        _check(_lib.riann_server_create(gray.handle if gray else None, rgb.handle if rgb else None,
                                        int(budget_bytes), int(max_tick_queries), int(max_streams),
                                        ctypes.byref(params), RIANN_SERVER_PLAIN if plain else 0,
                                        float(load_limit), ctypes.byref(h)), "riann_server_create")
        self.handle = h
        self.indexes = (gray, rgb)
        self._res = (riann_server_result_t * 1024)()

    def open(self, H: int, W: int, C: int, fps: float = 0.0) -> Optional[int]:
        """Admit a stream; None when the memory budget, the tick capacity or
        (with a load limit and fps > 0) the GPU-time budget is full."""
        sid = ctypes.c_int32(-1)
        rc = _lib.riann_server_open(self.handle, int(H), int(W), int(C), float(fps), ctypes.byref(sid))
        if rc == RIANN_ERR_ADMISSION:
            return None
        _check(rc, "riann_server_open")
        return int(sid.value)

    def close_stream(self, sid: int) -> None:
        _check(_lib.riann_server_close(self.handle, int(sid)), "riann_server_close")

    def submit(self, sid: int, frame, frame_id: int, t_arrival: float) -> None:
        """frame: contiguous CPU uint8 tensor or numpy array [H][W][C]."""
        ptr = frame.data_ptr() if isinstance(frame, torch.Tensor) else frame.ctypes.data
        _check(_lib.riann_server_submit(self.handle, int(sid), ctypes.c_void_p(ptr), int(frame_id),
                                        float(t_arrival)), "riann_server_submit")

    def step(self, wait: bool = False, stream=None) -> int:
        n = ctypes.c_int32(0)
        _check(_lib.riann_server_step(self.handle, _stream(stream), int(bool(wait)), ctypes.byref(n)),
               "riann_server_step")
        return int(n.value)

    def poll(self):
        n = ctypes.c_int32(0)
        _check(_lib.riann_server_poll(self.handle, self._res, 1024, ctypes.byref(n)), "riann_server_poll")
        return [(self._res[i].stream_id, self._res[i].frame_id, self._res[i].t_arrival, self._res[i].t_done)
                for i in range(n.value)]

    def field(self, sid: int, out: torch.Tensor) -> None:
        if out.is_cuda or out.dtype != torch.int32 or not out.is_contiguous():
            raise ValueError("out must be a contiguous int32 CPU tensor")
        _check(_lib.riann_server_field(self.handle, int(sid), ctypes.c_void_p(out.data_ptr())), "riann_server_field")

    def counts(self, sid: int):
        a, b, c = ctypes.c_int64(0), ctypes.c_int64(0), ctypes.c_int64(0)
        _check(_lib.riann_server_stream_counts(self.handle, int(sid), ctypes.byref(a), ctypes.byref(b),
                                               ctypes.byref(c)), "riann_server_stream_counts")
        return int(a.value), int(b.value), int(c.value)

    def info(self) -> dict:
        out = riann_server_info_t()
        _check(_lib.riann_server_info(self.handle, ctypes.byref(out)), "riann_server_info")
        return out.as_dict()

    def close(self):
        if self.handle and self.handle.value:
            _lib.riann_server_destroy(self.handle)
            self.handle = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
