"""Python binding of the matcher's C ABI (include/mpv.h), by ctypes.

Argument marshalling only: every step of the matcher runs in libmpv.so's CUDA kernels.
Device tensors are torch tensors (uint8 images, uint16 maps stored in int16/uint16
tensors), streams are torch CUDA streams.  If the library is missing the import of
this module fails loudly: there is no CPU path.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
# MPV_LIBRARY selects another build of the library (the bounds-checked libmpv_debug.so)
LIB_PATH = os.environ.get("MPV_LIBRARY") or os.path.join(HERE, "libmpv.so")

MPV_OK = 0
MPV_ERR_INVALID_ARG = 1
MPV_ERR_UNSUPPORTED = 2
MPV_ERR_OOM = 3
MPV_ERR_CUDA = 4
MPV_ERR_TIMEOUT = 5
MPV_ERR_INTERNAL = 6
MPV_INVALID = 0xFFFF
MPV_NO_TRUNC = 0x7FFFFFFF
MPV_MERGE_SUM = 0
MPV_MERGE_PAPER = 1
MPV_PROPOSAL_PYRAMID = 0
MPV_PROPOSAL_LEARNED = 1
MPV_FALLBACK_NONE = 0
MPV_FALLBACK_PYRAMID = 1
MPV_FALLBACK_FULL = 2
MPV_BATCH_AUTO = 0
MPV_BATCH_PERSISTENT = 1
MPV_BATCH_STREAMS = 2


class MpvError(RuntimeError):
    def __init__(self, status, what=""):
        self.status = status
        super().__init__(f"{what}: {mpv_status_string(status)} ({status})")


class mpv_params(C.Structure):
    _fields_ = [
        ("struct_size", C.c_uint32),
        ("max_disparity", C.c_int32),
        ("num_scales", C.c_int32),
        ("num_paths", C.c_int32),
        ("p1", C.c_int32),
        ("trunc", C.c_int32),
        ("ssim_window", C.c_int32),
        ("window", C.c_int32),
        ("block", C.c_int32 * 4),
        ("lr_check", C.c_int32),
        ("lr_tol", C.c_int32),
        ("merge_mode", C.c_int32),
        ("proposal", C.c_int32),
        ("top_block", C.c_int32),
        ("windows", C.c_int32 * 4),
        ("fallback", C.c_int32),
        ("fallback_edge_bp", C.c_int32),
    ]


class mpv_completion(C.Structure):
    _fields_ = [
        ("request_id", C.c_uint64),
        ("camera", C.c_int32),
        ("status", C.c_int),
        ("t_submit_ms", C.c_double),
        ("t_start_ms", C.c_double),
        ("t_done_ms", C.c_double),
    ]


class mpv_pair(C.Structure):
    _fields_ = [
        ("left", C.c_void_p),
        ("right", C.c_void_p),
        ("width", C.c_int32),
        ("height", C.c_int32),
        ("pitch", C.c_int32),
        ("max_disparity", C.c_int32),
        ("disp", C.c_void_p),
        ("disp_pitch", C.c_int32),
        ("disp_right", C.c_void_p),
    ]


EXPORTS = [
    "mpv_default_params", "mpv_create", "mpv_set_params", "mpv_get_params", "mpv_match",
    "mpv_match_host", "mpv_match_batch", "mpv_load_proposal_weights", "mpv_sync",
    "mpv_set_gradient_penalty", "mpv_road_detect", "mpv_server_set_proposal",
    "mpv_workspace_bytes", "mpv_set_workspace_limit", "mpv_debug_stage", "mpv_level_info",
    "mpv_status_string", "mpv_destroy", "mpv_profile_enable", "mpv_profile_read",
    "mpv_match_noalloc", "mpv_autotune", "mpv_server_create", "mpv_server_add_camera",
    "mpv_server_submit", "mpv_server_poll", "mpv_server_stats", "mpv_server_destroy",
    "mpv_cnn_conv3x3", "mpv_cnn_conv3x3_wgrad", "mpv_cnn_flip_transpose",
    "mpv_cnn_relu_backward", "mpv_cnn_huber", "mpv_cnn_adam", "mpv_cnn_to_bf16",
    "mpv_cnn_target", "mpv_proposal_features", "mpv_proposal_stats", "mpv_proposal_predict",
    "mpv_proposal_fallbacks", "mpv_batch_info", "mpv_debug_batch_stall", "mpv_set_batch_mode",
]
MPV_NOALLOC_SCRATCH_BYTES = 64 << 20
MPV_STAGES = ("pyramid", "seed", "cost", "aggregate", "wta", "lr")

_lib = None


def load(path: str = LIB_PATH):
    """Loads libmpv.so (built by paper_2001_09678_gb300.build) and declares its symbols."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libmpv.so not built at {path}; run paper_2001_09678_gb300/build.py")
    L = C.CDLL(path)
    vp, i32, ctx = C.c_void_p, C.c_int32, C.c_void_p
    pp = C.POINTER(mpv_params)
    L.mpv_default_params.argtypes = [pp]
    L.mpv_create.argtypes = [C.c_int, C.POINTER(C.c_void_p)]
    L.mpv_set_params.argtypes = [ctx, pp]
    L.mpv_get_params.argtypes = [ctx, pp]
    L.mpv_match.argtypes = [ctx, vp, vp, i32, i32, i32, vp, i32, vp]
    L.mpv_match_host.argtypes = [ctx, vp, vp, i32, i32, i32, vp, i32, vp]
    L.mpv_match_batch.argtypes = [ctx, C.POINTER(mpv_pair), i32, vp]
    L.mpv_load_proposal_weights.argtypes = [ctx, C.c_char_p]
    L.mpv_set_gradient_penalty.argtypes = [ctx, C.POINTER(C.c_int32)]
    L.mpv_road_detect.argtypes = [ctx, vp, i32, i32, i32, i32, i32, vp, vp, vp, vp, vp]
    L.mpv_sync.argtypes = [ctx]
    L.mpv_workspace_bytes.argtypes = [ctx, i32, i32, C.POINTER(C.c_size_t)]
    L.mpv_set_workspace_limit.argtypes = [ctx, C.c_size_t]
    L.mpv_debug_stage.argtypes = [ctx, vp, vp, i32, i32, i32, i32, i32, vp, vp, vp, vp, vp]
    L.mpv_level_info.argtypes = [ctx, i32, i32, i32] + [C.POINTER(i32)] * 4
    L.mpv_status_string.argtypes = [C.c_int]
    L.mpv_status_string.restype = C.c_char_p
    L.mpv_profile_enable.argtypes = [ctx, i32]
    L.mpv_profile_read.argtypes = [ctx, C.POINTER(C.c_double), C.POINTER(C.c_int64), i32]
    L.mpv_match_noalloc.argtypes = [pp, vp, vp, i32, i32, i32, vp, i32, vp]
    L.mpv_autotune.argtypes = [ctx, C.POINTER(mpv_pair), C.POINTER(i32)]
    L.mpv_server_create.argtypes = [C.c_int, pp, C.c_size_t, i32, C.POINTER(C.c_void_p)]
    L.mpv_server_add_camera.argtypes = [vp, i32, i32, i32, i32]
    L.mpv_server_set_proposal.argtypes = [vp, C.c_char_p]
    L.mpv_server_submit.argtypes = [vp, i32, vp, vp, i32, vp, i32, C.c_uint64]
    L.mpv_server_poll.argtypes = [vp, C.POINTER(mpv_completion), i32, C.POINTER(i32)]
    L.mpv_server_stats.argtypes = [vp, C.POINTER(i32), C.POINTER(i32), C.POINTER(C.c_size_t),
                                   C.POINTER(C.c_uint64), C.POINTER(i32)]
    L.mpv_server_destroy.argtypes = [vp]
    fp = C.POINTER(C.c_float)
    i64 = C.c_int64
    L.mpv_cnn_conv3x3.argtypes = [vp, i32, i32, i32, i32, i32, vp, vp, i32, i32, vp, vp, vp]
    L.mpv_cnn_conv3x3_wgrad.argtypes = [vp, i32, i32, vp, i32, i32, i32, vp, vp, vp]
    L.mpv_cnn_flip_transpose.argtypes = [vp, i32, i32, vp, vp]
    L.mpv_cnn_relu_backward.argtypes = [vp, vp, vp, i64, vp]
    L.mpv_cnn_huber.argtypes = [vp, vp, C.c_float, i64, vp, vp, vp]
    L.mpv_cnn_adam.argtypes = [vp, vp, vp, vp, i64, C.c_float, C.c_float, C.c_float, C.c_float,
                               i32, vp, vp]
    L.mpv_cnn_to_bf16.argtypes = [vp, vp, i64, vp]
    L.mpv_cnn_target.argtypes = [vp, i32, i32, i32, i32, i32, vp, vp]
    L.mpv_proposal_predict.argtypes = [ctx, vp, vp, i32, i32, i32, i32, vp, vp]
    L.mpv_proposal_features.argtypes = [ctx, vp, vp, i32, i32, i32, i32, vp, vp]
    L.mpv_proposal_stats.argtypes = [ctx, C.POINTER(C.c_uint64), C.POINTER(C.c_uint64)]
    L.mpv_proposal_fallbacks.argtypes = [ctx, C.POINTER(C.c_uint64), C.POINTER(C.c_uint64)]
    L.mpv_batch_info.argtypes = [ctx] + [C.POINTER(i32)] * 4 + [C.POINTER(C.c_float)] * 2 + [C.POINTER(i32)]
    L.mpv_debug_batch_stall.argtypes = [ctx, C.c_int64]
    L.mpv_set_batch_mode.argtypes = [ctx, i32]
    L.mpv_destroy.argtypes = [ctx]
    L.mpv_destroy.restype = None
    L.mpv_server_destroy.restype = None
    for name in EXPORTS:
        f = getattr(L, name)
        if name not in ("mpv_status_string", "mpv_destroy", "mpv_server_destroy"):
            f.restype = C.c_int
    _lib = L
    return L


def _check(st, what):
    if st != MPV_OK:
        raise MpvError(st, what)


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


# ---- C ABI, one Python function per entry point ----------------------------------

def mpv_status_string(status: int) -> str:
    return load().mpv_status_string(status).decode()


def mpv_default_params(**overrides) -> mpv_params:
    p = mpv_params()
    _check(load().mpv_default_params(C.byref(p)), "mpv_default_params")
    for k, v in overrides.items():
        if k in ("block", "windows"):
            blk = list(v) + [0] * (4 - len(v))
            arr = getattr(p, k)
            for i in range(4):
                arr[i] = blk[i]
        else:
            setattr(p, k, v)
    return p


def mpv_create(device: int = 0) -> C.c_void_p:
    h = C.c_void_p()
    _check(load().mpv_create(device, C.byref(h)), "mpv_create")
    return h


def mpv_set_params(ctx, p: mpv_params) -> None:
    _check(load().mpv_set_params(ctx, C.byref(p)), "mpv_set_params")


def mpv_get_params(ctx) -> mpv_params:
    p = mpv_params()
    _check(load().mpv_get_params(ctx, C.byref(p)), "mpv_get_params")
    return p


def mpv_match(ctx, left, right, disp, stream=None) -> None:
    """left, right: uint8 CUDA tensors [H, W] (rows may be padded); disp: 16-bit [H, W']."""
    H, W = left.shape[-2], left.shape[-1]
    _check(load().mpv_match(ctx, _ptr(left), _ptr(right), W, H, left.stride(-2), _ptr(disp),
                            disp.stride(-2), _stream(stream)), "mpv_match")


def mpv_match_host(ctx, left, right, disp, stream=None) -> None:
    """Host (CPU) tensors or numpy arrays; copies in and out inside the call."""
    def addr(a):
        return a.data_ptr() if hasattr(a, "data_ptr") else a.ctypes.data

    def rowstride(a):
        return a.stride(-2) if hasattr(a, "data_ptr") else a.strides[-2] // a.itemsize

    H, W = left.shape[-2], left.shape[-1]
    _check(load().mpv_match_host(ctx, C.c_void_p(addr(left)), C.c_void_p(addr(right)), W, H,
                                 rowstride(left), C.c_void_p(addr(disp)), rowstride(disp),
                                 _stream(stream)), "mpv_match_host")


def _pairs(pairs):
    arr = (mpv_pair * len(pairs))()
    for i, q in enumerate(pairs):
        left = q["left"]
        arr[i].left = left.data_ptr()
        arr[i].right = q["right"].data_ptr()
        arr[i].height, arr[i].width = left.shape[-2], left.shape[-1]
        arr[i].pitch = left.stride(-2)
        arr[i].max_disparity = q.get("max_disparity", 0)
        arr[i].disp = q["disp"].data_ptr()
        arr[i].disp_pitch = q["disp"].stride(-2)
        dr = q.get("disp_right")
        arr[i].disp_right = dr.data_ptr() if dr is not None else None
    return arr


def mpv_match_batch(ctx, pairs, stream=None) -> None:
    """pairs: list of dicts with left, right, disp tensors and optional max_disparity,
    disp_right."""
    arr = _pairs(pairs)
    _check(load().mpv_match_batch(ctx, arr, len(pairs), _stream(stream)), "mpv_match_batch")


def mpv_autotune(ctx, pair) -> int:
    """Tunes the launch shapes for pair's shape; returns the chosen lanes per path."""
    arr = _pairs([pair])
    lanes = C.c_int32()
    _check(load().mpv_autotune(ctx, arr, C.byref(lanes)), "mpv_autotune")
    return lanes.value


def mpv_set_gradient_penalty(ctx, slopes) -> None:
    """256 integer jump slopes indexed by |I0(p) - I0(p-r)| (None: plain p1)."""
    if slopes is None:
        _check(load().mpv_set_gradient_penalty(ctx, None), "mpv_set_gradient_penalty")
        return
    a = np.ascontiguousarray(slopes, dtype=np.int32)
    if a.shape != (256,):
        raise ValueError("the gradient table has 256 entries")
    _check(load().mpv_set_gradient_penalty(ctx, a.ctypes.data_as(C.POINTER(C.c_int32))),
           "mpv_set_gradient_penalty")


def mpv_road_detect(ctx, disp, max_disparity: int, eta: int, vdisp, profile, energy,
                    udisp=None, stream=None) -> None:
    """disp: [H][W] uint16 (int16 view) device tensor; vdisp [H][D] and udisp [W][D]
    int32 tensors (uint32 counts), profile [D] int32, energy [1] int64."""
    H, W = disp.shape[-2], disp.shape[-1]
    _check(load().mpv_road_detect(ctx, _ptr(disp), W, H, disp.stride(-2), max_disparity, eta,
                                  _ptr(vdisp), _ptr(udisp), _ptr(profile), _ptr(energy),
                                  _stream(stream)), "mpv_road_detect")


def mpv_load_proposal_weights(ctx, path: str) -> None:
    _check(load().mpv_load_proposal_weights(ctx, path.encode()), "mpv_load_proposal_weights")


def mpv_sync(ctx) -> None:
    _check(load().mpv_sync(ctx), "mpv_sync")


def mpv_workspace_bytes(ctx, width: int, height: int) -> int:
    n = C.c_size_t()
    _check(load().mpv_workspace_bytes(ctx, width, height, C.byref(n)), "mpv_workspace_bytes")
    return n.value


def mpv_set_workspace_limit(ctx, nbytes: int) -> None:
    _check(load().mpv_set_workspace_limit(ctx, nbytes), "mpv_set_workspace_limit")


def mpv_debug_stage(ctx, left, right, view, level, lo=None, cost=None, sum_=None, disp=None,
                    stream=None) -> None:
    H, W = left.shape[-2], left.shape[-1]
    _check(load().mpv_debug_stage(ctx, _ptr(left), _ptr(right), W, H, left.stride(-2), view,
                                  level, _ptr(lo), _ptr(cost), _ptr(sum_), _ptr(disp),
                                  _stream(stream)), "mpv_debug_stage")


def mpv_level_info(ctx, width: int, height: int, level: int):
    w, h, r, d = C.c_int32(), C.c_int32(), C.c_int32(), C.c_int32()
    _check(load().mpv_level_info(ctx, width, height, level, C.byref(w), C.byref(h), C.byref(r),
                                 C.byref(d)), "mpv_level_info")
    return w.value, h.value, r.value, d.value


def mpv_profile_enable(ctx, on: bool) -> None:
    _check(load().mpv_profile_enable(ctx, int(bool(on))), "mpv_profile_enable")


def mpv_profile_read(ctx):
    """{stage: (milliseconds, launches)} accumulated since the previous read."""
    n = len(MPV_STAGES)
    ms = (C.c_double * n)()
    cnt = (C.c_int64 * n)()
    _check(load().mpv_profile_read(ctx, ms, cnt, n), "mpv_profile_read")
    return {MPV_STAGES[i]: (ms[i], cnt[i]) for i in range(n)}


def mpv_match_noalloc(params: mpv_params, left, right, disp, stream=None) -> None:
    """The matcher with all scratch in the library's fixed device array (no allocation);
    see include/mpv.h for its size limit and its sharing rules."""
    H, W = left.shape[-2], left.shape[-1]
    _check(load().mpv_match_noalloc(C.byref(params), _ptr(left), _ptr(right), W, H,
                                    left.stride(-2), _ptr(disp), disp.stride(-2),
                                    _stream(stream)), "mpv_match_noalloc")


def mpv_server_create(params: mpv_params, hbm_budget: int = 0, max_inflight: int = 8,
                      device: int = 0):
    h = C.c_void_p()
    _check(load().mpv_server_create(device, C.byref(params), hbm_budget, max_inflight,
                                    C.byref(h)), "mpv_server_create")
    return h


def mpv_server_set_proposal(server, weights_path) -> None:
    """Learned proposal for cameras whose range fits the network (None: pyramid only)."""
    _check(load().mpv_server_set_proposal(server, weights_path.encode() if weights_path else None),
           "mpv_server_set_proposal")


def mpv_server_add_camera(srv, camera: int, width: int, height: int, max_disparity: int):
    _check(load().mpv_server_add_camera(srv, camera, width, height, max_disparity),
           "mpv_server_add_camera")


def mpv_server_submit(srv, camera: int, left, right, disp, request_id: int):
    """left, right: uint8 numpy arrays (kept alive by the caller until completion);
    disp: uint16 numpy array receiving the map."""
    _check(load().mpv_server_submit(srv, camera, C.c_void_p(left.ctypes.data),
                                    C.c_void_p(right.ctypes.data), left.strides[0],
                                    C.c_void_p(disp.ctypes.data), disp.strides[0] // 2,
                                    request_id), "mpv_server_submit")


def mpv_server_poll(srv, max_completions: int = 64):
    out = (mpv_completion * max_completions)()
    n = C.c_int32()
    _check(load().mpv_server_poll(srv, out, max_completions, C.byref(n)), "mpv_server_poll")
    return [out[i] for i in range(n.value)]


def mpv_server_stats(srv):
    a, b, c, d, e = C.c_int32(), C.c_int32(), C.c_size_t(), C.c_uint64(), C.c_int32()
    _check(load().mpv_server_stats(srv, C.byref(a), C.byref(b), C.byref(c), C.byref(d),
                                   C.byref(e)), "mpv_server_stats")
    return dict(inflight=a.value, waiting=b.value, resident_bytes=c.value, evictions=d.value,
                peak_inflight=e.value)


def mpv_server_destroy(srv) -> None:
    load().mpv_server_destroy(srv)


def mpv_cnn_conv3x3(x, weight_bf16, bias, cout, relu, out_bf16=None, out_f32=None,
                    stream=None):
    """x: [N, Cin, H, W] bfloat16 or float32 CUDA tensor; weight [cout, Cin, 3, 3] bf16."""
    N, Cin, H, W = x.shape
    in_f32 = 1 if x.dtype.is_floating_point and x.element_size() == 4 else 0
    _check(load().mpv_cnn_conv3x3(_ptr(x), in_f32, N, Cin, H, W, _ptr(weight_bf16), _ptr(bias),
                                  cout, int(relu), _ptr(out_bf16), _ptr(out_f32),
                                  _stream(stream)), "mpv_cnn_conv3x3")


def mpv_cnn_conv3x3_wgrad(x_bf16, grad, dweight, dbias, stream=None):
    N, Cin, H, W = x_bf16.shape
    _check(load().mpv_cnn_conv3x3_wgrad(_ptr(x_bf16), N, Cin, _ptr(grad), grad.shape[1], H, W,
                                        _ptr(dweight), _ptr(dbias), _stream(stream)),
           "mpv_cnn_conv3x3_wgrad")


def mpv_cnn_flip_transpose(weight_bf16, out, stream=None):
    cout, cin = weight_bf16.shape[0], weight_bf16.shape[1]
    _check(load().mpv_cnn_flip_transpose(_ptr(weight_bf16), cout, cin, _ptr(out),
                                         _stream(stream)), "mpv_cnn_flip_transpose")


def mpv_cnn_relu_backward(grad, act_bf16, out, stream=None):
    _check(load().mpv_cnn_relu_backward(_ptr(grad), _ptr(act_bf16), _ptr(out), grad.numel(),
                                        _stream(stream)), "mpv_cnn_relu_backward")


def mpv_cnn_huber(pred, target, delta, grad, loss=None, stream=None):
    _check(load().mpv_cnn_huber(_ptr(pred), _ptr(target), float(delta), pred.numel(),
                                _ptr(grad), _ptr(loss), _stream(stream)), "mpv_cnn_huber")


def mpv_cnn_adam(weight, grad, m, v, lr, step, beta1=0.9, beta2=0.999, eps=1e-8,
                 weight_bf16=None, stream=None):
    _check(load().mpv_cnn_adam(_ptr(weight), _ptr(grad), _ptr(m), _ptr(v), weight.numel(),
                               float(lr), float(beta1), float(beta2), float(eps), int(step),
                               _ptr(weight_bf16), _stream(stream)), "mpv_cnn_adam")


def mpv_cnn_to_bf16(x, out, stream=None):
    _check(load().mpv_cnn_to_bf16(_ptr(x), _ptr(out), x.numel(), _stream(stream)),
           "mpv_cnn_to_bf16")


def mpv_cnn_target(disp, factor, max_disparity, target, stream=None):
    H, W = disp.shape[-2], disp.shape[-1]
    _check(load().mpv_cnn_target(_ptr(disp), disp.stride(-2), W, H, factor, max_disparity,
                                 _ptr(target), _stream(stream)), "mpv_cnn_target")


def mpv_proposal_predict(ctx, left, right, view, out, stream=None) -> None:
    """The learned proposal's top-level prediction (disparity / D) of one view, FP32."""
    H, W = left.shape[-2], left.shape[-1]
    _check(load().mpv_proposal_predict(ctx, _ptr(left), _ptr(right), W, H, left.stride(-2), view,
                                       _ptr(out), _stream(stream)), "mpv_proposal_predict")


def mpv_proposal_features(ctx, left, right, view, out, stream=None):
    H, W = left.shape[-2], left.shape[-1]
    _check(load().mpv_proposal_features(ctx, _ptr(left), _ptr(right), W, H, left.stride(-2),
                                        view, _ptr(out), _stream(stream)),
           "mpv_proposal_features")


def mpv_proposal_stats(ctx):
    """(edge hits, pixels) of the last learned-proposal match (after mpv_sync)."""
    a, b = C.c_uint64(), C.c_uint64()
    _check(load().mpv_proposal_stats(ctx, C.byref(a), C.byref(b)), "mpv_proposal_stats")
    return a.value, b.value



def mpv_batch_info(ctx):
    """(persistent, lanes, queues, cost_blocks, persistent_ms, streams_ms, occupancy) of
    the context's last batch."""
    v = [C.c_int32() for _ in range(4)] + [C.c_float() for _ in range(2)] + [C.c_int32()]
    _check(load().mpv_batch_info(ctx, *[C.byref(x) for x in v]), "mpv_batch_info")
    return tuple(x.value for x in v)


def mpv_set_batch_mode(ctx, mode: int) -> None:
    _check(load().mpv_set_batch_mode(ctx, int(mode)), "mpv_set_batch_mode")


def mpv_debug_batch_stall(ctx, wait_cycles: int) -> None:
    _check(load().mpv_debug_batch_stall(ctx, int(wait_cycles)), "mpv_debug_batch_stall")


def mpv_proposal_fallbacks(ctx):
    """(learned frames, frames that fell back) since the context's creation."""
    a, b = C.c_uint64(), C.c_uint64()
    _check(load().mpv_proposal_fallbacks(ctx, C.byref(a), C.byref(b)), "mpv_proposal_fallbacks")
    return a.value, b.value

def mpv_destroy(ctx) -> None:
    load().mpv_destroy(ctx)


class Matcher:
    """Owns one context; convenience wrapper over the functions above."""

    def __init__(self, device: int = 0, **params):
        self.ctx = mpv_create(device)
        self.set_params(**params)

    def set_params(self, **params):
        self.params = mpv_default_params(**params)
        mpv_set_params(self.ctx, self.params)

    def match(self, left, right, disp=None, stream=None):
        import torch
        if disp is None:
            disp = torch.empty(left.shape[-2:], dtype=torch.int16, device=left.device)
        mpv_match(self.ctx, left, right, disp, stream)
        return disp

    def sync(self):
        mpv_sync(self.ctx)

    def close(self):
        if self.ctx is not None:
            mpv_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
