"""ctypes front end of the CPU oracle (oracle/mpv_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by the test suite, by the smoke check in
__graft_entry__ and by the benchmark's CPU-baseline leg.  The matcher's product path
never imports this module.  Every function wraps one C routine of the oracle and
returns numpy arrays; see the C file for the passage of the paper each one follows.
"""
import ctypes as C
import os

import numpy as np

from . import build_oracle

NO_TRUNC = 0x7FFFFFFF
INVALID = 0xFFFF
MERGE_SUM = 0
MERGE_PAPER = 1

_lib = None


class OraParams(C.Structure):
    _fields_ = [
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
        ("grad_lut", C.POINTER(C.c_int32)),
        ("top_block", C.c_int32),
        ("windows", C.c_int32 * 4),
    ]


class OraPenalty(C.Structure):
    _fields_ = [("p_up", C.c_int64), ("p_dn", C.c_int64), ("T_up", C.c_int64),
                ("T_dn", C.c_int64)]


def _lut(grad_lut):
    if grad_lut is None:
        return None, None
    a = np.ascontiguousarray(grad_lut, dtype=np.int32)
    assert a.shape == (256,)
    return a, a.ctypes.data_as(C.POINTER(C.c_int32))


def params(max_disparity=32, num_scales=1, num_paths=4, p1=10, trunc=30, ssim_window=5,
           window=0, block=(0, 0, 0, 0), lr_check=1, lr_tol=1, merge_mode=MERGE_SUM,
           grad_lut=None, top_block=0, windows=(0, 0, 0, 0)):
    p = OraParams()
    p.max_disparity = max_disparity
    p.num_scales = num_scales
    p.num_paths = num_paths
    p.p1 = p1
    p.trunc = trunc
    p.ssim_window = ssim_window
    p.window = window
    blk = list(block) + [0] * (4 - len(block))
    for i in range(4):
        p.block[i] = blk[i]
    p.lr_check = lr_check
    p.lr_tol = lr_tol
    p.merge_mode = merge_mode
    p.top_block = top_block
    win = list(windows) + [0] * (4 - len(windows))
    for i in range(4):
        p.windows[i] = win[i]
    p._lut_keep, ptr = _lut(grad_lut)   # the table must outlive the struct's pointer
    if ptr is not None:
        p.grad_lut = ptr
    return p


def lib():
    global _lib
    if _lib is None:
        path = build_oracle.build()
        L = C.CDLL(path)
        u8p = C.POINTER(C.c_uint8)
        i32p = C.POINTER(C.c_int32)
        i64p = C.POINTER(C.c_int64)
        u16p = C.POINTER(C.c_uint16)
        pp = C.POINTER(OraParams)
        i = C.c_int
        L.ora_c1.argtypes = [i]; L.ora_c1.restype = C.c_int64
        L.ora_c2.argtypes = [i]; L.ora_c2.restype = C.c_int64
        L.ora_ssim_cost.argtypes = [u8p, u8p, i, i, i, i, i, i, i]
        L.ora_ssim_cost.restype = C.c_int32
        L.ora_cost_volume.argtypes = [u8p, u8p, i, i, i, i, i32p, i, i32p]
        L.ora_cost_volume.restype = None
        for f in (L.ora_envelope_naive, L.ora_envelope_fast):
            f.argtypes = [i64p, i, i, i, C.c_int64, C.c_int64, i64p]
            f.restype = None
        L.ora_path.argtypes = [i32p, i32p, i, i, i, i, i, C.c_int64, C.c_int64, i, i, i, i64p]
        L.ora_path.restype = i
        L.ora_aggregate.argtypes = [i32p, i32p, i, i, i, i, C.c_int64, C.c_int64, i, i64p]
        L.ora_aggregate.restype = i
        penp = C.POINTER(OraPenalty)
        for f in (L.ora_envelope_naive_pen, L.ora_envelope_fast_pen):
            f.argtypes = [i64p, i, i, i, penp, i64p]
            f.restype = None
        L.ora_path_pen.argtypes = [i64p, i32p, i, i, i, i, i, C.c_int64, C.c_int64, i32p, u8p,
                                   i, i, i, i, i, i64p]
        L.ora_path_pen.restype = i
        for f in (L.ora_aggregate_grad, L.ora_aggregate_paper):
            f.argtypes = [i32p, i32p, i, i, i, i, C.c_int64, C.c_int64, i32p, u8p, i, i64p]
            f.restype = i
        L.ora_aggregate_blocks.argtypes = [i32p, i32p, i, i, i, i, C.c_int64, C.c_int64, i32p,
                                           u8p, i, i, i, i64p]
        L.ora_aggregate_blocks.restype = i
        u32p = C.POINTER(C.c_uint32)
        for f in (L.ora_vdisparity, L.ora_udisparity):
            f.argtypes = [u16p, i, i, i, i, u32p]
            f.restype = None
        L.ora_road_profile.argtypes = [u32p, i, i, i, i32p]
        L.ora_road_profile.restype = C.c_int64
        L.ora_wta.argtypes = [i64p, i32p, i, i, i, u16p]
        L.ora_wta.restype = None
        L.ora_downsample2.argtypes = [u8p, i, i, i, u8p, i]
        L.ora_downsample2.restype = None
        L.ora_seed.argtypes = [u16p, i, i, i, i, i, i, i, i32p]
        L.ora_seed.restype = None
        L.ora_level_dims.argtypes = [i, i, i, i, C.POINTER(i), C.POINTER(i)]
        L.ora_level_dims.restype = None
        L.ora_level_range.argtypes = [i, i, i]
        L.ora_level_range.restype = i
        L.ora_level_window.argtypes = [pp, i]
        L.ora_level_window.restype = i
        L.ora_node_count.argtypes = [i, i, pp]
        L.ora_node_count.restype = C.c_int64
        L.ora_check_params.argtypes = [i, i, pp]
        L.ora_check_params.restype = i
        L.ora_match_view.argtypes = [u8p, u8p, i, i, i, pp, u16p]
        L.ora_match_view.restype = i
        L.ora_match.argtypes = [u8p, u8p, i, i, i, pp, u16p, u16p]
        L.ora_match.restype = i
        L.ora_lr_check.argtypes = [u16p, u16p, i, i, i, u16p]
        L.ora_lr_check.restype = None
        L.ora_view_stage.argtypes = [u8p, u8p, i, i, i, pp, i, i32p, i32p, i64p, u16p]
        L.ora_view_stage.restype = i
        _lib = L
    return _lib


def _p(a, ctype):
    return a.ctypes.data_as(C.POINTER(ctype))


def _img(a):
    a = np.ascontiguousarray(a, dtype=np.uint8)
    assert a.ndim == 2
    return a


def c1(N):
    return lib().ora_c1(N)


def c2(N):
    return lib().ora_c2(N)


def ssim_cost(I0, I1, N, x, y, u):
    I0, I1 = _img(I0), _img(I1)
    H, W = I0.shape
    return lib().ora_ssim_cost(_p(I0, C.c_uint8), _p(I1, C.c_uint8), W, H, W, N, x, y, u)


def cost_volume(I0, I1, N, Dw, lo=None):
    I0, I1 = _img(I0), _img(I1)
    H, W = I0.shape
    out = np.zeros((H, W, Dw), np.int32)
    lop = None
    if lo is not None:
        lo = np.ascontiguousarray(lo, dtype=np.int32)
        lop = _p(lo, C.c_int32)
    lib().ora_cost_volume(_p(I0, C.c_uint8), _p(I1, C.c_uint8), W, H, W, N, lop, Dw,
                          _p(out, C.c_int32))
    return out


def envelope(A, lo_prev, lo, p1, T, naive=False):
    A = np.ascontiguousarray(A, dtype=np.int64)
    M = np.zeros(A.shape[0], np.int64)
    f = lib().ora_envelope_naive if naive else lib().ora_envelope_fast
    f(_p(A, C.c_int64), lo_prev, lo, A.shape[0], p1, T, _p(M, C.c_int64))
    return M


def path(Cv, dx, dy, p1, T, lo=None, normalized=True, naive=False, check=False):
    Cv = np.ascontiguousarray(Cv, dtype=np.int32)
    H, W, Dw = Cv.shape
    L = np.zeros((H, W, Dw), np.int64)
    lop = None
    if lo is not None:
        lo = np.ascontiguousarray(lo, dtype=np.int32)
        lop = _p(lo, C.c_int32)
    st = lib().ora_path(_p(Cv, C.c_int32), lop, W, H, Dw, dx, dy, p1, T, int(normalized),
                        int(naive), int(check), _p(L, C.c_int64))
    return L, st


def aggregate(Cv, num_paths, p1, T, lo=None, normalized=True):
    Cv = np.ascontiguousarray(Cv, dtype=np.int32)
    H, W, Dw = Cv.shape
    S = np.zeros((H, W, Dw), np.int64)
    lop = None
    if lo is not None:
        lo = np.ascontiguousarray(lo, dtype=np.int32)
        lop = _p(lo, C.c_int32)
    st = lib().ora_aggregate(_p(Cv, C.c_int32), lop, W, H, Dw, num_paths, p1, T,
                             int(normalized), _p(S, C.c_int64))
    assert st == 0
    return S


def envelope_pen(A, lo_prev, lo, p_up, p_dn, T_up, T_dn, naive=False):
    A = np.ascontiguousarray(A, dtype=np.int64)
    M = np.zeros(A.shape[0], np.int64)
    e = OraPenalty(p_up, p_dn, T_up, T_dn)
    f = lib().ora_envelope_naive_pen if naive else lib().ora_envelope_fast_pen
    f(_p(A, C.c_int64), lo_prev, lo, A.shape[0], C.byref(e), _p(M, C.c_int64))
    return M


def _opt_lo(lo):
    if lo is None:
        return None, None
    lo = np.ascontiguousarray(lo, dtype=np.int32)
    return lo, _p(lo, C.c_int32)


def _opt_img(I0, grad_lut):
    if grad_lut is None:
        return None, None
    I0 = _img(I0)
    return I0, _p(I0, C.c_uint8)


def path_pen(Q, dx, dy, p1, T, lo=None, grad_lut=None, I0=None, double_up=False,
             normalize_out=False, naive=False, check=False):
    """One pass over an int64 data term with per-step penalties (ora_path_pen)."""
    Q = np.ascontiguousarray(Q, dtype=np.int64)
    H, W, Dw = Q.shape
    L = np.zeros((H, W, Dw), np.int64)
    lo, lop = _opt_lo(lo)
    lut, lutp = _lut(grad_lut)
    img, imgp = _opt_img(I0, grad_lut)
    st = lib().ora_path_pen(_p(Q, C.c_int64), lop, W, H, Dw, dx, dy, p1, T, lutp, imgp, W,
                            int(double_up), int(normalize_out), int(naive), int(check),
                            _p(L, C.c_int64))
    return L, st


def _aggregate_pen(fn, Cv, num_paths, p1, T, lo, grad_lut, I0):
    Cv = np.ascontiguousarray(Cv, dtype=np.int32)
    H, W, Dw = Cv.shape
    S = np.zeros((H, W, Dw), np.int64)
    lo, lop = _opt_lo(lo)
    lut, lutp = _lut(grad_lut)
    img, imgp = _opt_img(I0, grad_lut)
    st = fn(_p(Cv, C.c_int32), lop, W, H, Dw, num_paths, p1, T, lutp, imgp, W,
            _p(S, C.c_int64))
    assert st == 0
    return S


def aggregate_grad(Cv, num_paths, p1, T, lo=None, grad_lut=None, I0=None):
    """Sum of bounded passes with gradient-weighted slopes (ora_aggregate_grad)."""
    return _aggregate_pen(lib().ora_aggregate_grad, Cv, num_paths, p1, T, lo, grad_lut, I0)


def aggregate_blocks(Cv, num_paths, p1, T, block, merge_mode=MERGE_SUM, lo=None,
                     grad_lut=None, I0=None):
    """Aggregation with the image split into independent block x block tiles."""
    Cv = np.ascontiguousarray(Cv, dtype=np.int32)
    H, W, Dw = Cv.shape
    S = np.zeros((H, W, Dw), np.int64)
    lo, lop = _opt_lo(lo)
    lut, lutp = _lut(grad_lut)
    img, imgp = _opt_img(I0, grad_lut)
    st = lib().ora_aggregate_blocks(_p(Cv, C.c_int32), lop, W, H, Dw, num_paths, p1, T, lutp,
                                    imgp, W, merge_mode, block, _p(S, C.c_int64))
    assert st == 0
    return S


def aggregate_paper(Cv, num_paths, p1, T, lo=None, grad_lut=None, I0=None):
    """The paper's layered merge (ora_aggregate_paper)."""
    return _aggregate_pen(lib().ora_aggregate_paper, Cv, num_paths, p1, T, lo, grad_lut, I0)


def wta(S, lo=None):
    S = np.ascontiguousarray(S, dtype=np.int64)
    H, W, Dw = S.shape
    d = np.zeros((H, W), np.uint16)
    lop = None
    if lo is not None:
        lo = np.ascontiguousarray(lo, dtype=np.int32)
        lop = _p(lo, C.c_int32)
    lib().ora_wta(_p(S, C.c_int64), lop, W, H, Dw, _p(d, C.c_uint16))
    return d


def downsample2(img):
    img = _img(img)
    H, W = img.shape
    out = np.zeros(((H + 1) // 2, (W + 1) // 2), np.uint8)
    lib().ora_downsample2(_p(img, C.c_uint8), W, H, W, _p(out, C.c_uint8), out.shape[1])
    return out


def seed(dprev, W, H, block, Dw, Dl):
    dprev = np.ascontiguousarray(dprev, dtype=np.uint16)
    Hp, Wp = dprev.shape
    lo = np.zeros((H, W), np.int32)
    lib().ora_seed(_p(dprev, C.c_uint16), Wp, Hp, W, H, block, Dw, Dl, _p(lo, C.c_int32))
    return lo


def level_dims(W, H, S, l):
    a, b = C.c_int(), C.c_int()
    lib().ora_level_dims(W, H, S, l, C.byref(a), C.byref(b))
    return a.value, b.value


def level_range(D, S, l):
    return lib().ora_level_range(D, S, l)


def level_window(p, l):
    return lib().ora_level_window(C.byref(p), l)


def node_count(W, H, p):
    return lib().ora_node_count(W, H, C.byref(p))


def check_params(W, H, p):
    return lib().ora_check_params(W, H, C.byref(p))


def match_view(I0, I1, p):
    I0, I1 = _img(I0), _img(I1)
    H, W = I0.shape
    d = np.zeros((H, W), np.uint16)
    st = lib().ora_match_view(_p(I0, C.c_uint8), _p(I1, C.c_uint8), W, H, W, C.byref(p),
                              _p(d, C.c_uint16))
    if st != 0:
        raise ValueError(f"oracle match_view failed: {st}")
    return d


def match(I0, I1, p, want_right=False):
    I0, I1 = _img(I0), _img(I1)
    H, W = I0.shape
    dL = np.zeros((H, W), np.uint16)
    dR = np.zeros((H, W), np.uint16) if want_right else None
    st = lib().ora_match(_p(I0, C.c_uint8), _p(I1, C.c_uint8), W, H, W, C.byref(p),
                         _p(dL, C.c_uint16), _p(dR, C.c_uint16) if want_right else None)
    if st != 0:
        raise ValueError(f"oracle match failed: {st}")
    return (dL, dR) if want_right else dL


def lr_check(dL, dR, tol):
    dL = np.ascontiguousarray(dL, dtype=np.uint16)
    dR = np.ascontiguousarray(dR, dtype=np.uint16)
    H, W = dL.shape
    out = np.zeros((H, W), np.uint16)
    lib().ora_lr_check(_p(dL, C.c_uint16), _p(dR, C.c_uint16), W, H, tol, _p(out, C.c_uint16))
    return out


def view_stage(I0, I1, p, level):
    """lo, cost volume, summed volume and WTA map of one pyramid level of one view."""
    I0, I1 = _img(I0), _img(I1)
    H, W = I0.shape
    Wl, Hl = level_dims(W, H, p.num_scales, level)
    Dw = level_window(p, level)
    lo = np.zeros((Hl, Wl), np.int32)
    Cv = np.zeros((Hl, Wl, Dw), np.int32)
    S = np.zeros((Hl, Wl, Dw), np.int64)
    d = np.zeros((Hl, Wl), np.uint16)
    st = lib().ora_view_stage(_p(I0, C.c_uint8), _p(I1, C.c_uint8), W, H, W, C.byref(p), level,
                              _p(lo, C.c_int32), _p(Cv, C.c_int32), _p(S, C.c_int64),
                              _p(d, C.c_uint16))
    if st != 0:
        raise ValueError(f"oracle view_stage failed: {st}")
    return lo, Cv, S, d


def vdisparity(U, D):
    """Row histograms over the disparities (ora_vdisparity): [H][D] uint32."""
    U = np.ascontiguousarray(U, dtype=np.uint16)
    H, W = U.shape
    out = np.zeros((H, D), np.uint32)
    lib().ora_vdisparity(_p(U, C.c_uint16), W, H, W, D, _p(out, C.c_uint32))
    return out


def udisparity(U, D):
    """Column histograms over the disparities (ora_udisparity): [W][D] uint32."""
    U = np.ascontiguousarray(U, dtype=np.uint16)
    H, W = U.shape
    out = np.zeros((W, D), np.uint32)
    lib().ora_udisparity(_p(U, C.c_uint16), W, H, W, D, _p(out, C.c_uint32))
    return out


def road_profile(Hx, eta):
    """(best sum, rows P[i] per disparity) of the road Viterbi (ora_road_profile)."""
    Hx = np.ascontiguousarray(Hx, dtype=np.uint32)
    H, D = Hx.shape
    P = np.zeros(D, np.int32)
    best = lib().ora_road_profile(_p(Hx, C.c_uint32), H, D, eta, _p(P, C.c_int32))
    return best, P
