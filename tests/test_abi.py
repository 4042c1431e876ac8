"""The C-ABI library loads and exports every symbol include/mpv.h declares (no GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "mpv.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mpv_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2001_09678_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_every_declared_symbol_is_exported(lib):
    names = declared_symbols()
    assert "mpv_match" in names and "mpv_match_batch" in names and len(names) >= 10
    for n in names:
        assert hasattr(lib, n), n


def test_binding_declares_every_header_symbol():
    from paper_2001_09678_gb300 import mpv
    assert sorted(mpv.EXPORTS) == declared_symbols()


def test_status_strings_and_null_safety(lib):
    from paper_2001_09678_gb300 import mpv
    mpv.load()
    assert mpv.mpv_status_string(0) == "ok"
    assert mpv.mpv_status_string(1) == "invalid argument"
    assert mpv.mpv_status_string(99) == "unknown status"
    mpv.load().mpv_destroy(None)          # NULL-safe
    L = mpv.load()
    assert L.mpv_set_params(None, None) == mpv.MPV_ERR_INVALID_ARG
    assert L.mpv_match(None, None, None, 8, 8, 8, None, 8, None) == mpv.MPV_ERR_INVALID_ARG
    assert L.mpv_sync(None) == mpv.MPV_ERR_INVALID_ARG


def test_default_params_match_header_defaults(lib):
    from paper_2001_09678_gb300 import mpv
    p = mpv.mpv_default_params()
    assert p.struct_size == ctypes.sizeof(mpv.mpv_params)
    assert (p.max_disparity, p.num_scales, p.num_paths, p.p1, p.trunc, p.ssim_window) == \
        (128, 3, 8, 10, 30, 5)
    assert (p.lr_check, p.lr_tol, p.window) == (1, 1, 0)
