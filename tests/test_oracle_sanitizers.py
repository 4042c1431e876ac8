"""The CPU oracle under AddressSanitizer and UndefinedBehaviorSanitizer.

compute-sanitizer is not available for the GPU side here; the host C code of the oracle
is checked instead: tests/oracle_sanitize_main.c drives its entry points on small,
ragged and degenerate cases (one and three scales, both merges, the gradient table,
tiles, per-level windows, N = 3 and 5, both maps of the left-right check, the stage dump,
the road functions), built with -fsanitize=address,undefined and no recovery, so that an
out-of-bounds access, a leak, a signed overflow or a misaligned load fails the run.
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_oracle_clean_under_asan_and_ubsan(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    exe = str(tmp_path / "oracle_sanitized")
    cmd = [cc, "-std=c11", "-O1", "-g", "-fsanitize=address,undefined",
           "-fno-sanitize-recover=all", "-fno-omit-frame-pointer",
           os.path.join(ROOT, "oracle", "mpv_oracle.c"),
           os.path.join(ROOT, "tests", "oracle_sanitize_main.c"), "-lm", "-o", exe]
    build = subprocess.run(cmd, capture_output=True, text=True)
    if build.returncode != 0 and "sanitize" in build.stderr:
        pytest.skip("the compiler has no sanitizer runtimes: " + build.stderr[-200:])
    assert build.returncode == 0, build.stderr[-2000:]
    env = dict(os.environ, ASAN_OPTIONS="detect_leaks=1:abort_on_error=0",
               UBSAN_OPTIONS="print_stacktrace=1")
    run = subprocess.run([exe], capture_output=True, text=True, env=env, timeout=300)
    assert run.returncode == 0, run.stdout[-2000:] + run.stderr[-4000:]
    assert "runtime error" not in run.stderr and "ERROR: AddressSanitizer" not in run.stderr
    assert run.stdout.count(": ok") == 11, run.stdout
