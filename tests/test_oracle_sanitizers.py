"""The FP64 oracle under AddressSanitizer and UndefinedBehaviorSanitizer: a
small tensile bar for every damage model through plastic flow, damage and
failure (tests/oracle_sanitize_driver.c, compiled with the oracle as one
translation unit).  Skipped where the compiler cannot build sanitized code."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def test_oracle_is_clean_under_asan_and_ubsan(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    exe = str(tmp_path / "oracle_asan")
    src = os.path.join(HERE, "oracle_sanitize_driver.c")
    build = subprocess.run([cc, "-O1", "-g", "-std=gnu11", "-ffp-contract=off", "-fno-omit-frame-pointer",
                            "-fsanitize=address,undefined", "-fno-sanitize-recover=all", src, "-o", exe, "-lm"],
                           capture_output=True, text=True)
    if build.returncode != 0:
        pytest.skip("sanitized build unavailable: " + build.stderr.strip()[-200:])
    env = dict(os.environ, ASAN_OPTIONS="detect_leaks=1", UBSAN_OPTIONS="print_stacktrace=1")
    run = subprocess.run([exe], capture_output=True, text=True, env=env, timeout=600)
    assert run.returncode == 0, run.stdout + run.stderr
    assert "runtime error" not in run.stderr and "AddressSanitizer" not in run.stderr, run.stderr
    assert run.stdout.count("damage") == 4, run.stdout
