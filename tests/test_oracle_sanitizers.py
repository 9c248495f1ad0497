"""The C oracle under AddressSanitizer and UndefinedBehaviorSanitizer: a
driver (tests/oracle_driver.c) runs both precisions over many small
problems, including clipped PSFs, flux triggers, replay, an overfull
component list and bad arguments; any out-of-bounds access, use of freed
memory, overflow or other undefined behaviour fails the test."""
import os
import shutil
import subprocess
import tempfile

import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))


def test_oracle_clean_under_sanitizers():
    cc = os.environ.get("CC", "gcc")
    if not shutil.which(cc):
        pytest.skip("no C compiler")
    src = os.path.join(os.path.dirname(os.path.abspath(oracle.__file__)), "clean_oracle.c")
    with tempfile.TemporaryDirectory() as d:
        exe = os.path.join(d, "driver")
        flags = [f for f in oracle.CFLAGS if f not in ("-shared", "-fPIC")]
        r = subprocess.run([cc, *flags, "-g", "-fsanitize=address,undefined",
                            "-fno-sanitize-recover=all", "-o", exe,
                            os.path.join(HERE, "oracle_driver.c"), src],
                           capture_output=True, text=True)
        if r.returncode != 0 and "sanitize" in r.stderr:
            pytest.skip("sanitizer runtime unavailable")
        assert r.returncode == 0, r.stderr
        env = dict(os.environ, ASAN_OPTIONS="detect_leaks=1", UBSAN_OPTIONS="print_stacktrace=1")
        run = subprocess.run([exe], capture_output=True, text=True, env=env, timeout=300)
        assert run.returncode == 0, run.stderr[-4000:]
