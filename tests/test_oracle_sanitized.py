"""The oracle under AddressSanitizer and UndefinedBehaviorSanitizer: every entry point runs
on small seeded inputs (tests/oracle_sanitize_driver.c) in a build with both sanitizers, and
neither reports anything (out-of-bounds reads or writes, leaks, signed overflow, ...)."""
import os
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_oracle_clean_under_asan_and_ubsan():
    if subprocess.run(["which", "gcc"], capture_output=True).returncode != 0:
        pytest.skip("no gcc")
    with tempfile.TemporaryDirectory() as tmp:
        exe = os.path.join(tmp, "oracle_sanitized")
        cmd = ["gcc", "-std=c11", "-O1", "-g", "-fopenmp", "-ffp-contract=off",
               "-fsanitize=address,undefined", "-fno-sanitize-recover=undefined",
               "-fno-omit-frame-pointer", "-o", exe,
               os.path.join(ROOT, "tests", "oracle_sanitize_driver.c"),
               os.path.join(ROOT, "oracle", "nssg_oracle.c"), "-lm"]
        build = subprocess.run(cmd, capture_output=True, text=True)
        if build.returncode != 0 and "sanitize" in build.stderr:
            pytest.skip("sanitizer runtime not available: " + build.stderr[:200])
        assert build.returncode == 0, build.stderr
        env = dict(os.environ, OMP_NUM_THREADS="4",
                   ASAN_OPTIONS="detect_leaks=1:abort_on_error=0",
                   UBSAN_OPTIONS="print_stacktrace=1")
        run = subprocess.run([exe], capture_output=True, text=True, env=env, timeout=300)
        assert run.returncode == 0, run.stderr[-3000:]
        assert "runtime error" not in run.stderr and "AddressSanitizer" not in run.stderr
        assert "oracle sanitized run ok" in run.stdout
