"""The host code of the C ABI under AddressSanitizer and UndefinedBehaviorSanitizer (the build
variant `sanitize`): a child process with the sanitizer runtime preloaded drives every entry point
with NULL arguments and several hundred edge-valued and random configurations
(tests/abi_host_paths.py); any invalid access or undefined behaviour aborts it.  Needs no GPU."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _libasan():
    try:
        path = subprocess.run(["gcc", "-print-file-name=libasan.so"], capture_output=True, text=True,
                              check=True).stdout.strip()
    except (OSError, subprocess.CalledProcessError):
        return None
    return path if os.path.isabs(path) and os.path.exists(path) else None


def test_abi_host_paths_under_address_and_ub_sanitizers():
    asan = _libasan()
    if asan is None:
        pytest.skip("the compiler's AddressSanitizer runtime is not installed")
    from paper_1912_10596_gb300 import build
    build.build(variant="sanitize")
    env = dict(os.environ, LD_PRELOAD=asan, XFLAT_VARIANT="sanitize",
               ASAN_OPTIONS="detect_leaks=0:protect_shadow_gap=0:abort_on_error=0:exitcode=97",
               UBSAN_OPTIONS="print_stacktrace=1:halt_on_error=1:exitcode=98")
    res = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "abi_host_paths.py")], cwd=ROOT,
                         env=env, capture_output=True, text=True, timeout=900)
    report = res.stdout[-2000:] + res.stderr[-4000:]
    assert res.returncode == 0, report
    assert "host paths ok" in res.stdout, report
    assert "AddressSanitizer" not in res.stderr and "runtime error" not in res.stderr, report
