"""The checking builds on the GPU.  The bounds-checked library (every plane, stage-plane, table and
piece access of the step kernel's pass body tested against its allocation) and the host-sanitizer
library (AddressSanitizer and UndefinedBehaviorSanitizer over the C ABI's host code, the CUDA
runtime underneath) each run the small cases of tests/checked_cases.py in a child process: every
call must succeed (a bounds violation would be reported as XFLAT_ERR_CUDA with its site, a
sanitizer finding would abort the child) and give the plain library's results."""
import os
import subprocess
import sys

import numpy as np
import pytest

from checked_cases import run_cases

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def plain_results(xf):
    return run_cases(xf)


def _child(variant, out, extra_env):
    env = dict(os.environ, XFLAT_VARIANT=variant, **extra_env)
    res = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "checked_cases.py"), out], cwd=ROOT, env=env,
                         capture_output=True, text=True, timeout=1200)
    report = res.stdout[-2000:] + res.stderr[-4000:]
    assert res.returncode == 0, report
    assert "cases ok" in res.stdout and f"libxflat_{variant}.so" in res.stdout, report
    return res


def _compare(plain, out, exact):
    """exact: the child ran the plain build's device code (bit-identical results).  Otherwise the
    checked kernels' extra branches may let the compiler contract a different multiply-add pair
    into an FMA: FP64 results then differ in the last bits, FP32 (mixed) ones by a few ulps per
    step, which an adaptive controller may turn into another step count."""
    got = np.load(out)
    assert sorted(got.files) == sorted(plain)
    for k in plain:
        a, b = got[k], plain[k]
        assert a.shape == b.shape, k
        mixed = k.startswith("mixed_")
        if exact:
            assert np.array_equal(a, b), k
        elif k.endswith("/steps"):
            assert mixed or np.array_equal(a, b), k
        else:
            tol = 1e-4 if mixed else 1e-12
            assert np.abs(a - b).max() <= tol * max(1.0, np.abs(b).max()), (k, np.abs(a - b).max())


def test_bounds_checked_build_runs_every_kernel_family_clean(plain_results, tmp_path):
    from paper_1912_10596_gb300 import build
    build.build(variant="bounds")
    out = str(tmp_path / "bounds.npz")
    _child("bounds", out, {})
    _compare(plain_results, out, exact=False)


def test_host_sanitizer_build_runs_every_kernel_family_clean(plain_results, tmp_path):
    asan = subprocess.run(["gcc", "-print-file-name=libasan.so"], capture_output=True, text=True).stdout.strip()
    if not (os.path.isabs(asan) and os.path.exists(asan)):
        pytest.skip("the compiler's AddressSanitizer runtime is not installed")
    from paper_1912_10596_gb300 import build
    build.build(variant="sanitize")
    out = str(tmp_path / "sanitize.npz")
    res = _child("sanitize", out, {"LD_PRELOAD": asan,
                                   "ASAN_OPTIONS": "detect_leaks=0:protect_shadow_gap=0:replace_intrin=0:exitcode=97",
                                   "UBSAN_OPTIONS": "print_stacktrace=1:halt_on_error=1:exitcode=98"})
    assert "AddressSanitizer" not in res.stderr and "runtime error" not in res.stderr, res.stderr[-4000:]
    _compare(plain_results, out, exact=True)
