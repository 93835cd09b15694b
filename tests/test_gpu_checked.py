"""The bounds-checked build (libcollage_checked.so, -DCOLLAGE_CHECKED) against the whole GPU suite.

In that build every guarded index of the hot kernels is tested before its access; a failed test
latches the status bit for an internal error and skips the access, and the next call that reads
the status word returns COLLAGE_ERR_STATE (the binding raises).  The GPU suite is run again in a
child process with COLLAGE_CHECKED=1, so every case of it doubles as a check that no index of the
kernels strays past its bound."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_checked_build_is_the_one_loaded():
    code = ("from paper_2406_04008_gb300 import build, _lib; build.build(); "
            "print(_lib.load()._name)")
    out = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True,
                         env=dict(os.environ, COLLAGE_CHECKED="1"), timeout=600)
    assert out.returncode == 0, out.stderr
    assert out.stdout.strip().endswith("libcollage_checked.so"), out.stdout


def test_gpu_suite_passes_on_the_checked_build():
    cmd = [sys.executable, "-m", "pytest", "tests", "-m", "gpu", "-q", "-x", "-p", "no:cacheprovider",
           "--ignore=tests/test_gpu_checked.py"]
    out = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True,
                         env=dict(os.environ, COLLAGE_CHECKED="1"), timeout=1800)
    assert out.returncode == 0, out.stdout[-4000:] + out.stderr[-2000:]
