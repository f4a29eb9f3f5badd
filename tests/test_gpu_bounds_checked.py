"""The GPU tests again under the bounds-checked build (libflood_checked.so).

The checked build (-DFLOOD_BOUNDS_CHECK) tests every data-dependent index of
the kernels before use: cell and bucket ids, record, group and point ranges,
bulk-copy sources and destinations, output rows. An index out of range skips
the access and comes back as FLOOD_EINTERNAL instead of reading or writing
out of range. This runs the parity, random-set, persistence, general-landmark,
asynchronous-boundary and serving tests in a child process that loads the
checked library (FLOOD_LIBRARY=checked): every call must still succeed and
give the same results, i.e. no index of those workloads is out of range.
"""
import os
import subprocess
import sys

import pytest

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SUBSET = ["tests/test_gpu_parity.py", "tests/test_gpu_given.py", "tests/test_gpu_persistence.py",
          "tests/test_gpu_general_landmarks.py", "tests/test_gpu_async.py", "tests/test_serve.py",
          "tests/test_gpu_wait_timeout.py", "tests/test_gpu_nd.py"]


def test_gpu_suite_under_the_bounds_checked_library():
    from paper_2509_22432_b300 import build
    build.build(checked=True)
    env = dict(os.environ, FLOOD_LIBRARY="checked")
    probe = subprocess.run([sys.executable, "-c", "from paper_2509_22432_b300 import _lib; "
                            "print(_lib.get()._name)"], cwd=ROOT, env=env, capture_output=True, text=True)
    assert probe.returncode == 0 and probe.stdout.strip().endswith("libflood_checked.so"), probe.stderr
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-m", "gpu and not slow", *SUBSET], cwd=ROOT,
                       env=env, capture_output=True, text=True, timeout=1500)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-2000:]
    assert " passed" in r.stdout
