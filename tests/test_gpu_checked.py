"""The bounds-checked build (nvcc -DXS_CHECKED) on the GPU.

A subset of the GPU tests runs in a child process on libxs_checked.so: the line
sums (every wing form, the near kernels' polynomial and series zones, ragged and
empty inputs) and their adjoints, the optical-depth and emission kernels, MODIT,
the weak-line pre-filter, the response operators and the Gaussian-process prior.
After each of the child's tests the autouse fixture in conftest.py asserts that
no index check failed in any translation unit."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SUBSET = ["tests/test_gpu_xs.py", "tests/test_gpu_rt.py", "tests/test_gpu_modit.py", "tests/test_gpu_filter.py",
          "tests/test_gpu_response.py", "tests/test_gpu_prior.py"]


@pytest.mark.gpu
def test_gpu_subset_on_the_checked_build():
    if os.environ.get("XS_CHECKED") == "1":
        pytest.skip("this process already runs on the checked build")
    env = dict(os.environ, XS_CHECKED="1")
    p = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-m", "gpu", "-p", "no:cacheprovider"] + SUBSET,
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=1800)
    assert p.returncode == 0, p.stdout[-4000:] + p.stderr[-2000:]
    assert " passed" in p.stdout and "failed" not in p.stdout
