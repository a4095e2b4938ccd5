"""The debug bounds build (libhc_debug.so, compiled with -DHC_DEBUG): every
bucket and slot index a kernel forms is checked against the table and every
key range against its call; a violation sets error bit 4 of the table header
instead of faulting.  The parity scripts run on that build in a child process
(HC_LIBRARY selects it) and must pass with the bit clear: their check() reads
it after every comparison with the oracle."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.slow
def test_parity_scripts_on_the_debug_bounds_build():
    from paper_1908_05936_gb300 import build
    lib = build.build_debug()
    env = dict(os.environ, HC_LIBRARY=lib)
    cmd = [sys.executable, "-m", "pytest", "tests/test_gpu_parity.py", "tests/test_gpu_batch.py",
           "tests/test_gpu_device_api.py", "-m", "gpu", "-q", "-x", "-p", "no:cacheprovider",
           "-k", "random_scripts or batch_sizes or overflow or rehash or streaming or batch or tombstone or device"]
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=1500)
    tail = (r.stdout + r.stderr)[-4000:]
    assert r.returncode == 0, tail
    assert " passed" in tail
    # the child really ran the debug build
    probe = subprocess.run([sys.executable, "-c", "from paper_1908_05936_gb300 import _lib as L; print(L.LIB_PATH)"],
                           cwd=ROOT, env=env, capture_output=True, text=True, timeout=120)
    assert probe.stdout.strip() == lib
