"""The kernels' index checks: a build with -DEMG_BOUNDS_CHECK runs the parity
and batching suites, and every test must leave the error word clear (the
autouse fixture in conftest.py asserts it).  A check that must fail shows the
word records it and the access is skipped."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(args, env, timeout):
    return subprocess.run([sys.executable, *args], cwd=ROOT, env=env, capture_output=True, text=True,
                          timeout=timeout)


def test_suites_pass_with_the_index_checks():
    env = dict(os.environ, EMG_BUILD_VARIANT="boundscheck")
    b = _run(["-c", "import paper_2511_01793_gb300 as emg; print(emg.build())"], env, 900)
    assert b.returncode == 0, b.stdout[-3000:] + b.stderr[-3000:]
    probe = _run(["-c", "import paper_2511_01793_gb300 as emg; print(emg.emg_debug_bounds_selftest())"], env, 300)
    assert probe.returncode == 0 and probe.stdout.split()[-1] == str(1 << 2), probe.stdout + probe.stderr
    r = _run(["-m", "pytest", "tests/test_gpu_parity.py", "tests/test_gpu_batch.py", "-m", "gpu", "-q", "-x",
              "-p", "no:cacheprovider", "-k", "not fifty_epochs and not full_size"], env, 1800)
    assert r.returncode == 0, r.stdout[-4000:] + r.stderr[-2000:]
    summary = [ln for ln in r.stdout.splitlines() if " passed" in ln][-1]
    print(summary)
    assert int(summary.split(" passed")[0].split()[-1]) >= 30, summary


def test_the_default_build_has_no_checks(lib):
    assert lib.emg_debug_bounds_errors() is None
    assert lib.emg_debug_bounds_selftest() is None
