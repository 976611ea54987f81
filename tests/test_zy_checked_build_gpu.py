"""The checked build (every shared-memory and global index of the fused step
verified on the device; a failure returns SPG_ECHECK and skips the access)
runs the fused-step parity cases: odd and ragged shapes, every tile variant,
both iterate storages, batches, BF16 data, the restart and Fourier paths and
graph replay. It stands in for a memory checker, which is not available."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CASES = ("few_steps_odd_shapes or tile_variants or batch_equals or bf16_storage or gradient_restart "
         "or graph_replay or vol64_full_schedule or fourier_solve")


def test_fused_step_index_checks():
    env = dict(os.environ, SPG_CHECKED="1")
    cmd = [sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider",
           "tests/test_gpu_parity.py", "tests/test_fourier_gpu.py", "-k", CASES]
    res = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=1800)
    tail = (res.stdout + res.stderr)[-3000:]
    print(tail)
    assert res.returncode == 0, tail
    assert "passed" in res.stdout and "SPG_ECHECK" not in res.stdout
