"""The bounds-checking build (-DIPC_DEBUG_BOUNDS; the stand-in for a memory
checker): tests/bounds_workload.py runs every kind of level launch through it
in a child process and requires the oracle's results and no access outside
an array."""
import os
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def test_bounds_checked_build_runs_clean():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2502_04093_gb300 import build
    build.build(bounds=True)
    env = dict(os.environ, IPC_BOUNDS_CHECK="1")
    r = subprocess.run([sys.executable, os.path.join(HERE, "bounds_workload.py")], env=env,
                       capture_output=True, text=True, timeout=1800)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert "no access out of bounds" in r.stdout


def test_regular_build_has_no_record():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    if os.environ.get("IPC_BOUNDS_CHECK") == "1":
        pytest.skip("this process runs the checked build")
    from paper_2502_04093_gb300 import ipc
    with pytest.raises(ipc.IpcError) as e:
        ipc.ipc_debug_bounds()
    assert e.value.rc == ipc.IPC_EINVAL
