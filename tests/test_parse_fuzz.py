"""Robustness of the host-side parsers of untrusted bytes (the selection
from a container's tables, its byte ranges, the coded-container decoder):
seeded mutations of valid containers (bytes, bits, truncation, insertion,
extreme table fields) must each be parsed or refused with a status code,
never crash. Runs in a child process so that a crash fails the test."""
import os
import subprocess
import sys

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.mark.parametrize("seed", [1, 2])
def test_mutated_containers_are_parsed_or_refused(seed):
    from paper_2502_04093_gb300 import build
    build.build()
    r = subprocess.run([sys.executable, os.path.join(HERE, "parse_fuzz_worker.py"), str(seed), "400"],
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    ok, err = map(int, r.stdout.split()[-2:])
    assert ok + err == 3 * 400 and err > 0
