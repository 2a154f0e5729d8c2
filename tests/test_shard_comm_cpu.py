"""Host check of the collectives that the row-sharded tableau's rank threads
use (csrc/shard_comm.h): correctness over many rounds, and an aborting rank
releases the others.  Compiled with the host C++ compiler; no GPU."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2408_00384_gb300", "csrc")


def test_thread_rank_collectives(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    exe = str(tmp_path / "shard_comm_check")
    subprocess.run([cxx, "-O2", "-std=c++17", "-pthread", "-I", CSRC,
                    os.path.join(HERE, "cpp", "shard_comm_check.cpp"), "-o", exe],
                   check=True, capture_output=True, text=True)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
