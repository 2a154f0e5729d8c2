"""Host logic of the gate compilers, without a GPU.

The C++ checks in tests/cpp compile random gate lists with the library's own
compiler (program.cpp, blocks.cpp):
* into two-qubit blocks, applied to random 32-row words with the device
  kernel's block formulas and compared with the gates applied one at a time
  by the Aaronson-Gottesman rules;
* into ASAP layers (the form the single-CTA and batched engines run),
  checked against the list: segments, codes, per-qubit order, each gate's
  ASAP layer computed independently, disjoint qubits within a layer, the
  noise table.
A third check covers tab_batch_run's chunking of a circuit list.
"""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(ROOT, "paper_2408_00384_gb300", "csrc")


def _cuda_include():
    for d in (os.environ.get("CUDA_HOME", ""), "/usr/local/cuda"):
        if d and os.path.exists(os.path.join(d, "include", "cuda_runtime.h")):
            return os.path.join(d, "include")
    return None


def test_block_compiler_matches_gate_rules(tmp_path):
    cxx = shutil.which("g++")
    inc = _cuda_include()
    if cxx is None or inc is None:
        pytest.skip("needs g++ and the CUDA headers")
    exe = str(tmp_path / "block_compiler_check")
    cmd = [cxx, "-O2", "-std=c++17", "-pthread", "-I", inc, "-I", CSRC, "-I", os.path.join(ROOT, "include"),
           os.path.join(HERE, "cpp", "block_compiler_check.cpp"),
           os.path.join(CSRC, "program.cpp"), os.path.join(CSRC, "blocks.cpp"),
           os.path.join(CSRC, "pool.cpp"), "-o", exe]
    subprocess.run(cmd, check=True, capture_output=True, text=True)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "bad 0" in r.stdout


def test_layer_compiler_matches_list(tmp_path):
    cxx = shutil.which("g++")
    inc = _cuda_include()
    if cxx is None or inc is None:
        pytest.skip("needs g++ and the CUDA headers")
    exe = str(tmp_path / "layer_compiler_check")
    cmd = [cxx, "-O2", "-std=c++17", "-pthread", "-I", inc, "-I", CSRC, "-I", os.path.join(ROOT, "include"),
           os.path.join(HERE, "cpp", "layer_compiler_check.cpp"),
           os.path.join(CSRC, "program.cpp"), os.path.join(CSRC, "blocks.cpp"),
           os.path.join(CSRC, "pool.cpp"), "-o", exe]
    subprocess.run(cmd, check=True, capture_output=True, text=True)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "bad 0" in r.stdout


def test_batch_chunk_cuts(tmp_path):
    cxx = shutil.which("g++")
    inc = _cuda_include()
    if cxx is None or inc is None:
        pytest.skip("needs g++ and the CUDA headers")
    exe = str(tmp_path / "chunk_cuts_check")
    cmd = [cxx, "-O2", "-std=c++17", "-I", inc, "-I", CSRC, "-I", os.path.join(ROOT, "include"),
           os.path.join(HERE, "cpp", "chunk_cuts_check.cpp"), "-o", exe]
    subprocess.run(cmd, check=True, capture_output=True, text=True)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "bad 0" in r.stdout
