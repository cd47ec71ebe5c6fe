"""The benchmark's algorithmic FLOP table (paper_2109_07719_gb300/flops.json) is the
output of the counting build of the kernels' step functions (flopcount.cpp): a
change to the step code that is not followed by regenerating the table fails here."""
import json
import os
import shutil
import subprocess

import pytest

PKG = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2109_07719_gb300")


def _build_and_run(tmp_path, name, *args):
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    exe = tmp_path / name
    subprocess.run([cxx, "-O1", "-std=c++17", "-o", str(exe), os.path.join(PKG, name + ".cpp")], check=True,
                   cwd=PKG)
    return subprocess.run([str(exe), *args], check=True, capture_output=True, text=True, cwd=PKG).stdout


def test_flop_table_matches_the_step_code(tmp_path):
    fresh = json.loads(_build_and_run(tmp_path, "flopcount"))
    with open(os.path.join(PKG, "flops.json")) as f:
        stored = json.load(f)
    assert fresh == stored, "flops.json is stale: regenerate it with flopcount.cpp"
