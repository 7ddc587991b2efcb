"""The index walks of the ghost fill (csrc/mpw_index.cuh), compiled for the
host with stand-ins for the CUDA qualifiers: the strided walk over a
two-field block agrees with the quotient/remainder decomposition it replaces
for every block shape up to 70 x 40 x 34 and thread strides 128 and 256, and
the hollow-box enumeration of the outer ghost shell (walls three cells thick,
Sec. 2.4) visits every shell point exactly once, identically in its 32-bit
and 64-bit forms."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def index_host(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    exe = str(tmp_path_factory.mktemp("index") / "index_host")
    subprocess.run([cxx, "-O2", "-std=c++17", "-o", exe, os.path.join(HERE, "host", "index_host.cpp")], check=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    return {line.split()[0]: int(line.split()[1]) for line in out.splitlines()}


def test_block_walk_matches_divisions(index_host):
    assert index_host["walk_checked"] > 10_000_000
    assert index_host["walk_mismatches"] == 0


def test_shell_enumeration_covers_each_point_once(index_host):
    # 262^3 - 256^3 + 134^3 - 128^3 + ... : the 256^3 global's shell alone has 1,207,512 points
    assert index_host["shell_points"] > 1_207_512
    assert index_host["shell_mismatches"] == 0
