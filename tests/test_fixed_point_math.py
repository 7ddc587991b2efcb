"""The fixed-point exp and square root of the analytic boundary
(csrc/mpw_fxmath.cuh), compiled for the host with stand-ins for its CUDA
intrinsics and checked against the long double functions: exp within 1.5
units in the last place over the whole range it serves (x in [-704, 0]),
exact at 0, 0 at and below -704 and for -inf, NaN propagated; sqrt(y) and
1/(2 sqrt(y)) within 0.53 units over [2^-40, 2^40], exact at powers of 4.
The same header is compiled into the device closed forms (Sec. 3), whose
values the GPU tests compare with the oracle."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def exp_host(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    exe = str(tmp_path_factory.mktemp("fxmath") / "fxmath_host")
    subprocess.run([cxx, "-O2", "-std=c++17", "-o", exe, os.path.join(HERE, "host", "fxmath_host.cpp")], check=True)
    return exe


def run(exe, count):
    out = subprocess.run([exe, str(count)], check=True, capture_output=True, text=True).stdout
    return {line.split()[0]: line.split()[1:] for line in out.splitlines()}


def test_error_bounds(exp_host):
    r = run(exp_host, 500000)
    assert float(r["worst_ulp"][0]) <= 1.5, r["worst_ulp"]
    assert float(r["worst_sqrt_ulp"][0]) <= 0.53, r["worst_sqrt_ulp"]
    assert float(r["worst_half_inv_ulp"][0]) <= 0.53, r["worst_half_inv_ulp"]


def test_special_values(exp_host):
    r = run(exp_host, 1)
    assert float(r["zero"][0]) == 1.0
    assert float(r["negzero"][0]) == 1.0
    assert float(r["tiny"][0]) == 1.0
    assert float(r["m704"][0]) == 0.0
    assert float(r["minf"][0]) == 0.0
    assert r["nan"][0] == "1"
    got, want = (float(v) for v in r["m703"])
    assert abs(got - want) <= 2e-16 * want
    assert [float(v) for v in r["sqrt4"]] == [2.0, 0.25]
    assert r["sqrtnan"][0] == "1"
