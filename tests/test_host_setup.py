"""The library's host-side set-up (csrc/setup.cpp), compiled with g++ alone
and run on the CPU, against the oracle: the canonical mesh (Sec. 3), the
truncated Chebyshev coefficients of e^{tL} (Sec. 2.4) with the widest
exponential the library accepts, and the Riemann-sum shifts and weights
(Sec. 2.2).  The GPU tests reach the same code only through a context."""

import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import averaging, expo
from oracle.mesh import build_mesh

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
R = 6.37122e6


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    exe = tmp_path_factory.mktemp("host_setup") / "harness"
    csrc = os.path.join(ROOT, "paper_2103_07706_gb300", "csrc")
    subprocess.run([gxx, "-O2", "-std=c++17", "-ffp-contract=off", "-I", os.path.join(ROOT, "include"), "-I", csrc,
                    os.path.join(ROOT, "tests", "host_setup_harness.cpp"), os.path.join(csrc, "setup.cpp"),
                    "-o", str(exe)], check=True)
    return exe


def run(exe, *args):
    out = subprocess.run([str(exe), *map(str, args)], check=True, capture_output=True, text=True).stdout
    return out.strip().split("\n")


@pytest.mark.parametrize("r", [0, 1, 2, 3])
def test_mesh_matches_oracle(harness, tmp_path, r):
    V, F, E = map(int, run(harness, "mesh", r, repr(R), tmp_path / "m")[0].split())
    assert (F, E, V) == (20 * 4 ** r, 30 * 4 ** r, 10 * 4 ** r + 2)
    verts = np.fromfile(tmp_path / "m.verts", dtype=np.float64).reshape(V, 3)
    cells = np.fromfile(tmp_path / "m.cells", dtype=np.int32).reshape(F, 3)
    o = build_mesh(r, R)
    assert np.array_equal(cells, o.cells)
    assert np.abs(verts - o.verts).max() <= 1e-15 * R


@pytest.mark.parametrize("Lb", [0.0, 0.5, 3.0, 42.0, 168.0])
def test_chebyshev_coefficients_match_oracle(harness, Lb):
    out = run(harness, "cheb", repr(Lb), "1e-6")
    c = np.array([float(x) for x in out[1:1 + int(out[0])]])
    want = expo.truncated_coefficients(Lb, 1.0, 1e-6)  # lambda_max |t| = Lb
    assert len(c) == len(want)
    assert np.abs(c - want).max() <= 1e-13


@pytest.mark.parametrize("Lb", ["16384.5", "1e300", "inf", "nan", "-1"])
def test_exponentials_beyond_the_limit_are_refused(harness, Lb):
    """lambda_max |t| above 16384 (PAVG_MAX_CHEB_ARG), not finite or negative:
    an empty list, which the entry points turn into PAVG_ERR_INVAL before
    the O(N^2) transform would run."""
    assert run(harness, "cheb", Lb, "1e-6") == ["0"]


@pytest.mark.parametrize("T,M,rule", [(3600.0, 8, 0), (3600.0, 5, 0), (7200.0, 7, 1), (14400.0, 128, 0)])
def test_shifts_and_weights_match_oracle(harness, T, M, rule):
    out = run(harness, "shifts", repr(T), M, rule)
    assert out[0] == "0"
    sw = np.array([[float(v) for v in line.split()] for line in out[1:]])
    s, w = averaging.shifts_and_weights(T, M, rule)
    assert sw.shape == (M, 2)
    assert np.abs(sw[:, 0] - s).max() <= 1e-12 * T
    assert np.abs(sw[:, 1] - w).max() <= 1e-15


@pytest.mark.parametrize("T,M,rule", [(3600.0, 4, 1), (3600.0, 1, 1), (3600.0, 0, 0), (3600.0, 3, 7)])
def test_invalid_point_sets_are_refused(harness, T, M, rule):
    """The closed rule needs an odd M >= 3; M >= 1; the rule must exist."""
    assert run(harness, "shifts", repr(T), M, rule)[0] != "0"
