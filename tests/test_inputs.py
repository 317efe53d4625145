"""The seeded input generators (paper_2103_07706_gb300/inputs.py) against
library routines and their own stated properties."""

import numpy as np
import pytest

from paper_2103_07706_gb300.inputs import batch_workload, harmonic_state, real_sph_harm_sum


def test_real_harmonics_match_scipy():
    scipy_special = pytest.importorskip("scipy.special")
    if not hasattr(scipy_special, "sph_harm_y"):
        pytest.skip("scipy without sph_harm_y")
    rng = np.random.default_rng(0)
    P = rng.standard_normal((60, 3))
    L = 7
    coeffs = rng.standard_normal((L + 1, 2 * L + 1))
    got = real_sph_harm_sum(P, coeffs, L)
    th = np.arccos(P[:, 2] / np.linalg.norm(P, axis=1))
    ph = np.arctan2(P[:, 1], P[:, 0])
    want = np.zeros(len(P))
    for l in range(1, L + 1):
        for m in range(-l, l + 1):
            Y = scipy_special.sph_harm_y(l, abs(m), th, ph)
            # real orthonormal harmonics; scipy includes the Condon-Shortley phase
            if m == 0:
                want += coeffs[l, L] * Y.real
            elif m > 0:
                want += coeffs[l, L + m] * np.sqrt(2) * (-1) ** m * Y.real
            else:
                want += coeffs[l, L + m] * np.sqrt(2) * (-1) ** m * Y.imag
    assert np.abs(got - want).max() <= 1e-13 * np.abs(want).max()


def test_harmonic_state_is_seeded_and_scaled():
    from oracle.mesh import build_mesh
    m = build_mesh(2, 6.37122e6)
    U1, info = harmonic_state(m.verts, m.cells, 3, 8)
    U2, _ = harmonic_state(m.verts, m.cells, 3, 8)
    U3, _ = harmonic_state(m.verts, m.cells, 4, 8)
    assert np.array_equal(U1, U2) and not np.array_equal(U1, U3)
    eta = U1[-3 * len(m.cells):]
    assert np.sqrt(np.mean(eta ** 2)) == pytest.approx(100.0, rel=1e-12)
    assert 0.0 < info["rossby"] < 1.0


def test_batch_workload_recipe():
    w = batch_workload()
    assert len(w) == 64
    assert {x["refinement"] for x in w} == {4, 5, 6}
    assert all(0.25 * 3600 <= x["T"] <= 4 * 3600 for x in w)
    assert {x["M"] for x in w} <= {16, 32, 64, 128}
    assert len({x["state_seed"] for x in w}) == 64
    assert w == batch_workload()
