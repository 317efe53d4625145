"""Pins of the oracle's phase average (paper Sec. 2.2) and Lawson RK4 (Sec. 2.3)."""

import numpy as np
import pytest
from scipy.linalg import expm

from oracle import averaging, spectrum
from paper_2103_07706_gb300.inputs import harmonic_state


def test_bump_and_weights():
    assert averaging.bump(np.array([0.5, -0.5, 0.7]))[:].max() == 0.0
    assert abs(averaging.bump(np.array([0.0]))[0] - np.exp(-4.0)) < 1e-18
    for M in (1, 2, 8, 64, 128):
        s, w = averaging.shifts_and_weights(3600.0, M)
        assert abs(w.sum() - 1.0) < 1e-15
        assert np.allclose(w, w[::-1], rtol=0, atol=1e-17)
        assert np.allclose(s, -s[::-1], rtol=0, atol=1e-9)
        assert (np.abs(s) < 1800.0).all()
    s, w = averaging.shifts_and_weights(3600.0, 5, averaging.QUAD_CLOSED)
    assert s[0] == -1800.0 and s[-1] == 1800.0 and w[0] == 0.0 and w[-1] == 0.0
    assert abs(w.sum() - 1.0) < 1e-15
    s, w = averaging.shifts_and_weights(3600.0, 1)
    assert s[0] == 0.0 and w[0] == 1.0


def test_riemann_sum_converges_to_integral():
    """sum_m w_m g(s_m) -> int rho(s/T) g / int rho(s/T) for smooth g."""
    T = 2.0
    x = np.linspace(-0.5, 0.5, 200001)
    rho = averaging.bump(x)
    g = np.cos(3.0 * x * T)
    exact = np.trapezoid(rho * g, x) / np.trapezoid(rho, x)
    s, w = averaging.shifts_and_weights(T, 64)
    assert abs((w * np.cos(3.0 * s)).sum() - exact) < 1e-8


@pytest.fixture(scope="module")
def r1_model():
    from tests.conftest import oracle_model
    m = oracle_model(1, cheb_tol=1e-14)
    A = spectrum.dense_L(m.ops)
    m.lam = np.abs(np.linalg.eigvals(A)).max() * 1.0001
    U, _ = harmonic_state(m.mesh.verts, m.mesh.cells, 2103, 4)
    return m, A, U


def test_averaged_rhs_against_dense_exponentials(r1_model):
    """sum_m w_m expm(-s_m L) N(expm(s_m L) U) with dense expm (Eq. vt_discretised)."""
    m, A, U = r1_model
    T, M = 3600.0, 6
    s, w = averaging.shifts_and_weights(T, M)
    ref = sum(w[k] * expm(-s[k] * A) @ m.N(expm(s[k] * A) @ U) for k in range(M))
    got = m.averaged_rhs(T, M, U)
    assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref)


def test_T_to_zero_recovers_N(r1_model):
    """Sec. 2.2: as T -> 0 the average tends to the unaveraged nonlinearity,
    at second order for the symmetric rule; T = 0 and M = 1 give it exactly."""
    m, A, U = r1_model
    N0 = m.N(U)
    assert np.array_equal(m.averaged_rhs(0.0, 8, U), N0)
    assert np.array_equal(m.averaged_rhs(3600.0, 1, U), N0)
    e = [np.linalg.norm(m.averaged_rhs(T, 4, U) - N0) for T in (200.0, 20.0)]
    assert 80.0 < e[0] / e[1] < 120.0


def test_average_settles_beyond_four_points_per_period(om):
    """Sec. 2.2: the average stops depending on M once the shifts sample the
    fastest oscillation at four points per period, M >= 2 lambda_max T / pi
    (3.25 here).  Against M = 64: errors of percents below that, under 1e-3
    from M = 8 on.  Shifts spread over [-T, T] instead of [-T/2, T/2] would
    halve the effective M and break the second bound."""
    m = om(2, lambda_max=0.00142)
    m.lam = 0.00142
    T = 3600.0
    assert 3.0 < 2 * m.lam * T / np.pi < 4.0
    U, _ = harmonic_state(m.mesh.verts, m.mesh.cells, 2103, 8)
    ref = m.averaged_rhs(T, 64, U)
    nu = m.n_u

    def err(M):
        d = m.averaged_rhs(T, M, U) - ref
        return (np.linalg.norm(d[:nu]) / np.linalg.norm(ref[:nu]),
                np.linalg.norm(d[nu:]) / np.linalg.norm(ref[nu:]))

    below = [err(M) for M in (2, 3)]
    above = [err(M) for M in (8, 16)]
    for k in range(2):
        assert min(e[k] for e in below) > 20 * max(e[k] for e in above)
        assert max(e[k] for e in above) < 1e-3


def test_rest_state_and_mass(om):
    m = om(2)
    m.lam = 0.00142
    rest = np.zeros(m.n)
    rest[m.n_u:] = 2.0
    assert np.abs(m.averaged_rhs(3600.0, 4, rest)).max() < 1e-14
    U, _ = harmonic_state(m.mesh.verts, m.mesh.cells, 2103, 8)
    S = m.averaged_rhs(1800.0, 4, U)
    assert abs(m.ops.mass(S)) <= 1e-14 * m.ops.norms(S)[2] * np.sqrt(4 * np.pi) * 6.37122e6


class _SmoothModel:
    """A small model with a skew linear part and a smooth quadratic N, so that
    the Lawson RK4 formula can be checked for its order against an accurate
    ODE solve (the shallow-water N is only piecewise smooth: its upwind
    switch breaks the smoothness the order argument needs)."""

    def __init__(self):
        rng = np.random.default_rng(11)
        B = rng.standard_normal((6, 6))
        self.A = 3e-4 * (B - B.T)
        self.C = 2e-5 * rng.standard_normal((6, 6, 6))

    def expL(self, t, V):
        return expm(t * self.A) @ V

    def N(self, V):
        return np.einsum("ijk,j,k->i", self.C, V, V)

    def averaged_rhs(self, T, M, V, rule=0):
        return averaging.averaged_rhs(self, T, M, V, rule)


def test_lawson_rk4_fourth_order_on_smooth_problem():
    """Sec. 2.3: the averaged Lawson RK4 step is fourth order for
    U' = L U + N-bar(U) (N-bar at fixed T, M); checked against solve_ivp."""
    from scipy.integrate import solve_ivp
    from oracle.timestep import lawson_rk4_step
    mdl = _SmoothModel()
    T, M, span = 2000.0, 4, 20000.0
    U0 = np.array([1.0, -0.5, 0.3, 0.8, -1.2, 0.4])
    sol = solve_ivp(lambda t, y: mdl.A @ y + mdl.averaged_rhs(T, M, y), (0, span), U0,
                    method="DOP853", rtol=1e-13, atol=1e-15)
    ref = sol.y[:, -1]
    errs = []
    for n in (20, 40, 80):
        U = U0.copy()
        for _ in range(n):
            U = lawson_rk4_step(mdl, span / n, T, M, U)
        errs.append(np.linalg.norm(U - ref))
    assert 14.0 < errs[0] / errs[1] < 21.0 and 14.0 < errs[1] / errs[2] < 21.0


def test_shallow_water_timestep_converges(om):
    """The full model's step converges as dt shrinks (first order at worst,
    because the upwind switch makes N only Lipschitz)."""
    from tests.conftest import oracle_model
    m = oracle_model(1, cheb_tol=1e-13)
    m.lam = 0.00071 * 1.001
    U0, _ = harmonic_state(m.mesh.verts, m.mesh.cells, 7, 4, eta_rms=400.0)
    T, M, span = 1800.0, 3, 2 * 3600.0
    ref = m.timestep(span / 32, T, M, U0, 32)
    e = [np.linalg.norm(m.timestep(span / n, T, M, U0, n) - ref) for n in (2, 4)]
    assert e[1] < 0.5 * e[0]
    assert e[1] < 1e-3 * np.linalg.norm(U0)


def test_timestep_rest_state_and_mass(om):
    m = om(1)
    m.lam = 0.00071
    rest = np.zeros(m.n)
    rest[m.n_u:] = 1.5
    out = m.timestep(900.0, 3600.0, 4, rest, 2)
    # the average of the rest state is exactly zero; the truncated exponential
    # keeps the steady mode to within the truncation threshold (its even
    # coefficients sum to 1 minus the dropped tail)
    assert np.abs(out - rest).max() < 2 * 2 * m.p.cheb_tol * 1.5
    U, _ = harmonic_state(m.mesh.verts, m.mesh.cells, 2103, 4)
    out = m.timestep(900.0, 3600.0, 4, U, 2)
    assert abs(m.ops.mass(out) - m.ops.mass(U)) < 1e-12 * abs(U[m.n_u:]).max() * 4 * np.pi * 6.37122e6 ** 2


def test_parallel_literal_sum_is_bitwise_the_sequential_one():
    """oracle/parallel.py spreads the terms of Eq. vt_discretised over spawned
    processes and adds them in shift order: the result must be the sequential
    oracle's, bit for bit."""
    from oracle.model import OracleModel, OracleParams
    from oracle.parallel import OraclePool
    from paper_2103_07706_gb300.inputs import harmonic_state
    p = OracleParams(refinement=1, lambda_max=0.00072)
    m = OracleModel(p)
    U, _ = harmonic_state(m.mesh.verts, m.mesh.cells, 2103, 4)
    want = m.averaged_rhs(3600.0, 6, U)
    with OraclePool(p, workers=2) as pool:
        got = pool.averaged_rhs(3600.0, 6, U)
        nu, ne = pool.norms(want)
    assert np.array_equal(got, want)
    u, e = want[: m.n_u], want[m.n_u:]
    assert nu == np.sqrt(u @ (m.ops.M1 @ u)) and ne == np.sqrt(e @ (m.ops.M2 @ e))


def test_shift_groups_partition_the_sum():
    """Partial sums over contiguous shift groups (Sec. 2.5's distribution of
    the independent terms) add up to the whole Riemann sum, for uneven groups,
    the closed rule with its zero-weight endpoints, and T = 0."""
    from tests.conftest import oracle_model
    m = oracle_model(1, lambda_max=0.00072)
    U, _ = harmonic_state(m.mesh.verts, m.mesh.cells, 2103, 4)
    for T, M, rule, cuts in [(3600.0, 8, 0, [0, 3, 4, 8]), (1800.0, 7, 1, [0, 1, 6, 7]), (0.0, 4, 0, [0, 1, 4])]:
        full = m.averaged_rhs(T, M, U, rule)
        parts = [averaging.averaged_rhs_group(m, T, M, a, b, U, rule) for a, b in zip(cuts[:-1], cuts[1:])]
        tot = sum(parts)
        assert np.abs(tot - full).max() <= 1e-13 * np.abs(full).max()
        assert all(np.abs(p).max() > 0 for p, a, b in zip(parts, cuts[:-1], cuts[1:]) if rule == 0 or 0 < a < M - 1)


def test_shift_marching_equals_the_direct_sum():
    """Shift marching (V_{m+1} = e^{ds L} V_m forward, Horner in e^{-ds L}
    backward) is the same sum as the direct per-shift form: with a tail
    threshold of 1e-15 the two agree to 1e-12, for both point rules; with
    the paper's 1e-6 they differ by the extra truncations (more than 1e-9,
    so the comparison does see the marching path)."""
    from oracle.model import OracleModel, OracleParams
    for rule, M in ((averaging.QUAD_MIDPOINT, 8), (averaging.QUAD_CLOSED, 7)):
        m = OracleModel(OracleParams(refinement=1, lambda_max=0.00072, cheb_tol=1e-15, quad_rule=rule))
        U, _ = harmonic_state(m.mesh.verts, m.mesh.cells, 2103, 4)
        U[m.n_u:] += np.random.default_rng(1).standard_normal(m.n_eta)
        a = m.averaged_rhs(7200.0, M, U)
        b = averaging.averaged_rhs_marching(m, 7200.0, M, U, rule)
        assert np.abs(a - b).max() <= 1e-12 * np.abs(a).max()
    m6 = OracleModel(OracleParams(refinement=1, lambda_max=0.00072))
    a = m6.averaged_rhs(7200.0, 8, U)
    b = averaging.averaged_rhs_marching(m6, 7200.0, 8, U)
    assert np.abs(a - b).max() > 1e-9 * np.abs(a).max()
