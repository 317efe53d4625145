"""Pins of the oracle's L and N (paper Sec. 2.5) against closed forms and invariants."""

import numpy as np
import pytest

from oracle import spectrum
from oracle.elements import dg1_values
from oracle.operators import UPWIND_AS_PRINTED
from oracle.quadrature import triangle_rule
from paper_2103_07706_gb300.inputs import harmonic_state

R = 6.37122e6


def _state(m, seed=2103, lmax=8):
    U, _ = harmonic_state(m.mesh.verts, m.mesh.cells, seed, lmax)
    return U


def proj_u(ops, v):
    """L2 projection of a 3-vector field v(x) onto BDM2."""
    A = ops.asm
    xq, wq = triangle_rule(4)
    psi = A.element.values(xq)
    x = A.a[:, None, :] + np.einsum("fxa,qa->fqx", A.J, xq)
    b_loc = np.einsum("q,fxa,qia,fqx->fi", wq, A.J, psi, v(x)) * A.sign
    b = np.zeros(ops.n_u)
    np.add.at(b, A.udofs.ravel(), b_loc.ravel())
    return ops.solve_M1(b)


def proj_eta(ops, f):
    A = ops.asm
    xq, wq = triangle_rule(4)
    x = A.a[:, None, :] + np.einsum("fxa,qa->fqx", A.J, xq)
    b = np.einsum("q,f,qi,fq->fi", wq, A.det, dg1_values(xq), f(x)).ravel()
    return ops.solve_M2(b)


def test_spectrum_purely_imaginary(om):
    """L is skew in the energy inner product, so its eigenvalues are imaginary (Sec. 2.5)."""
    m = om(1)
    ev = np.linalg.eigvals(spectrum.dense_L(m.ops))
    assert np.abs(ev.real).max() <= 1e-10 * np.abs(ev).max()


@pytest.mark.parametrize("r", [2, 3])
def test_energy_skewness(om, r):
    m = om(r)
    U = np.random.default_rng(3).standard_normal(m.n)
    LU = m.L(U)
    assert abs(spectrum.w_inner(m.ops, LU, U)) <= 1e-13 * np.sqrt(
        spectrum.w_inner(m.ops, LU, LU) * spectrum.w_inner(m.ops, U, U))
    u = U[: m.n_u]
    assert abs(u @ (m.ops.C @ u)) <= 1e-14 * abs(u) @ (abs(m.ops.C) @ abs(u))


def test_rest_state_is_steady(om):
    """(u, eta) = (0, const): L U = 0 and N(U) = 0."""
    m = om(3)
    U = np.zeros(m.n)
    U[m.n_u:] = 7.0
    LU = m.L(U)
    scale = m.ops.g * 7.0 * np.abs(m.ops.D).sum(axis=0).max()
    assert np.abs(m.ops.linear_rhs(U)).max() <= 1e-14 * scale
    assert np.abs(m.N(U)).max() == 0.0
    assert np.isfinite(LU).all()


def test_mass_conservation_and_homogeneity(om):
    m = om(3)
    U = _state(m)
    NR = m.ops.nonlinear_rhs(U)
    LR = m.ops.linear_rhs(np.random.default_rng(4).standard_normal(m.n))
    assert abs(NR[m.n_u:].sum()) <= 1e-15 * np.abs(NR[m.n_u:]).sum()
    assert abs(LR[m.n_u:].sum()) <= 1e-14 * np.abs(LR[m.n_u:]).sum()
    # b = 0: N is quadratic and the upwind choice is invariant under positive scaling
    N2 = m.ops.nonlinear_rhs(2.0 * U)
    assert np.abs(N2 - 4.0 * NR).max() <= 1e-14 * np.abs(NR).max()


def test_upwind_elevation_flux_dissipates(om):
    """With a divergence-free velocity, the upwind elevation flux makes
    eta . r_eta = -1/2 sum_facets int |u.n| [[eta]]^2 <= 0 (Sec. 2.5: upwinding is
    the scheme's only dissipation).  A downwind (or centred-with-wrong-sign)
    reading breaks the sign."""
    m = om(3)
    U = _state(m)
    rng = np.random.default_rng(5)
    U[m.n_u:] = rng.standard_normal(m.n_eta) * 50.0
    r = m.ops.nonlinear_rhs(U)[m.n_u:]
    eta = U[m.n_u:]
    assert eta @ r < 0.0
    assert abs(m.ops.D @ U[: m.n_u]).max() < 1e-12 * abs(m.ops.D).max() * abs(U[: m.n_u]).max()


@pytest.mark.parametrize("upwind", [0, UPWIND_AS_PRINTED])
def test_velocity_terms_do_no_work_on_divergence_free_flow(om, upwind):
    """Tested against w = u, the vorticity term's cell and facet integrands
    carry u^perp . u = 0, and the kinetic-energy term carries div u.  So for a
    discretely divergence-free u the velocity part of N does no work,
    u . r_u = 0 to rounding, whichever side u~ is taken from (Sec. 2.5).  For
    the same reason the energy of a long run cannot tell the two readings of
    the velocity upwind rule apart.  Dropping a product-rule term in the
    derivative of u^perp . w, or taking the other cell's u in a facet's
    u^perp . w, leaves a residual of 1e-5 or more of sum |u_i r_i|."""
    m = om(3, upwind=upwind)
    U = _state(m)
    u = U[: m.n_u]
    assert abs(m.ops.D @ u).max() < 1e-12 * abs(m.ops.D).max() * abs(u).max()
    r = m.ops.nonlinear_rhs(U)[: m.n_u]
    assert abs(u @ r) <= 1e-13 * np.abs(u * r).sum()


def _solid_body_errors(m, omega_body=1e-5, amp=100.0):
    ops = m.ops
    ub = lambda x: omega_body * np.stack([-x[..., 1], x[..., 0], 0 * x[..., 0]], -1)  # noqa: E731

    def n_u_exact(x):
        # -(u.grad)u for zonal solid-body rotation: the tangential part of the
        # centripetal acceleration, omega^2 P (x, y, 0)
        xp = np.stack([x[..., 0], x[..., 1], 0 * x[..., 0]], -1)
        xh = x / np.linalg.norm(x, axis=-1, keepdims=True)
        return omega_body ** 2 * (xp - (xp * xh).sum(-1, keepdims=True) * xh)

    eta_f = lambda x: amp * x[..., 0] / R                      # noqa: E731
    n_eta_exact = lambda x: omega_body * amp * x[..., 1] / R    # noqa: E731  (-u . grad eta)
    U = np.concatenate([proj_u(ops, ub), proj_eta(ops, eta_f)])
    nu, ne = ops.split(m.N(U))
    pu, pe = proj_u(ops, n_u_exact), proj_eta(ops, n_eta_exact)
    eu, ee = nu - pu, ne - pe
    return (np.sqrt(eu @ (ops.M1 @ eu) / (pu @ (ops.M1 @ pu))),
            np.sqrt(ee @ (ops.M2 @ ee) / (pe @ (ops.M2 @ pe))))


@pytest.mark.parametrize("upwind", [0, UPWIND_AS_PRINTED])
def test_nonlinear_consistency_solid_body(om, upwind):
    """N converges to -(u.grad)u and -div(u eta) for solid-body rotation.

    On flat facets the rate is first order (facet normals differ from the
    sphere's by O(h)).  A flipped facet sign, a dropped kinetic-energy term or
    mismatched facet points leave an O(1) error that does not decrease.
    """
    errs = [_solid_body_errors(om(r, upwind=upwind)) for r in (2, 3, 4)]
    for k in range(2):
        e = [x[k] for x in errs]
        assert e[2] < 0.06
        assert e[0] / e[1] > 1.8 and e[1] / e[2] > 1.8


def _geostrophic_residual(m, u0=20.0):
    """Relative size of L U for the zonal geostrophic steady state.

    Sec. 2.1 writes the linear operator as (-f u_perp - g grad eta, -H div u)
    with f = 2 Omega z / R.  The zonal solid-body flow u = u0 cos(lat) e_lon
    = (u0 / R) (-y, x, 0) is divergence-free, and with
    eta = -(Omega u0 R / g) (z / R)^2 the Coriolis force f k x u is balanced by
    the pressure gradient g grad eta, so the continuous L U is zero.  The
    discrete velocity part -M1^{-1} (C u - g D^T eta) must vanish as the mesh
    is refined, measured against the size of the Coriolis term alone.
    """
    ops = m.ops
    om_, g = ops.asm.omega, ops.g
    ub = lambda x: (u0 / R) * np.stack([-x[..., 1], x[..., 0], 0 * x[..., 0]], -1)  # noqa: E731
    eta_f = lambda x: -(om_ * u0 * R / g) * (x[..., 2] / R) ** 2                      # noqa: E731
    U = np.concatenate([proj_u(ops, ub), proj_eta(ops, eta_f)])
    lu = ops.L(U)[: m.n_u]
    cor = ops.solve_M1(ops.C @ U[: m.n_u])
    return np.sqrt(lu @ (ops.M1 @ lu) / (cor @ (ops.M1 @ cor)))


def test_geostrophic_balance_is_steady(om):
    """L annihilates the discrete geostrophic state at the discretisation's rate.

    The Coriolis matrix is the only part of L that the energy, skewness,
    spectrum and rest-state pins cannot see (they hold for any sign or scale
    of f).  The correct operator converges at first order on flat facets
    (2.7 %, 1.0 %, 0.44 %, 0.21 % at refinements 2-5; the facet normals
    differ from the sphere's by O(h)).  A flipped sign of -C u leaves a
    residual of 2.0 (twice the Coriolis term) and f at half its value leaves
    1.0 (an unbalanced pressure gradient as large as the halved Coriolis
    term); neither decreases with refinement.
    """
    e = [_geostrophic_residual(om(r)) for r in (2, 3, 4)]
    assert e[0] < 0.04 and e[2] < 0.006, e
    assert e[0] / e[1] > 1.8 and e[1] / e[2] > 1.8, e


def test_strong_form_of_the_elevation_terms_is_the_same_quantity():
    """The elevation equation's weak form of Sec. 2.5 (int grad phi . u (eta-b)
    minus the upwinded facet flux) integrated by parts on each cell is
    -int phi div(u (eta-b)) + int_dK phi (u.n)((eta-b)_own - (eta-b)~): the
    same numbers for these polynomial integrands under exact quadrature.
    The library evaluates the strong form (no cancellation between cell and
    facet terms, which both grow like 1/h); the oracle's option gives the
    same values to rounding, and the velocity part is untouched."""
    from oracle.operators import ELEVATION_STRONG, ELEVATION_WEAK
    from tests.conftest import oracle_model
    for r in (2, 3):
        m = oracle_model(r)
        U = _state(m)
        U[m.n_u:] += np.random.default_rng(r).standard_normal(m.n_eta) * 20.0
        a = m.ops.nonlinear_rhs(U)
        m.ops.elevation_form = ELEVATION_STRONG
        b = m.ops.nonlinear_rhs(U)
        m.ops.elevation_form = ELEVATION_WEAK
        assert np.array_equal(a[: m.n_u], b[: m.n_u])
        assert np.abs(a[m.n_u:] - b[m.n_u:]).max() <= 1e-14 * np.abs(a[m.n_u:]).max()
        assert abs(b[m.n_u:].sum()) <= 1e-15 * np.abs(b[m.n_u:]).sum()   # mass conserved in both forms
