"""Pins of the oracle's BDM2 / DG1 elements and assembly (paper Sec. 2.5)."""

import numpy as np
import pytest

from oracle.assembly import Assembly
from oracle.elements import BDM2, EDGE_DIR, EDGE_START, dg1_values
from oracle.mesh import build_mesh
from oracle.quadrature import gauss_legendre_01, triangle_rule

R = 6.37122e6


def test_quadrature_exactness():
    # int_T x^a y^b = a! b! / (a + b + 2)!
    from math import factorial
    x, w = triangle_rule(4)
    for a in range(8):
        for b in range(8 - a):
            exact = factorial(a) * factorial(b) / factorial(a + b + 2)
            assert abs((w * x[:, 0] ** a * x[:, 1] ** b).sum() - exact) < 1e-15
    t, wt = gauss_legendre_01(4)
    for k in range(8):
        assert abs((wt * t ** k).sum() - 1.0 / (k + 1)) < 1e-15


def test_bdm2_dofs_of_closed_form_fields():
    """DOF functionals on fields whose moments are known in closed form."""
    el = BDM2()
    # constant field (1, 0): flux through e0 (d = (-1, 1)) is cross2((1,0), d) = 1,
    # through e1 (d = (0, -1)) is -1, through e2 (d = (1, 0)) is 0; interior
    # moments are area * (1, 0, centroid-weighted -y) = (1/2, 0, -1/6).
    dofs = el.dofs_of(lambda x: np.tile([1.0, 0.0], (len(x), 1)))
    want = np.array([1, 0, 0, -1, 0, 0, 0, 0, 0, 0.5, 0.0, -1.0 / 6.0])
    assert np.abs(dofs - want).max() < 1e-15
    # radial field (x, y): zero flux through e1, e2; flux 1 through e0 with
    # u . n ds constant; interior: (1/6, 1/6, 0)
    dofs = el.dofs_of(lambda x: x.copy())
    want = np.array([1, 0, 0, 0, 0, 0, 0, 0, 0, 1 / 6.0, 1 / 6.0, 0.0])
    assert np.abs(dofs - want).max() < 1e-15


def test_bdm2_reproduces_p2_fields():
    """Interpolating any [P2]^2 field and evaluating the interpolant returns it."""
    el = BDM2()
    rng = np.random.default_rng(1)
    C = rng.standard_normal((2, 6))

    def field(x):
        m = np.stack([np.ones(len(x)), x[:, 0], x[:, 1], x[:, 0] ** 2, x[:, 0] * x[:, 1], x[:, 1] ** 2], 1)
        return m @ C.T

    d = el.dofs_of(field)
    pts = rng.random((20, 2)) * 0.5
    got = np.einsum("i,qic->qc", d, el.values(pts))
    assert np.abs(got - field(pts)).max() < 1e-12


def test_bdm2_edge_flux_support():
    """The normal trace of edge basis functions vanishes on the other edges, and
    interior functions have zero normal trace everywhere."""
    el = BDM2()
    tau, _ = gauss_legendre_01(5)
    for i in range(3):
        pts = EDGE_START[i] + tau[:, None] * EDGE_DIR[i]
        v = el.values(pts)
        flux = v[:, :, 0] * EDGE_DIR[i][1] - v[:, :, 1] * EDGE_DIR[i][0]
        for k in range(12):
            if k // 3 != i:
                assert np.abs(flux[:, k]).max() < 1e-12


@pytest.mark.parametrize("r", [1, 2])
def test_hdiv_conformity_across_edges(r):
    """Normal flux of every global edge basis function agrees from both cells.

    The physical flux density u . nu (nu = t x k on each side) is evaluated on
    the shared edge from the plus and the minus cell at the same physical points.
    """
    m = build_mesh(r, R)
    A = Assembly(m, 7.292e-5, R)
    el = A.element
    tau, _ = gauss_legendre_01(5)
    for e in range(0, m.n_edges, max(1, m.n_edges // 40)):
        lo, hi = m.verts[m.edges[e]]
        t = (hi - lo) / np.linalg.norm(hi - lo)
        vals = []
        for side in (0, 1):
            c, i = m.edge_cells[e, side], m.edge_local[e, side]
            s = tau if side == 0 else 1.0 - tau
            xi = EDGE_START[i] + s[:, None] * EDGE_DIR[i]
            x = A.a[c] + xi @ A.J[c].T
            assert np.abs(x - (lo + tau[:, None] * (hi - lo))).max() < 1e-6
            nu = np.cross(t, A.k[c])
            w = np.einsum("xa,qia->qix", A.J[c], el.values(xi)) / A.det[c]
            w = w * A.sign[c][None, :, None]
            flux = np.einsum("qix,x->qi", w, nu)
            full = np.zeros((len(tau), 3 * m.n_edges))
            for k in range(9):
                full[:, A.udofs[c, k]] = flux[:, k]
            vals.append(full[:, 3 * e: 3 * e + 3])
        assert np.abs(vals[0] - vals[1]).max() < 1e-12 * np.abs(vals[0]).max()


@pytest.mark.parametrize("r", [1, 3])
def test_divergence_of_global_basis_integrates_to_zero(r):
    """sum_K int_K div w = 0 for every global basis function (closed surface),
    i.e. D^T 1 = 0; the interior functions also satisfy it per cell."""
    m = build_mesh(r, R)
    A = Assembly(m, 7.292e-5, R)
    _, _, D, M2 = A.global_matrices()
    ones = np.ones(A.n_eta)
    s = D.T @ ones
    assert np.abs(s).max() < 1e-13


def test_dg1_mass_is_cell_area():
    m = build_mesh(2, R)
    A = Assembly(m, 7.292e-5, R)
    _, _, _, M2 = A.global_matrices()
    P = m.verts[m.cells]
    area = 0.5 * np.linalg.norm(np.cross(P[:, 1] - P[:, 0], P[:, 2] - P[:, 0]), axis=1).sum()
    assert abs(M2.sum() / area - 1) < 1e-14
    # dg1 partition of unity
    assert np.abs(dg1_values(np.random.default_rng(0).random((7, 2))).sum(axis=1) - 1).max() < 1e-15


def test_mass_matrix_spd_and_velocity_mass_closed_form():
    """M1 is symmetric positive definite, and the mass of a constant-in-cell
    field integrates exactly: for the interpolant of a field that is constant
    on the reference cell, the element mass equals |J u_hat|^2 / det."""
    m = build_mesh(1, R)
    A = Assembly(m, 7.292e-5, R)
    M1, C, D, M2 = A.global_matrices()
    dense = M1.toarray()
    assert np.abs(dense - dense.T).max() < 1e-12 * np.abs(dense).max()
    assert np.linalg.eigvalsh(dense).min() > 0
    assert np.abs(C + C.T).max() == 0.0
    el = A.element
    d = el.dofs_of(lambda x: np.tile([0.3, -0.7], (len(x), 1)))
    uh = np.array([0.3, -0.7])
    for c in range(3):
        e = d @ (A.M1_e[c] * np.outer(A.sign[c], A.sign[c])) @ d
        want = uh @ A.G[c] @ uh / A.det[c] * 0.5
        assert abs(e / want - 1) < 1e-13


def test_dual_basis_is_exact():
    """The BDM2 basis is dual to the DOF functionals (l_k(psi_i) = delta_ki).
    Its coefficients come from an exact rational inverse of V; they are
    integers, V times them is the identity without rounding, the exact V
    equals the functionals applied by quadrature, and a floating-point
    inverse of the quadrature V agrees to its own rounding (cond(V) ~ 530)."""
    from oracle.elements import BDM2, _dof_functionals, _vector_monomials
    b = BDM2()
    C = b.coeffs
    assert np.array_equal(C, np.round(C)) and np.abs(C).max() == 120.0
    assert np.abs(b.vandermonde @ C - np.eye(12)).max() <= 1e-13  # V rounded to doubles (1/3, 1/60, ...)
    Vq = _dof_functionals(_vector_monomials)
    assert np.abs(b.vandermonde - Vq).max() <= 1e-15
    assert np.abs(np.linalg.inv(Vq) - C).max() <= 1e-11
