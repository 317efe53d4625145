"""Reference BDM2 (velocity) and DG1 (elevation) elements (paper Sec. 2.5).

Reference triangle V0 = (0,0), V1 = (1,0), V2 = (0,1).  Local edge i is the
one opposite V_i, traversed counter-clockwise:
  e0: V1 -> V2,  e1: V2 -> V0,  e2: V0 -> V1.

BDM2 = [P2]^2 (dimension 12).  Degrees of freedom (the reading of this build;
the paper uses Firedrake's element, whose DOF functionals it does not print):
  l_{3i+j}(u) = int_0^1 cross2(u(start_i + tau d_i), d_i) p_j(tau) dtau,
      i = local edge, d_i its counter-clockwise direction vector,
      cross2(a, b) = a0 b1 - a1 b0, so cross2(u, d) dtau = u . n_out ds,
      p_0 = 1, p_1 = 2 tau - 1, p_2 = 6 tau^2 - 6 tau + 1 (Legendre on [0,1]);
  l_{9+j}(u) = int_T u . q_j dx,  q_0 = (1,0), q_1 = (0,1), q_2 = (-y, x)
      (moments against the lowest-order Nedelec space of the first kind).
The basis psi_i is dual to these functionals: l_k(psi_i) = delta_ki.

DG1: nodal at the reference vertices, phi_0 = 1 - x - y, phi_1 = x, phi_2 = y.
"""

import numpy as np

from .quadrature import gauss_legendre_01, triangle_rule

EDGE_START = np.array([[1.0, 0.0], [0.0, 1.0], [0.0, 0.0]])
EDGE_DIR = np.array([[-1.0, 1.0], [0.0, -1.0], [1.0, 0.0]])


def legendre01(j, tau):
    if j == 0:
        return np.ones_like(tau)
    if j == 1:
        return 2.0 * tau - 1.0
    return 6.0 * tau * tau - 6.0 * tau + 1.0


def _monomials(xi):
    """Scalar P2 monomials [1, x, y, x^2, xy, y^2] at points (Q, 2) -> (Q, 6)."""
    x, y = xi[:, 0], xi[:, 1]
    return np.stack([np.ones_like(x), x, y, x * x, x * y, y * y], axis=1)


def _monomial_grads(xi):
    """d/dx and d/dy of the monomials -> (Q, 6, 2)."""
    x, y = xi[:, 0], xi[:, 1]
    z, o = np.zeros_like(x), np.ones_like(x)
    dx = np.stack([z, o, z, 2 * x, y, z], axis=1)
    dy = np.stack([z, z, o, z, x, 2 * y], axis=1)
    return np.stack([dx, dy], axis=2)


def _vector_monomials(xi):
    """The 12 vector monomials m_{6c+p} = e_c * mono_p at points -> (Q, 12, 2)."""
    m = _monomials(xi)
    Q = len(xi)
    out = np.zeros((Q, 12, 2))
    out[:, 0:6, 0] = m
    out[:, 6:12, 1] = m
    return out


def _dof_functionals(fields):
    """Apply the 12 DOF functionals to a callable field(xi) -> (Q, K, 2). Returns (12, K)."""
    tau, wt = gauss_legendre_01(6)
    rows = []
    for i in range(3):
        pts = EDGE_START[i][None, :] + tau[:, None] * EDGE_DIR[i][None, :]
        v = fields(pts)                                     # (Q, K, 2)
        flux = v[:, :, 0] * EDGE_DIR[i][1] - v[:, :, 1] * EDGE_DIR[i][0]
        for j in range(3):
            rows.append(np.einsum("q,qk->k", wt * legendre01(j, tau), flux))
    xq, wq = triangle_rule(6)
    v = fields(xq)
    qf = [np.stack([np.ones(len(xq)), np.zeros(len(xq))], 1),
          np.stack([np.zeros(len(xq)), np.ones(len(xq))], 1),
          np.stack([-xq[:, 1], xq[:, 0]], 1)]
    for j in range(3):
        rows.append(np.einsum("q,qkc,qc->k", wq, v, qf[j]))
    return np.array(rows)


def _exact_vandermonde():
    """V[k][l] = l_k(m_l) in exact rational arithmetic.

    Along edge i, x = sx + tau dx and y = sy + tau dy with integer start and
    direction, so a monomial is a polynomial in tau with integer coefficients
    and int_0^1 tau^k dtau = 1/(k+1); over the triangle,
    int x^a y^b = a! b! / (a + b + 2)!."""
    from fractions import Fraction
    from math import factorial

    def mul(a, b):
        r = [0] * (len(a) + len(b) - 1)
        for i, x in enumerate(a):
            for j, y in enumerate(b):
                r[i + j] += x * y
        return r

    def power(p, n):
        r = [1]
        for _ in range(n):
            r = mul(r, p)
        return r

    powers = [(0, 0), (1, 0), (0, 1), (2, 0), (1, 1), (0, 2)]      # the scalar monomials' (a, b)
    legendre = [[1], [-1, 2], [1, -6, 6]]                           # p_j in powers of tau
    V = [[Fraction(0)] * 12 for _ in range(12)]
    for i in range(3):
        sx, sy = (int(v) for v in EDGE_START[i])
        dx, dy = (int(v) for v in EDGE_DIR[i])
        for j in range(3):
            for l in range(12):
                a, b = powers[l % 6]
                m = mul(power([sx, dx], a), power([sy, dy], b))
                flux = [c * (dy if l < 6 else -dx) for c in m]  # cross2(m_l, d_i)
                V[3 * i + j][l] = sum(Fraction(c, k + 1) for k, c in enumerate(mul(flux, legendre[j])))

    def tri(a, b):
        return Fraction(factorial(a) * factorial(b), factorial(a + b + 2))

    for l in range(12):
        a, b = powers[l % 6]
        V[9][l] = tri(a, b) if l < 6 else Fraction(0)               # q_0 = (1, 0)
        V[10][l] = tri(a, b) if l >= 6 else Fraction(0)             # q_1 = (0, 1)
        V[11][l] = -tri(a, b + 1) if l < 6 else tri(a + 1, b)       # q_2 = (-y, x)
    return V


def _exact_inverse(V):
    """Gauss-Jordan elimination in exact rational arithmetic."""
    from fractions import Fraction
    n = len(V)
    A = [list(row) + [Fraction(int(i == k)) for k in range(n)] for i, row in enumerate(V)]
    for col in range(n):
        piv = next(r for r in range(col, n) if A[r][col] != 0)
        A[col], A[piv] = A[piv], A[col]
        pv = A[col][col]
        A[col] = [x / pv for x in A[col]]
        for r in range(n):
            if r != col and A[r][col] != 0:
                f = A[r][col]
                A[r] = [x - f * y for x, y in zip(A[r], A[col])]
    return [row[n:] for row in A]


class BDM2:
    """Reference BDM2 basis as coefficients over the vector monomials.

    The basis is dual to the DOF functionals, l_k(psi_i) = delta_ki: the
    coefficients are the inverse of V[k][l] = l_k(m_l), computed exactly in
    rational arithmetic (it has integer entries) so that the basis carries no
    rounding from an inversion of the moderately conditioned V (cond ~ 530)."""

    def __init__(self):
        Vq = _exact_vandermonde()
        self.vandermonde = np.array([[float(x) for x in row] for row in Vq])
        self.coeffs = np.array([[float(x) for x in row] for row in _exact_inverse(Vq)])  # psi_i = sum_l coeffs[l, i] m_l

    def values(self, xi):
        """psi_i(xi) -> (Q, 12, 2)."""
        return np.einsum("qlc,li->qic", _vector_monomials(np.atleast_2d(xi)), self.coeffs)

    def grads(self, xi):
        """d psi_i[c] / d xi[a] -> (Q, 12, 2 (c), 2 (a))."""
        g = _monomial_grads(np.atleast_2d(xi))               # (Q, 6, 2)
        Q = g.shape[0]
        gm = np.zeros((Q, 12, 2, 2))
        gm[:, 0:6, 0, :] = g
        gm[:, 6:12, 1, :] = g
        return np.einsum("qlca,li->qica", gm, self.coeffs)

    def divs(self, xi):
        g = self.grads(xi)
        return g[:, :, 0, 0] + g[:, :, 1, 1]

    def dofs_of(self, field):
        """Apply the DOF functionals to field(xi) -> (Q, 2). Returns (12,)."""
        return _dof_functionals(lambda x: field(x)[:, None, :])[:, 0]


def dg1_values(xi):
    xi = np.atleast_2d(xi)
    x, y = xi[:, 0], xi[:, 1]
    return np.stack([1.0 - x - y, x, y], axis=1)


DG1_GRADS = np.array([[-1.0, -1.0], [1.0, 0.0], [0.0, 1.0]])
