"""Quadrature rules for the oracle (test infrastructure only).

The flat-facet discretisation makes every cell integrand of L and N a
polynomial in the reference coordinates (degree <= 5), so any rule exact to
that degree gives the exact integral; the oracle uses a Stroud conical
product rule with 4 x 4 points (exact to degree 7).  On the piecewise cubic
surface the integrands carry 1/det and are not polynomials: the 5 x 5 rule
(exact to degree 9 for polynomials) is then part of the discretisation, and
every implementation has to use it.

The facet rule is different: the upwind choice in N (Sec. 2.5, the definition
of u-tilde) is taken point by point, so the facet integral depends on where
the points are.  The facet rule is therefore part of the method's definition:
Gauss-Legendre on each edge, parametrised from its low to its high vertex,
with 4 points on flat cells and 5 on cubic ones.
"""

import numpy as np
from scipy.special import roots_jacobi, roots_legendre


def gauss_legendre_01(n):
    """n-point Gauss-Legendre on [0, 1]: nodes, weights (weights sum to 1)."""
    x, w = roots_legendre(n)
    return 0.5 * (x + 1.0), 0.5 * w


def triangle_rule(n=4):
    """Stroud conical product rule on the reference triangle (0,0),(1,0),(0,1).

    Collapsed coordinates x = s, y = t (1 - s); Gauss-Jacobi (alpha=1, beta=0)
    in s absorbs the Jacobian (1 - s); Gauss-Legendre in t.  Exact for total
    degree 2n - 1.  Returns points (Q, 2) and weights (Q,) summing to 1/2.
    """
    xs, ws = roots_jacobi(n, 1.0, 0.0)
    s = 0.5 * (xs + 1.0)
    ws = ws / 4.0
    t, wt = gauss_legendre_01(n)
    pts, wts = [], []
    for i in range(n):
        for j in range(n):
            pts.append((s[i], t[j] * (1.0 - s[i])))
            wts.append(ws[i] * wt[j])
    return np.array(pts), np.array(wts)


FACET_POINTS = 4


def cell_rule_points(geometry_degree):
    """Points per direction of the Stroud cell rule: 4 (flat), 5 (cubic)."""
    return 4 if geometry_degree == 1 else 5


def facet_points(geometry_degree):
    """Gauss-Legendre points per facet: 4 (flat), 5 (cubic)."""
    return FACET_POINTS if geometry_degree == 1 else 5
