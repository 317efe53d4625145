"""Cell maps of the icosahedral mesh (paper Sec. 3: the sphere is approximated
by a piecewise cubic surface; degree 1 is the flat-facet reading).

Degree d in {1, 3}.  Each cell's map x(xi) from the reference triangle
(0,0), (1,0), (0,1) is the degree-d Lagrange interpolant of its nodes:
reference node (i/d, j/d), i + j <= d, is sent to the point with barycentric
coordinates (1 - i/d - j/d, i/d, j/d) of the flat triangle (v0, v1, v2),
projected radially onto the sphere of radius R.  For d = 1 the nodes are the
vertices and x is affine; for d = 3 the two nodes on an edge depend only on
its end points, so neighbouring cells share their common edge curve.

The Lagrange basis is written over the monomials xi0^p xi1^q (p + q <= d);
its coefficients are the inverse of the nodes' Vandermonde matrix, which has
rational entries and is inverted exactly.  At reference points the module
returns, per cell and point,
  J = dx/dxi (3 x 2), det = |J0 x J1|, G = J^T J, k = J0 x J1 / det,
  grad_det[a] = d det / d xi_a = k . (d_a J0 x J1 + J0 x d_a J1).
Test infrastructure only (see oracle/__init__.py).
"""

from fractions import Fraction

import numpy as np

from .elements import _exact_inverse


def _powers(d):
    return [(p, q) for s in range(d + 1) for q in range(s + 1) for p in [s - q]]


def reference_nodes(d):
    """Reference coordinates of the degree-d nodes: (i/d, j/d), j-major."""
    return [(Fraction(i, d), Fraction(j, d)) for j in range(d + 1) for i in range(d + 1 - j)]


def _mono(xi, powers, dx=0, dy=0):
    """d^dx/dxi0^dx d^dy/dxi1^dy of every monomial at points xi (Q, 2) -> (Q, n)."""
    out = np.zeros((len(xi), len(powers)))
    for m, (p, q) in enumerate(powers):
        if p < dx or q < dy:
            continue
        cp = np.prod(np.arange(p - dx + 1, p + 1)) if dx else 1.0
        cq = np.prod(np.arange(q - dy + 1, q + 1)) if dy else 1.0
        out[:, m] = cp * cq * xi[:, 0] ** (p - dx) * xi[:, 1] ** (q - dy)
    return out


class CellMaps:
    def __init__(self, mesh, degree):
        if degree not in (1, 3):
            raise ValueError("geometry degree must be 1 or 3")
        self.degree = degree
        self.radius = mesh.radius
        self.powers = _powers(degree)
        nodes = reference_nodes(degree)
        V = [[x ** p * y ** q for (p, q) in self.powers] for (x, y) in nodes]
        A = np.array([[float(v) for v in row] for row in _exact_inverse(V)])   # N_a = sum_m A[m, a] mono_m
        v = mesh.verts[mesh.cells]                                              # (F, 3, 3)
        lam = np.array([[1.0 - float(x) - float(y), float(x), float(y)] for (x, y) in nodes])
        X = np.einsum("al,flx->fax", lam, v)                                    # flat positions of the nodes
        if degree > 1:
            X = X * (self.radius / np.linalg.norm(X, axis=2))[:, :, None]
        self.nodes = X                                                          # (F, n, 3)
        self.P = np.einsum("ma,fax->fmx", A, X)                                 # monomial coefficients (F, n, 3)

    def points(self, xi):
        return np.einsum("qm,fmx->fqx", _mono(xi, self.powers), self.P)

    def jacobian(self, xi):
        d0 = np.einsum("qm,fmx->fqx", _mono(xi, self.powers, 1, 0), self.P)
        d1 = np.einsum("qm,fmx->fqx", _mono(xi, self.powers, 0, 1), self.P)
        return np.stack([d0, d1], axis=3)                                       # (F, Q, 3, 2)

    def second_derivatives(self, xi):
        """H[..., a, b] = d^2 x / dxi_a dxi_b -> (F, Q, 3, 2, 2)."""
        h00 = np.einsum("qm,fmx->fqx", _mono(xi, self.powers, 2, 0), self.P)
        h01 = np.einsum("qm,fmx->fqx", _mono(xi, self.powers, 1, 1), self.P)
        h11 = np.einsum("qm,fmx->fqx", _mono(xi, self.powers, 0, 2), self.P)
        return np.stack([np.stack([h00, h01], axis=3), np.stack([h01, h11], axis=3)], axis=4)

    def geometry(self, xi):
        """dict of J, det, G, k, grad_det at reference points xi (Q, 2)."""
        J = self.jacobian(xi)
        J0, J1 = J[..., 0], J[..., 1]
        cr = np.cross(J0, J1)
        det = np.linalg.norm(cr, axis=-1)
        k = cr / det[..., None]
        G = np.einsum("fqxa,fqxb->fqab", J, J)
        H = self.second_derivatives(xi)
        gd = np.stack([np.einsum("fqx,fqx->fq", k, np.cross(H[..., 0, a], J1) + np.cross(J0, H[..., 1, a]))
                       for a in range(2)], axis=-1)                              # d_a J_b = H[..., b, a]
        return {"J": J, "det": det, "G": G, "k": k, "grad_det": gd}
