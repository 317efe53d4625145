"""Cell geometry, element matrices and global sparse matrices (paper Sec. 2.5).

Geometry (oracle/geometry.py): degree 1, flat triangles through the mesh
vertices, or degree 3, the piecewise cubic surface of Sec. 3.  At every
quadrature point of a cell, with J = dx/dxi (3 x 2), det = |J0 x J1|,
G = J^T J and k = (J0 x J1) / det (outward unit normal; cells are
counter-clockwise):
Contravariant Piola map: u = J u_hat / det, div u = div_hat u_hat / det.
Pointwise identities (hold on curved cells too, J and det taken at the point):
  (k x J a) . (J b) = det * cross2(a, b)
  grad_perp q := k x grad q = J curl_hat(q) / det,  curl_hat q = (-dq/dy, dq/dx)
so that, with dA = det dA_hat,
  M1_ij = int_ref psi_i . G psi_j / det,   M2_ij = int_ref phi_i phi_j det,
  C_ij  = int_ref f cross2(psi_j, psi_i),  D_ij  = int_ref phi_i div_hat psi_j
(D does not depend on the geometry).  On flat cells every integrand is a
polynomial and the 4 x 4 cell rule integrates it exactly; on cubic cells the
integrands are rational and the 5 x 5 rule is part of the discretisation.
The attributes a, J, det, G, k are the flat (vertex) triangle's, for both
degrees (cell-size features; the degree-1 geometry).

Global numbering (the reading of this build):
  velocity: edge e, moment j -> 3 e + j;  interior DOF j of cell c -> 3 E + 3 c + j
  elevation: local vertex i of cell c -> 3 c + i
Edge DOFs are the moments of the flux across the edge towards the side of
(t_e x k), t_e the edge's low -> high tangent.  Relative to a cell's local
(counter-clockwise) edge DOFs this is the identity when the cell traverses
the edge low -> high, and a factor (-1)^(j+1) otherwise.
"""

import numpy as np
import scipy.sparse as sp

from .elements import BDM2, DG1_GRADS, dg1_values
from .geometry import CellMaps
from .quadrature import cell_rule_points, triangle_rule


def cross2(a, b):
    return a[..., 0] * b[..., 1] - a[..., 1] * b[..., 0]


class Assembly:
    def __init__(self, mesh, omega, radius, geometry_degree=1):
        self.mesh = mesh
        self.degree = geometry_degree
        self.maps = CellMaps(mesh, geometry_degree)
        self.cell_n = cell_rule_points(geometry_degree)
        self.element = BDM2()
        F, E = mesh.n_cells, mesh.n_edges
        self.n_u = 3 * E + 3 * F
        self.n_eta = 3 * F
        P = mesh.verts[mesh.cells]                           # (F, 3, 3)
        self.a = P[:, 0]
        J0 = P[:, 1] - P[:, 0]
        J1 = P[:, 2] - P[:, 0]
        self.J = np.stack([J0, J1], axis=2)                 # (F, 3, 2)
        cr = np.cross(J0, J1)
        self.det = np.linalg.norm(cr, axis=1)
        self.k = cr / self.det[:, None]
        self.G = np.einsum("fxa,fxb->fab", self.J, self.J)  # (F, 2, 2)
        # signs and global indices of the 12 local velocity DOFs
        sign = np.ones((F, 12))
        dofs = np.zeros((F, 12), dtype=np.int64)
        for i in range(3):
            for j in range(3):
                aligned = mesh.cell_edge_aligned[:, i]
                sign[:, 3 * i + j] = np.where(aligned, 1.0, (-1.0) ** (j + 1))
                dofs[:, 3 * i + j] = 3 * mesh.cell_edges[:, i] + j
        for j in range(3):
            dofs[:, 9 + j] = 3 * E + 3 * np.arange(F) + j
        self.sign = sign
        self.udofs = dofs
        self.etadofs = 3 * np.arange(F)[:, None] + np.arange(3)[None, :]
        self.omega = float(omega)
        self.radius = float(radius)
        self._element_matrices()

    def coriolis(self, xi):
        """f = 2 Omega z / R at reference points xi (Q, 2) of every cell -> (F, Q),
        z the third coordinate of the cell map's point."""
        return 2.0 * self.omega * self.maps.points(xi)[..., 2] / self.radius

    def _element_matrices(self):
        xq, wq = triangle_rule(self.cell_n)
        psi = self.element.values(xq)                       # (Q, 12, 2)
        div = self.element.divs(xq)                         # (Q, 12)
        phi = dg1_values(xq)                                # (Q, 3)
        f = self.coriolis(xq)                               # (F, Q)
        geo = self.maps.geometry(xq)
        Gd = geo["G"] / geo["det"][..., None, None]         # (F, Q, 2, 2)
        m1 = np.einsum("q,qia,fqab,qjb->fij", wq, psi, Gd, psi)
        # C_ij = int w_i . f (k x w_j) dx = int_ref f cross2(psi_j, psi_i)
        cr = psi[:, None, :, 0] * psi[:, :, None, 1] - psi[:, None, :, 1] * psi[:, :, None, 0]  # (Q, i, j) = cross2(psi_j, psi_i)
        c = np.einsum("q,fq,qij->fij", wq, f, cr)
        d = np.einsum("q,qi,qj->ij", wq, phi, div)          # (3, 12) reference
        m2 = np.einsum("q,fq,qi,qj->fij", wq, geo["det"], phi, phi)
        S = self.sign
        self.M1_e = S[:, :, None] * m1 * S[:, None, :]
        self.C_e = S[:, :, None] * c * S[:, None, :]
        self.D_e = d[None, :, :] * S[:, None, :]
        self.M2_e = m2

    def global_matrices(self):
        F = self.mesh.n_cells
        ii = np.repeat(self.udofs[:, :, None], 12, axis=2)
        jj = np.repeat(self.udofs[:, None, :], 12, axis=1)
        M1 = sp.coo_matrix((self.M1_e.ravel(), (ii.ravel(), jj.ravel())), shape=(self.n_u, self.n_u)).tocsr()
        C = sp.coo_matrix((self.C_e.ravel(), (ii.ravel(), jj.ravel())), shape=(self.n_u, self.n_u)).tocsr()
        ei = np.repeat(self.etadofs[:, :, None], 12, axis=2)
        uj = np.repeat(self.udofs[:, None, :], 3, axis=1)
        D = sp.coo_matrix((self.D_e.ravel(), (ei.ravel(), uj.ravel())), shape=(self.n_eta, self.n_u)).tocsr()
        e2i = np.repeat(self.etadofs[:, :, None], 3, axis=2)
        e2j = np.repeat(self.etadofs[:, None, :], 3, axis=1)
        M2 = sp.coo_matrix((self.M2_e.ravel(), (e2i.ravel(), e2j.ravel())), shape=(self.n_eta, self.n_eta)).tocsr()
        assert F * 3 == self.n_eta
        return M1, C, D, M2


DG1_GRAD = DG1_GRADS
