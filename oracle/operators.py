"""Discrete linear operator L and nonlinear operator N (paper Sec. 2.5).

L(u, eta) = (u1, eta1) with (Eq. ueq_int and the eta equation after it)
    M1 u1   = -C u + g D^T eta,      C_ij = int w_i . f (k x w_j),
    M2 eta1 = -H D u,                D_ij = int phi_i div w_j.

N(u, eta) = (u2, eta2) with (the two weak forms following Eq. ueq_int)
    int w . u2   = int u . grad_perp(u_perp . w) - int_Gamma [[n_perp (u_perp . w)]] . u~
                   + int div w (|u|^2 / 2)
    int phi eta2 = int grad phi . u (eta - b) - int_Gamma [[phi u]] (eta - b)~
Readings (the printed facet terms are garbled, so these are this
implementation's choices):
  * [[n_perp q]] = t (q+ - q-) with t the edge's low -> high unit tangent;
  * the elevation facet term carries a minus sign (integration by parts with
    outward normals) and the upwind value of (eta - b);
  * the upwind side is the one the flow leaves: + when u+ . n+ > 0, else -
    ("standard"); the printed rule (+ when u . n+ < 0) is kept as the
    "as_printed" option for the velocity term;
  * the flux u . n+ is evaluated from the + side for both cells, so the
    elevation flux is single-valued and mass is conserved exactly;
  * the + cell of an edge is the one whose counter-clockwise boundary runs
    low -> high along it.
All facet integrals use the Gauss-Legendre rule on [0, 1] (4 points on flat
cells, 5 on cubic ones), tau = 0 at the low vertex; the upwind choice is made
point by point.

Cell integrand, in reference form at each quadrature point (J, det, G = J^T J
and grad_hat det taken at the point; u_hat the pulled-back velocity, psi_i the
reference test function, q_i = cross2(u_hat, psi_i) / det = u_perp . w_i):
  u . grad_perp q_i dA = (G u_hat) . curl_hat(q_i) / det dA_hat
                       = [d_tau cross2(u_hat, psi_i) - cross2(u_hat, psi_i) d_tau det / det] / det^2,
  div w_i |u|^2 / 2 dA = div_hat psi_i (u_hat . G u_hat) / (2 det^2) dA_hat,
with d_tau = (G u_hat)_1 d/dxi0 - (G u_hat)_0 d/dxi1.  The d_tau det term
vanishes on flat cells.  On a facet, each side uses its own J and det at the
point: t . u |dx/dtau| = d . G u_hat / det for the reference edge direction
d, and u . n ds = cross2(u_hat, d) dtau (the Piola map preserves fluxes).
"""

import numpy as np
import scipy.sparse.linalg as spla

from .assembly import Assembly, cross2
from .elements import DG1_GRADS, EDGE_DIR, EDGE_START, dg1_values
from .quadrature import facet_points, gauss_legendre_01, triangle_rule

UPWIND_STANDARD = 0
UPWIND_AS_PRINTED = 1


ELEVATION_WEAK = 0
ELEVATION_STRONG = 1


class Operators:
    def __init__(self, mesh, g, H, omega, radius, upwind=UPWIND_STANDARD, elevation_form=ELEVATION_WEAK,
                 geometry_degree=1):
        self.mesh = mesh
        self.asm = Assembly(mesh, omega, radius, geometry_degree)
        self.g = float(g)
        self.H = float(H)
        self.upwind = upwind
        self.elevation_form = elevation_form
        self.n_u = self.asm.n_u
        self.n_eta = self.asm.n_eta
        self.n = self.n_u + self.n_eta
        self.M1, self.C, self.D, self.M2 = self.asm.global_matrices()
        self._M1_lu = spla.splu(self.M1.tocsc())
        self._M2_lu = spla.splu(self.M2.tocsc())
        self.b = np.zeros(self.n_eta)

    # ------------------------------------------------------------------ basics
    def split(self, U):
        return U[: self.n_u], U[self.n_u:]

    def solve_M1(self, r):
        return self._M1_lu.solve(r)

    def solve_M2(self, r):
        return self._M2_lu.solve(r)

    def mass_solve(self, R):
        ru, re = self.split(R)
        return np.concatenate([self.solve_M1(ru), self.solve_M2(re)])

    def set_topography(self, b):
        self.b = np.array(b, dtype=np.float64)

    # ------------------------------------------------------------------ L
    def linear_rhs(self, U):
        """The weak-form right-hand sides (-C u + g D^T eta, -H D u)."""
        u, eta = self.split(U)
        return np.concatenate([-(self.C @ u) + self.g * (self.D.T @ eta), -self.H * (self.D @ u)])

    def L(self, U):
        return self.mass_solve(self.linear_rhs(U))

    # ------------------------------------------------------------------ N
    def nonlinear_rhs(self, U):
        """Weak-form right-hand sides of N (before the mass solves)."""
        A = self.asm
        el = A.element
        u, eta = self.split(U)
        F = self.mesh.n_cells
        c = A.sign * u[A.udofs]                                  # (F, 12) local coefficients
        h = eta[A.etadofs] - self.b[A.etadofs]                   # (F, 3)
        # ---- cell integrals
        xq, wq = triangle_rule(A.cell_n)
        geo = A.maps.geometry(xq)
        G, det, gdet = geo["G"], geo["det"], geo["grad_det"]    # (F, Q, 2, 2), (F, Q), (F, Q, 2)
        psi = el.values(xq)                                      # (Q, 12, 2)
        dpsi = el.grads(xq)                                      # (Q, 12, 2c, 2a)
        divpsi = el.divs(xq)                                     # (Q, 12)
        phi = dg1_values(xq)                                     # (Q, 3)
        uh = np.einsum("fj,qjc->fqc", c, psi)                    # (F, Q, 2)
        duh = np.einsum("fj,qjca->fqca", c, dpsi)                # (F, Q, 2, 2)
        hh = np.einsum("fk,qk->fq", h, phi)                      # (F, Q)
        Guh = np.einsum("fqab,fqb->fqa", G, uh)                  # (F, Q, 2)
        # q_i = cross2(uh, psi_i);  d q_i / d xi_a = cross2(d_a uh, psi_i) + cross2(uh, d_a psi_i)
        dq = np.zeros((F, len(wq), 12, 2))
        for a_ in range(2):
            dq[..., a_] = (duh[:, :, None, 0, a_] * psi[None, :, :, 1] - duh[:, :, None, 1, a_] * psi[None, :, :, 0]
                           + uh[:, :, None, 0] * dpsi[None, :, :, 1, a_] - uh[:, :, None, 1] * dpsi[None, :, :, 0, a_])
        curl_q = np.stack([-dq[..., 1], dq[..., 0]], axis=-1)   # (F, Q, 12, 2)
        q0 = cross2(uh[:, :, None, :], psi[None])                # (F, Q, 12)
        dtau_det = Guh[..., 1] * gdet[..., 0] - Guh[..., 0] * gdet[..., 1]
        integrand = np.einsum("fqa,fqia->fqi", Guh, curl_q) - q0 * (dtau_det / det)[..., None]
        vort = np.einsum("q,fq,fqi->fi", wq, 1.0 / det ** 2, integrand)
        ke = 0.5 * np.einsum("fqa,fqa->fq", uh, Guh)             # det^2 |u|^2 / 2
        kin = np.einsum("q,qi,fq->fi", wq, divpsi, ke / det ** 2)
        ru = vort + kin
        strong = self.elevation_form == ELEVATION_STRONG
        if strong:
            # -int phi_i div(u h) = -int_ref phi_i (h div_hat u_hat + u_hat . grad_hat h)
            divu = np.einsum("fj,qj->fq", c, divpsi)
            gradh = np.einsum("fk,ka->fa", h, DG1_GRADS)               # DG1: constant per cell
            g_ = hh * divu + np.einsum("fqa,fa->fq", uh, gradh)
            re = -np.einsum("q,qi,fq->fi", wq, phi, g_)
        else:
            re = np.einsum("q,ia,fqa,fq->fi", wq, DG1_GRADS, uh, hh)
        # ---- facet integrals
        tau, wt = gauss_legendre_01(facet_points(A.degree))
        cp, cm = self.mesh.edge_cells[:, 0], self.mesh.edge_cells[:, 1]
        ip, im = self.mesh.edge_local[:, 0], self.mesh.edge_local[:, 1]
        xp = EDGE_START[ip][:, None, :] + tau[None, :, None] * EDGE_DIR[ip][:, None, :]            # (E, P, 2)
        xm = EDGE_START[im][:, None, :] + (1.0 - tau)[None, :, None] * EDGE_DIR[im][:, None, :]
        # each side's geometry at the facet points: evaluate every cell on each
        # of its three edges (both parametrisations), then pick the edge's cells
        gp = [A.maps.geometry(EDGE_START[i][None, :] + tau[:, None] * EDGE_DIR[i][None, :]) for i in range(3)]
        gm = [A.maps.geometry(EDGE_START[i][None, :] + (1.0 - tau)[:, None] * EDGE_DIR[i][None, :]) for i in range(3)]
        Gp = np.stack([g["G"] for g in gp])[ip, cp]              # (E, P, 2, 2)
        Gm = np.stack([g["G"] for g in gm])[im, cm]
        detp = np.stack([g["det"] for g in gp])[ip, cp]          # (E, P)
        detm = np.stack([g["det"] for g in gm])[im, cm]
        E, P = xp.shape[0], xp.shape[1]
        psip = el.values(xp.reshape(-1, 2)).reshape(E, P, 12, 2)
        psim = el.values(xm.reshape(-1, 2)).reshape(E, P, 12, 2)
        phip = dg1_values(xp.reshape(-1, 2)).reshape(E, P, 3)
        phim = dg1_values(xm.reshape(-1, 2)).reshape(E, P, 3)
        up = np.einsum("ej,epjc->epc", c[cp], psip)
        um = np.einsum("ej,epjc->epc", c[cm], psim)
        hp = np.einsum("ek,epk->ep", h[cp], phip)
        hm = np.einsum("ek,epk->ep", h[cm], phim)
        dp = EDGE_DIR[ip][:, None, :]                            # (E, 1, 2)
        dm = EDGE_DIR[im][:, None, :]
        flux = cross2(up, dp)                                    # u+ . n+ ds / dtau
        plus_up = flux > 0.0
        plus_up_vel = plus_up if self.upwind == UPWIND_STANDARD else (flux < 0.0)
        tan_p = np.einsum("epa,epab,epb->ep", np.broadcast_to(dp, up.shape), Gp, up) / detp
        tan_m = -np.einsum("epa,epab,epb->ep", np.broadcast_to(dm, um.shape), Gm, um) / detm
        tan = np.where(plus_up_vel, tan_p, tan_m)               # |e| (t . u~)
        h_up = np.where(plus_up, hp, hm)
        qp = cross2(up[:, :, None, :], psip) / detp[:, :, None]           # (E, P, 12)
        qm = cross2(um[:, :, None, :], psim) / detm[:, :, None]
        fp = -np.einsum("p,epi,ep->ei", wt, qp, tan)
        fm = np.einsum("p,epi,ep->ei", wt, qm, tan)
        if strong:   # int_dK phi (h_own - h~) u . n_out, u . n_out = +flux (plus cell), -flux (minus cell)
            gp = np.einsum("p,epi,ep->ei", wt, phip, flux * (hp - h_up))
            gm = np.einsum("p,epi,ep->ei", wt, phim, flux * (h_up - hm))
        else:
            gp = -np.einsum("p,epi,ep->ei", wt, phip, flux * h_up)
            gm = np.einsum("p,epi,ep->ei", wt, phim, flux * h_up)
        np.add.at(ru, cp, fp)
        np.add.at(ru, cm, fm)
        np.add.at(re, cp, gp)
        np.add.at(re, cm, gm)
        # ---- to global numbering
        r_u = np.zeros(self.n_u)
        np.add.at(r_u, A.udofs.ravel(), (A.sign * ru).ravel())
        r_eta = np.zeros(self.n_eta)
        r_eta[A.etadofs.ravel()] = re.ravel()
        return np.concatenate([r_u, r_eta])

    def N(self, U):
        return self.mass_solve(self.nonlinear_rhs(U))

    # ------------------------------------------------------------------ diagnostics
    def energy(self, U):
        """E = (H u^T M1 u + g eta^T M2 eta) / 2, conserved by L (Sec. 2.5)."""
        u, eta = self.split(U)
        return 0.5 * (self.H * u @ (self.M1 @ u) + self.g * eta @ (self.M2 @ eta))

    def mass(self, U):
        """int eta dx."""
        _, eta = self.split(U)
        return float(np.sum(self.M2 @ eta))

    def norms(self, U):
        """(||u||_M1, ||u||_Hdiv, ||eta||_M2): the paper's error norms (Sec. 3)."""
        u, eta = self.split(U)
        du = self.solve_M2(self.D @ u)           # DG1 field equal to div u
        return (np.sqrt(u @ (self.M1 @ u)),
                np.sqrt(u @ (self.M1 @ u) + du @ (self.M2 @ du)),
                np.sqrt(eta @ (self.M2 @ eta)))
