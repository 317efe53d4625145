"""Seeded synthetic states for the rotating shallow-water model.

This module holds no part of the method (no L, N, exponential, average or
timestep): it only turns a seeded random spherical-harmonic field into degree
of freedom vectors in the library's canonical numbering, so that tests and the
benchmark feed the same inputs to every implementation.

Recipe (balanced flow plus small-scale content, the regime of the paper's
experiments: Rossby number ~0.1, mean depth ~5 km):
  eta'(x) = sum_{l=1..lmax} sum_{m=-l..l} a_lm Y_lm(x/|x|),  a_lm ~ N(0, 1) l^{-3/2}
            (real orthonormal spherical harmonics; numpy PCG64 seeded), scaled to
            `eta_rms` metres rms over its DG1 degrees of freedom;
  psi = g eta' / f0,  f0 = 2 Omega sin(45 deg);  u = k x grad psi (geostrophic,
            divergence free).
Degrees of freedom (canonical numbering: edge e, moment j -> 3e + j; interior
j of cell c -> 3E + 3c + j; elevation vertex i of cell c -> 3c + i):
  * elevation: eta' at the cell's vertices (DG1 nodal values);
  * velocity edge moments int_e (u . nu) p_j ds with nu = t x k, t the low->high
    tangent: since u . nu = -d psi / ds these need only psi along the edge
    (integration by parts against the Legendre polynomials p_j on [0, 1]);
  * velocity interior moments int_ref u_hat . q_j with u_hat = curl_ref psi_hat
    (contravariant pull-back of k x grad psi on a flat cell), again reduced to
    point values of psi by integration by parts.
The discrete velocity is therefore exactly divergence free.
"""

import math

import numpy as np


def _gl01(n):
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (x + 1.0), 0.5 * w


def real_sph_harm_sum(points, coeffs, lmax):
    """sum_lm coeffs[l, m + lmax] Y_lm(points/|points|), normalised recurrence.

    For each order m the associated Legendre values are summed over l first;
    cos(m phi) and sin(m phi) come from the angle-addition recurrence."""
    p = np.asarray(points, dtype=np.float64)
    r = np.linalg.norm(p, axis=-1)
    ct = np.clip(p[..., 2] / r, -1.0, 1.0)
    st = np.sqrt(np.maximum(0.0, 1.0 - ct * ct))
    rho = np.hypot(p[..., 0], p[..., 1])
    safe = np.where(rho > 0.0, rho, 1.0)
    c1 = np.where(rho > 0.0, p[..., 0] / safe, 1.0)  # cos(phi), sin(phi)
    s1 = np.where(rho > 0.0, p[..., 1] / safe, 0.0)
    out = np.zeros_like(ct)
    pmm = np.full_like(ct, math.sqrt(1.0 / (4.0 * math.pi)))
    cm, sm = np.ones_like(ct), np.zeros_like(ct)  # cos(m phi), sin(m phi)
    for m in range(0, lmax + 1):
        if m > 0:
            pmm = math.sqrt((2.0 * m + 1.0) / (2.0 * m)) * st * pmm
            cm, sm = cm * c1 - sm * s1, sm * c1 + cm * s1
        acc_c = np.zeros_like(ct)
        acc_s = np.zeros_like(ct)
        plm2 = None
        plm1 = pmm
        for l in range(m, lmax + 1):
            if l == m:
                plm = pmm
            elif l == m + 1:
                plm = math.sqrt(2.0 * m + 3.0) * ct * pmm
            else:
                a = math.sqrt((4.0 * l * l - 1.0) / (l * l - m * m))
                b = math.sqrt(((l - 1.0) ** 2 - m * m) / (4.0 * (l - 1.0) ** 2 - 1.0))
                plm = a * (ct * plm1 - b * plm2)
            if l >= m + 1:
                plm2, plm1 = plm1, plm
            if l == 0:
                continue
            acc_c += coeffs[l, lmax + m] * plm
            if m > 0:
                acc_s += coeffs[l, lmax - m] * plm
        if m == 0:
            out += acc_c
        else:
            out += math.sqrt(2.0) * (acc_c * cm + acc_s * sm)
    return out


def canonical_edges(cells):
    cells = np.asarray(cells)
    pairs = np.concatenate([cells[:, [1, 2]], cells[:, [2, 0]], cells[:, [0, 1]]])
    pairs = np.sort(pairs, axis=1)
    return np.unique(pairs, axis=0)


def velocity_dofs_from_streamfunction(verts, cells, edges, psi):
    """BDM2 degrees of freedom of u = k x grad psi (divergence free), from point
    values of psi only (see the module docstring); psi maps points (..., 3)
    to values (...)."""
    F, E = len(cells), len(edges)
    u = np.zeros(3 * E + 3 * F)
    # edge moments: -int_0^1 psi'(tau) p_j(tau) dtau by parts
    tau, wt = _gl01(6)
    xlo, xhi = verts[edges[:, 0]], verts[edges[:, 1]]
    pts = xlo[:, None, :] + tau[None, :, None] * (xhi - xlo)[:, None, :]
    ps = psi(pts)                                           # (E, 6)
    p0, p1 = psi(xlo), psi(xhi)
    u[0:3 * E:3] = -(p1 - p0)
    u[1:3 * E:3] = -p1 - p0 + 2.0 * ps @ wt
    u[2:3 * E:3] = p0 - p1 + ps @ (wt * (12.0 * tau - 6.0))
    # interior moments int_ref curl_ref(psi_hat) . q_j
    #   = -int psi_hat rot(q_j) + sum_edges int_0^1 psi_hat (d . q_j) dtau
    a = verts[cells[:, 0]]
    J0 = verts[cells[:, 1]] - a
    J1 = verts[cells[:, 2]] - a
    starts = np.array([[1.0, 0.0], [0.0, 1.0], [0.0, 0.0]])
    dirs = np.array([[-1.0, 1.0], [0.0, -1.0], [1.0, 0.0]])
    mom = np.zeros((F, 3))
    for i in range(3):
        xi = starts[i][None, :] + tau[:, None] * dirs[i][None, :]          # (6, 2)
        x = a[:, None, :] + xi[None, :, 0:1] * J0[:, None, :] + xi[None, :, 1:2] * J1[:, None, :]
        pv = psi(x)                                                         # (F, 6)
        d = dirs[i]
        q = np.stack([np.full(len(tau), d[0]),                              # d . (1, 0)
                      np.full(len(tau), d[1]),                              # d . (0, 1)
                      -xi[:, 1] * d[0] + xi[:, 0] * d[1]], axis=1)          # d . (-y, x)
        mom += pv @ (wt[:, None] * q)
    # -int psi_hat rot(q): rot = 0, 0, 2 ; collapsed Gauss rule on the triangle
    s, ws = _gl01(4)
    t, wt2 = _gl01(4)
    xi = np.stack([np.repeat(s, 4), (np.outer(1.0 - s, t)).reshape(-1)], axis=1)
    wtri = (np.outer(ws * (1.0 - s), wt2)).reshape(-1)
    x = a[:, None, :] + xi[None, :, 0:1] * J0[:, None, :] + xi[None, :, 1:2] * J1[:, None, :]
    mom[:, 2] -= 2.0 * psi(x) @ wtri
    u[3 * E:] = mom.reshape(-1)
    return u


def harmonic_state(verts, cells, seed, lmax, eta_rms=100.0, g=9.80616, omega=7.292e-5, rossby=None):
    """Balanced seeded state U = [u (3E + 3F), eta (3F)] as float64.

    With `rossby` given, the amplitude is chosen instead so that the Rossby
    number (below) takes that value: u and eta are both proportional to the
    amplitude, so the state at eta_rms is scaled by rossby / Ro(eta_rms), and
    info["eta_rms"] reports the resulting elevation rms.

    Returns (U, info) with info = {"rossby": ..., "u_rms": ..., "eta_rms": ...}.
    """
    if rossby is not None:
        U, info = harmonic_state(verts, cells, seed, lmax, eta_rms, g, omega)
        f = rossby / info["rossby"]
        info = dict(info, rossby=info["rossby"] * f, u_rms=info["u_rms"] * f, eta_rms=eta_rms * f)
        return U * f, info
    verts = np.asarray(verts, dtype=np.float64)
    cells = np.asarray(cells, dtype=np.int64)
    edges = canonical_edges(cells)
    F, E = len(cells), len(edges)
    rng = np.random.Generator(np.random.PCG64(seed))
    coeffs = np.zeros((lmax + 1, 2 * lmax + 1))
    for l in range(1, lmax + 1):
        coeffs[l, lmax - l: lmax + l + 1] = rng.standard_normal(2 * l + 1) * l ** -1.5
    # elevation at vertices, scaled to the requested rms over the DG1 DOFs
    eta_v = real_sph_harm_sum(verts, coeffs, lmax)
    eta = eta_v[cells].reshape(-1)
    scale = eta_rms / math.sqrt(np.mean(eta * eta))
    eta *= scale
    f0 = 2.0 * omega * math.sin(math.pi / 4.0)

    def psi(x):
        return g * scale * real_sph_harm_sum(x, coeffs, lmax) / f0

    u = velocity_dofs_from_streamfunction(verts, cells, edges, psi)
    # diagnostics: rms velocity from the edge flux densities, Rossby number
    elen = np.linalg.norm(verts[edges[:, 1]] - verts[edges[:, 0]], axis=1)
    u_rms = math.sqrt(np.mean((u[0:3 * E:3] / elen) ** 2))
    radius = float(np.linalg.norm(verts[0]))
    l_eff = max(1.0, float(np.sqrt(np.sum(coeffs ** 2 * np.arange(lmax + 1)[:, None] ** 2) / np.sum(coeffs ** 2))))
    rossby = u_rms / (f0 * math.pi * radius / l_eff)
    return np.concatenate([u, eta]), {"rossby": rossby, "u_rms": u_rms, "eta_rms": eta_rms, "edges": E, "cells": F}


def tc5_state(verts, cells, u0=20.0, H=5960.0, g=9.8, omega=7.292e-5, b0=2000.0, lat_c=math.pi / 6.0,
              lon_c=-math.pi / 2.0, r0=math.pi / 9.0):
    """Williamson's test case 5 as Sec. 3 states it: zonal flow
    u = (u0 / R)(-y, x, 0) in geostrophic balance with the layer depth
    h = H - (R Omega u0 + u0^2 / 2) z^2 / (g R^2), over a cone-shaped mountain
    b = b0 (1 - min(r0, d) / r0), d^2 = (lat - lat_c)^2 + (lon - lon_c)^2, the
    longitude difference wrapped to [-pi, pi].  The paper's constants are the
    defaults (Omega = 7.292e-5 s^-1 and u0 = 20 m/s, where the printed
    exponent and unit are typographical slips).

    Returns (U, b): U = [u, eta] with eta = h - H the elevation of the free
    surface (the depth is H + eta - b), and b at the DG1 nodes (cell vertices).
    u = k x grad psi with psi = -u0 R z / |x| (divergence free; psi is
    evaluated at the radial projection of each sample point onto the sphere,
    so that its variation along an edge chord is the sphere's); eta and b are
    nodal values at the cell vertices."""
    verts = np.asarray(verts, dtype=np.float64)
    cells = np.asarray(cells, dtype=np.int64)
    edges = canonical_edges(cells)
    R = float(np.linalg.norm(verts[0]))
    u = velocity_dofs_from_streamfunction(verts, cells, edges,
                                          lambda x: -u0 * R * x[..., 2] / np.linalg.norm(x, axis=-1))
    z = verts[:, 2]
    eta_v = -(R * omega * u0 + 0.5 * u0 * u0) * z * z / (g * R * R)
    lat = np.arcsin(np.clip(z / R, -1.0, 1.0))
    lon = np.arctan2(verts[:, 1], verts[:, 0])
    dlon = (lon - lon_c + math.pi) % (2.0 * math.pi) - math.pi
    d = np.sqrt((lat - lat_c) ** 2 + dlon ** 2)
    b_v = b0 * (1.0 - np.minimum(r0, d) / r0)
    return np.concatenate([u, eta_v[cells].reshape(-1)]), b_v[cells].reshape(-1)


# lambda_max of L per refinement (R = 6.37122e6 m, Omega = 7.292e-5 s^-1,
# g = 9.80616 m s^-2, H = 5000 m): the refinement-6 power-iteration estimate
# widened by 2 % (0.02335 s^-1), halved per coarser level (the fastest
# discrete gravity wave scales with the inverse cell size).
def lambda_max_for(refinement):
    return 0.02335 / 2.0 ** (6 - refinement)


def batch_workload(seed=2103, n=64, refinements=(4, 5, 6), t_hours=(0.25, 4.0), shifts=(16, 32, 64, 128)):
    """Independent instances of the batched evaluation: a list of dicts with
    refinement r (uniform over `refinements`), window T in seconds (uniform in
    `t_hours`), shift count M (uniform over `shifts`) and a state seed.  The
    state of each instance is harmonic_state(..., seed=state_seed, lmax=16)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        out.append({"refinement": int(rng.choice(refinements)),
                    "T": float(3600.0 * rng.uniform(*t_hours)),
                    "M": int(rng.choice(shifts)),
                    "state_seed": seed + 1 + i})
    return out
