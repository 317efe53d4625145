"""Oracle of the learned mesh-local surrogate of the large-M average.

TEST INFRASTRUCTURE: imported only by tests/, __graft_entry__.smoke() and
bench.py's CPU baseline; the product path never calls it.

The paper's average N-bar(U) = sum_m w_m e^{-s_m L} N(e^{s_m L} U)
(Sec. 2.2, Eq. vt_discretised) needs many shifts M for wide windows T
(Sec. 2.2: the Riemann sum must resolve the fast oscillations inside the
window).  The surrogate keeps a cheap average with few shifts, V = N-bar_Mc(U),
and adds a learned correction towards the large-M average N-bar_Mf(U):

    S(U) = V + scatter(sigma_y * MLP((features(U, V) - mu_x) / sigma_x) + mu_y)

features: for each cell, its own 15 values (12 velocity coefficients in the
cell's local frame, i.e. times the local-to-global signs of Sec. 2.5, and 3
elevation values) of U and of V, the same for the three cells across its
edges (in their own local frames, in local edge order), and 4 geometric
values: z_c / R at the centroid (f / 2 Omega) and G / det (the cell's metric
over its area).  124 inputs.  The velocity coefficients are moments of a
flux (velocity times length, Sec. 2.5), so every velocity value of a row is
divided by the row cell's length scale l_c = sqrt(det_c): rows of meshes of
different refinement then carry values of the same size.
MLP: two hidden layers of tanh units, linear output of 15 values per cell.
targets: the cell's 15 local values of N-bar_Mf(U) - V, velocity values
divided by l_c.
scatter: velocity values times l_c; elevation and interior velocity values
go to their DOFs; an edge DOF takes the mean of the two cells' values (times
their signs).
Loss: mean squared error over cells and outputs of the standardised
targets.  Training: Adam (Kingma & Ba 2015), beta1 0.9, beta2 0.999,
eps 1e-8.

Everything here is plain FP64 numpy in the order the definitions state.
"""

import numpy as np

N_LOCAL = 15
N_IN = 8 * N_LOCAL + 4
N_OUT = N_LOCAL


def neighbours(mesh):
    """(F, 3): the cell across local edge i of each cell."""
    F = mesh.n_cells
    nb = np.zeros((F, 3), dtype=np.int64)
    for c in range(F):
        for i in range(3):
            e = mesh.cell_edges[c, i]
            a, b = mesh.edge_cells[e]
            nb[c, i] = b if a == c else a
    return nb


def local_values(asm, X):
    """(F, 15): the cell's signed local velocity coefficients and its elevation values."""
    return np.concatenate([asm.sign * X[asm.udofs], X[asm.n_u + asm.etadofs]], axis=1)


def geometry(asm):
    """(F, 4): z_c / R, G00 / det, G01 / det, G11 / det."""
    zc = asm.a[:, 2] + (asm.J[:, 2, 0] + asm.J[:, 2, 1]) / 3.0
    return np.stack([zc / asm.radius, asm.G[:, 0, 0] / asm.det, asm.G[:, 0, 1] / asm.det,
                     asm.G[:, 1, 1] / asm.det], axis=1)


def length_scale(asm):
    """(F,): l_c = sqrt(det_c), det_c = |J0 x J1| (twice the flat cell's area)."""
    return np.sqrt(asm.det)


def _velocity_scaled(block, ell):
    """A (F, 15) block with its 12 velocity columns divided by ell (F,)."""
    out = block.copy()
    out[:, :12] /= ell[:, None]
    return out


def features(asm, U, V):
    """(F, 124) raw (unstandardised) inputs of every cell."""
    nb = neighbours(asm.mesh)
    ell = length_scale(asm)
    lu, lv = local_values(asm, U), local_values(asm, V)
    parts = [_velocity_scaled(lu, ell), _velocity_scaled(lv, ell)]
    for i in range(3):
        parts += [_velocity_scaled(lu[nb[:, i]], ell), _velocity_scaled(lv[nb[:, i]], ell)]
    parts.append(geometry(asm))
    return np.concatenate(parts, axis=1)


def targets(asm, D):
    """(F, 15) local values of a correction vector D, velocity values over l_c."""
    return _velocity_scaled(local_values(asm, D), length_scale(asm))


def scatter(asm, Y):
    """Vector of n values from per-cell local values Y (F, 15), velocity values times l_c."""
    out = np.zeros(asm.n_u + asm.n_eta)
    ell = length_scale(asm)
    for c in range(asm.mesh.n_cells):
        for k in range(12):
            d = asm.udofs[c, k]
            v = asm.sign[c, k] * Y[c, k] * ell[c]
            out[d] += 0.5 * v if k < 9 else v  # local DOFs 0-8 sit on edges, 9-11 inside
        out[asm.n_u + asm.etadofs[c]] = Y[c, 12:15]
    return out


def column_stats(X):
    """Column means and population standard deviations (1 where a column is constant)."""
    mu = X.mean(axis=0)
    sd = np.sqrt(((X - mu) ** 2).mean(axis=0))
    sd = np.where(sd > 0.0, sd, 1.0)
    return mu, sd


def init_params(rng, n_in=N_IN, hidden=128, n_out=N_OUT):
    """Uniform Glorot initialisation, zero biases."""
    def glorot(a, b):
        lim = np.sqrt(6.0 / (a + b))
        return rng.uniform(-lim, lim, size=(a, b))
    return {"W1": glorot(hidden, n_in), "b1": np.zeros(hidden), "W2": glorot(hidden, hidden),
            "b2": np.zeros(hidden), "W3": glorot(n_out, hidden), "b3": np.zeros(n_out)}


PARAM_ORDER = ("W1", "b1", "W2", "b2", "W3", "b3")


def forward(p, X):
    """Hidden activations and output of the MLP for rows X (B, n_in)."""
    H1 = np.tanh(X @ p["W1"].T + p["b1"])
    H2 = np.tanh(H1 @ p["W2"].T + p["b2"])
    Y = H2 @ p["W3"].T + p["b3"]
    return H1, H2, Y


def loss_and_grads(p, X, Z):
    """Mean squared error over all B x n_out outputs and its gradient (backpropagation)."""
    H1, H2, Y = forward(p, X)
    n = Y.size
    R = Y - Z
    loss = float((R * R).sum() / n)
    dY = 2.0 * R / n
    g = {"W3": dY.T @ H2, "b3": dY.sum(axis=0)}
    dA2 = (dY @ p["W3"]) * (1.0 - H2 * H2)
    g["W2"] = dA2.T @ H1
    g["b2"] = dA2.sum(axis=0)
    dA1 = (dA2 @ p["W2"]) * (1.0 - H1 * H1)
    g["W1"] = dA1.T @ X
    g["b1"] = dA1.sum(axis=0)
    return loss, g


def adam_step(p, g, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (step number t >= 1) of p in place; m, v updated in place."""
    for k in PARAM_ORDER:
        m[k] = beta1 * m[k] + (1.0 - beta1) * g[k]
        v[k] = beta2 * v[k] + (1.0 - beta2) * g[k] * g[k]
        mh = m[k] / (1.0 - beta1 ** t)
        vh = v[k] / (1.0 - beta2 ** t)
        p[k] = p[k] - lr * mh / (np.sqrt(vh) + eps)


def flatten(p):
    return np.concatenate([np.asarray(p[k], dtype=np.float64).ravel() for k in PARAM_ORDER])


def unflatten(vec, n_in=N_IN, hidden=128, n_out=N_OUT):
    shapes = {"W1": (hidden, n_in), "b1": (hidden,), "W2": (hidden, hidden), "b2": (hidden,),
              "W3": (n_out, hidden), "b3": (n_out,)}
    out, o = {}, 0
    for k in PARAM_ORDER:
        size = int(np.prod(shapes[k]))
        out[k] = np.asarray(vec[o:o + size], dtype=np.float64).reshape(shapes[k])
        o += size
    return out


def apply(asm, p, stats, U, V):
    """S(U) = V + scatter(de-standardised MLP output) for one state."""
    mu_x, sd_x, mu_y, sd_y = stats
    X = (features(asm, U, V) - mu_x) / sd_x
    _, _, Y = forward(p, X)
    return V + scatter(asm, Y * sd_y + mu_y)
