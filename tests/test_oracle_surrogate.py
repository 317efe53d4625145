"""Pins of the surrogate oracle (oracle/surrogate.py) to facts outside it:
central finite differences for the backpropagated gradient, closed forms for
a zero network and for Adam's first step, mesh adjacency found from vertex
sets for the features, and the gather/scatter identity."""

import numpy as np
import pytest

from oracle import surrogate as S


def tiny(rng, n_in=7, hidden=5, n_out=3):
    p = S.init_params(rng, n_in, hidden, n_out)
    for k in ("b1", "b2", "b3"):
        p[k] = rng.standard_normal(p[k].shape) * 0.3
    return p


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(11)
    p = tiny(rng)
    X = rng.standard_normal((9, 7))
    Z = rng.standard_normal((9, 3))
    _, g = S.loss_and_grads(p, X, Z)
    h = 1e-6
    for k in S.PARAM_ORDER:
        num = np.zeros_like(p[k])
        for idx in np.ndindex(p[k].shape):
            q = {kk: vv.copy() for kk, vv in p.items()}
            q[k][idx] += h
            lp, _ = S.loss_and_grads(q, X, Z)
            q[k][idx] -= 2 * h
            lm, _ = S.loss_and_grads(q, X, Z)
            num[idx] = (lp - lm) / (2 * h)
        assert np.abs(num - g[k]).max() <= 1e-8 * max(1.0, np.abs(g[k]).max()), k


def test_zero_network_closed_form():
    """All weights zero: the output is b3 for every row, the loss is the mean
    of (b3 - z)^2, and only b3 has a gradient, 2 mean over rows of (b3 - z) / n_out."""
    rng = np.random.default_rng(3)
    p = {k: np.zeros_like(v) for k, v in tiny(rng).items()}
    p["b3"] = np.array([0.5, -1.0, 2.0])
    X = rng.standard_normal((6, 7))
    Z = rng.standard_normal((6, 3))
    loss, g = S.loss_and_grads(p, X, Z)
    assert loss == pytest.approx(((p["b3"] - Z) ** 2).mean(), rel=1e-14)
    assert np.allclose(g["b3"], 2.0 * (p["b3"] - Z).mean(axis=0) / 3, rtol=1e-14, atol=0)
    for k in ("W1", "b1", "W2", "b2", "W3"):
        assert not g[k].any(), k


def test_adam_first_step_is_lr_times_sign():
    """From zero moments the bias-corrected first step is -lr g / (|g| + eps)."""
    rng = np.random.default_rng(5)
    p = tiny(rng)
    g = {k: rng.standard_normal(v.shape) for k, v in p.items()}
    m = {k: np.zeros_like(v) for k, v in p.items()}
    v = {k: np.zeros_like(v) for k, v in p.items()}
    before = {k: x.copy() for k, x in p.items()}
    S.adam_step(p, g, m, v, 1, 1e-3)
    for k in S.PARAM_ORDER:
        assert np.allclose(p[k] - before[k], -1e-3 * g[k] / (np.abs(g[k]) + 1e-8), rtol=1e-12, atol=0)


@pytest.fixture(scope="module")
def asm1():
    from oracle.assembly import Assembly
    from oracle.mesh import build_mesh
    m = build_mesh(1, 6.37122e6)
    return Assembly(m, 7.292e-5, 6.37122e6)


def test_neighbours_from_vertex_sets(asm1):
    mesh = asm1.mesh
    nb = S.neighbours(mesh)
    sets = [set(c) for c in mesh.cells.tolist()]
    for c, (v0, v1, v2) in enumerate(mesh.cells.tolist()):
        # local edge i is opposite local vertex i
        for i, pair in enumerate(({v1, v2}, {v2, v0}, {v0, v1})):
            others = [d for d in range(len(sets)) if d != c and pair <= sets[d]]
            assert others == [nb[c, i]]


def test_features_place_a_single_dof(asm1):
    """A state with one nonzero edge DOF shows up, with the cell's sign and over
    the row cell's length scale sqrt(det), in the own slot of its two cells and
    in the neighbour slot of every cell next to either of them (2 + 2 x 3
    entries), and nowhere else."""
    mesh = asm1.mesh
    n = asm1.n_u + asm1.n_eta
    nb = S.neighbours(mesh)
    e, j = 7, 0
    U = np.zeros(n)
    U[3 * e + j] = 1.0
    X = S.features(asm1, U, np.zeros(n))
    want = np.zeros_like(X[:, :120])
    ell = np.sqrt(asm1.det)  # each row's velocity values are in units of its cell's length
    for side in range(2):
        c, i = mesh.edge_cells[e, side], mesh.edge_local[e, side]
        s = asm1.sign[c, 3 * i + j]
        want[c, 3 * i + j] = s / ell[c]
        for other in range(mesh.n_cells):
            for k in range(3):
                if nb[other, k] == c:
                    want[other, 30 + 30 * k + 3 * i + j] = s / ell[other]
    assert np.allclose(X[:, :120], want, rtol=1e-15, atol=0)
    assert np.count_nonzero(want) == 8


def test_scatter_inverts_local_values(asm1):
    rng = np.random.default_rng(2)
    D = rng.standard_normal(asm1.n_u + asm1.n_eta)
    assert np.allclose(S.scatter(asm1, S.targets(asm1, D)), D, rtol=0, atol=1e-15)


def test_geometry_features(asm1):
    g = S.geometry(asm1)
    # the centroid height over R lies in [-1, 1]; G / det of a near-equilateral
    # flat triangle: G00 = G11 = |e|^2, G01 = |e|^2 / 2, det = sqrt(3)/2 |e|^2
    assert np.all(np.abs(g[:, 0]) <= 1.0)
    assert np.allclose(g[:, 1], 2 / np.sqrt(3), rtol=0.25)
    assert np.allclose(g[:, 2], 1 / np.sqrt(3), rtol=0.35)
