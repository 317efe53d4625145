"""lambda_max: the eigenvalue of L of largest magnitude (paper Sec. 2.4).

The paper does not say how it is found.  Reading used here: L is skew-adjoint
in the energy inner product <U, V>_W = H u.M1 v + g eta.M2 zeta, so its
eigenvalues are imaginary and -L^2 is W-self-adjoint and positive
semi-definite; power iteration on -L^2 from a seeded random start gives
lambda_max^2 as the Rayleigh quotient ||L v||_W^2 / ||v||_W^2.
For small meshes the dense eigenvalues of L are the exact answer.
"""

import numpy as np


def w_inner(ops, U, V):
    u, eta = ops.split(U)
    v, zeta = ops.split(V)
    return ops.H * u @ (ops.M1 @ v) + ops.g * eta @ (ops.M2 @ zeta)


def power_iteration(ops, iters=300, seed=7706, rtol=1e-12):
    rng = np.random.default_rng(seed)
    v = rng.standard_normal(ops.n)
    v /= np.sqrt(w_inner(ops, v, v))
    est = 0.0
    for _ in range(iters):
        Lv = ops.L(v)
        rq = w_inner(ops, Lv, Lv)
        new = np.sqrt(rq)
        w = -ops.L(Lv)
        v = w / np.sqrt(w_inner(ops, w, w))
        if est > 0.0 and abs(new - est) <= rtol * new:
            est = new
            break
        est = new
    return est


def dense_L(ops):
    """Dense matrix of L (small meshes only)."""
    n = ops.n
    out = np.zeros((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        out[:, j] = ops.L(e)
    return out
