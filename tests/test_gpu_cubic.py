"""The piecewise cubic surface (Sec. 3, geometry_degree = 3) on the GPU
against the FP64 oracle on the same surface.

Tolerance: relative L2 per field in the finite element norms, 1e-12 for the
FP64 path (the parity bound of the flat surface), 1e-5 for N in mixed
precision.  The oracle evaluates the cubic map through monomial
coefficients; the library through its closed-form barycentric basis, with
the same 5 x 5 cell rule and 5-point facet rule.
"""

import numpy as np
import pytest

from tests.test_gpu_parity import LAM, assert_close, dev, gpu, orc, rel, state

pytestmark = pytest.mark.gpu

CUBIC = 3


def cg(r, **kw):
    return gpu(r, geometry_degree=CUBIC, **kw)


def co(r, **kw):
    return orc(r, geometry_degree=CUBIC, **kw)


@pytest.mark.parametrize("r", [2, 3, 4])
def test_cubic_linear_parity(r):
    g, o = cg(r), co(r)
    U = np.random.default_rng(r).standard_normal(o.n) * 1e6
    U[o.n_u:] *= 1e-4
    assert_close(o, g.linear(dev(U)).cpu().numpy(), o.L(U))
    g.sync()


@pytest.mark.parametrize("r,upwind", [(2, 0), (3, 0), (4, 0), (3, 1)])
def test_cubic_nonlinear_parity(r, upwind):
    g, o = cg(r, upwind_convention=upwind), co(r, upwind=upwind)
    U = state(o, eta_noise=20.0)
    assert_close(o, g.nonlinear(dev(U)).cpu().numpy(), o.N(U))
    g.sync()


def test_cubic_nonlinear_with_topography():
    g, o = cg(3), co(3)
    b = 300.0 * np.random.default_rng(9).random(o.n_eta)
    U = state(o)
    g.set_topography(dev(b))
    o.ops.set_topography(b)
    try:
        assert_close(o, g.nonlinear(dev(U)).cpu().numpy(), o.N(U))
    finally:
        g.set_topography(dev(np.zeros(o.n_eta)))
        o.ops.set_topography(np.zeros(o.n_eta))


@pytest.mark.parametrize("r,t", [(2, 900.0), (3, -3600.0), (4, 3600.0)])
def test_cubic_expL_parity(r, t):
    g, o = cg(r), co(r)
    U = state(o)
    assert_close(o, g.expL(t, dev(U)).cpu().numpy(), o.expL(t, U))
    g.sync()


@pytest.mark.parametrize("r,T,M", [(2, 3600.0, 8), (3, 1800.0, 5), (4, 7200.0, 16)])
def test_cubic_averaged_rhs_parity(r, T, M):
    g, o = cg(r), co(r)
    U = state(o, eta_noise=5.0)
    want = o.averaged_rhs(T, M, U)
    assert_close(o, g.averaged_rhs(T, M, dev(U)).cpu().numpy(), want)
    assert_close(o, g.averaged_rhs_literal(T, M, dev(U)).cpu().numpy(), want)
    g.sync()


def test_cubic_timestep_and_norms():
    g, o = cg(3), co(3)
    U = state(o)
    want = o.timestep(900.0, 3600.0, 8, U, 3)
    Ud = dev(U)
    g.timestep(900.0, 3600.0, 8, Ud, 3)
    assert_close(o, Ud.cpu().numpy(), want)
    got = g.norms(dev(want))
    ref = o.ops.norms(want)
    assert np.allclose(got, ref, rtol=1e-12, atol=0.0), (got, ref)
    g.sync()


def test_cubic_solvers_agree():
    """The subdomain, mixed and FP64 solvers reach the same FP64 result on
    the cubic surface's mass matrix."""
    o = co(4)
    U = np.random.default_rng(44).standard_normal(o.n) * 1e6  # not divergence free: eta part of L is O(1)
    U[o.n_u:] *= 1e-4
    want = o.L(U)
    for solver in (0, 1, 2):
        g = cg(4, solver=solver)
        assert_close(o, g.linear(dev(U)).cpu().numpy(), want)
        g.sync()


def test_cubic_mixed_precision_nonlinear():
    g, o = cg(3, precision=1), co(3)
    U = state(o, eta_noise=20.0)
    ru, re = rel(o, g.nonlinear(dev(U)).cpu().numpy(), o.N(U))
    print(f"cubic mixed precision N r3: rel L2 u {ru:.2e} eta {re:.2e}")
    assert ru <= 1e-5 and re <= 1e-5, (ru, re)
    g.sync()


def test_flat_and_cubic_contexts_side_by_side():
    """Contexts of both surfaces on one mesh level keep their own operator
    data (the shared-mesh cache is keyed by the geometry) and differ by the
    geometry's O(h^2) change of the operators."""
    gf, gc_ = gpu(3), cg(3)
    of, oc = orc(3), co(3)
    U = np.random.default_rng(33).standard_normal(of.n) * 1e6  # not balanced: every part of L is O(1)
    U[of.n_u:] *= 1e-4
    Lf = gf.linear(dev(U)).cpu().numpy()
    Lc = gc_.linear(dev(U)).cpu().numpy()
    assert_close(of, Lf, of.L(U))
    assert_close(oc, Lc, oc.L(U))
    ru, _ = rel(of, Lc, Lf)
    assert 1e-5 < ru < 0.1, ru


def test_cubic_lambda_max_estimate():
    """The library's own estimate on the cubic surface lies within 1.0-1.05
    times the spectral radius of the oracle's cubic L (ARPACK)."""
    import scipy.sparse.linalg as spla
    g = cg(2, lambda_max=0.0)
    o = co(2)
    op = spla.LinearOperator((o.n, o.n), matvec=o.ops.L, dtype=np.float64)
    true = np.abs(spla.eigs(op, k=4, which="LM", tol=1e-12, return_eigenvectors=False)).max()
    assert 1.0 * true <= g.lambda_max <= 1.05 * true, (g.lambda_max, true)
    print(f"cubic refinement 2: lambda_max {true:.6g} (estimate {g.lambda_max:.6g}; flat {LAM[2]:.6g})")


def test_cubic_batch_matches_single_instances():
    """Batched evaluation of cubic-surface instances (both strategies) equals
    the single-instance path."""
    from paper_2103_07706_gb300 import pavg
    spec = [(2, 3600.0, 8), (3, 1800.0, 5), (2, 0.0, 4)]
    ms = [pavg.Model(r, lambda_max=LAM[r], geometry_degree=CUBIC) for r, _, _ in spec]
    U = [dev(state(co(r), seed=2200 + i, eta_noise=5.0)) for i, (r, _, _) in enumerate(spec)]
    T = [t for _, t, _ in spec]
    M = [m for _, _, m in spec]
    b = pavg.Batch(ms)
    try:
        b.averaged_rhs(T, M, U)
        keep = b.config()
        single = [m.averaged_rhs(t, mm, u).cpu().numpy() for m, t, mm, u in zip(ms, T, M, U)]
        for k in (0, 1):
            b.set_config(keep["threads"], keep["blocks_per_sm"], keep["resident"], keep["weighting"], k)
            got = [x.cpu().numpy() for x in b.averaged_rhs(T, M, U)]
            b.sync()
            for i, (r, _, _) in enumerate(spec):
                assert_close(co(r), got[i], single[i])
    finally:
        b.close()
        for m in ms:
            m.close()
