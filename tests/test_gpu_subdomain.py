"""The subdomain mass solver (PAVG_SOLVER_SUBDOMAIN, the default): FP32
Chebyshev iterations on one part of the mesh per block with neighbour-only
exchange, refined by FP64 residuals.  Against the oracle's L (sparse LU mass
solves) and the library's two other solvers, on meshes up to the benchmark's;
bitwise repeatable; and its bounded waits, made to run out on purpose through
the test hook (one block withholds its arrival or its shared contributions):
PAVG_ERR_TIMEOUT is latched, and after pavg_reset_stats the same context
computes L U correctly again."""

import numpy as np
import pytest

from tests.test_gpu_parity import LAM, assert_close, dev, orc

pytestmark = pytest.mark.gpu


def _model(r, **kw):
    from paper_2103_07706_gb300 import pavg
    kw.setdefault("lambda_max", LAM.get(r, 0.02335 / 2 ** (6 - r)))
    return pavg.Model(r, **kw)


@pytest.mark.parametrize("r", [1, 2, 3, 4])
def test_linear_parity_against_oracle(r):
    g, o = _model(r), orc(r)
    # a random state: the harmonic states are divergence-free, so the eta
    # part of their L U is round-off and has no meaningful relative error
    U = np.random.default_rng(r).standard_normal(o.n) * 10.0
    assert_close(o, g.linear(dev(U)).cpu().numpy(), o.L(U), tol=1e-13)
    g.sync()
    st = g.stats()
    assert st["cg_sweeps_mean"] >= 2 and st["cg_iters_mean"] > 0
    g.close()


@pytest.mark.parametrize("r", [5, 6])
def test_three_solvers_agree(r):
    """Subdomain, global mixed (FP32 CG) and FP64 Jacobi CG: the same M1^{-1}
    to their common tolerance (relative residual 1e-14)."""
    import torch

    from paper_2103_07706_gb300 import pavg
    outs, U, nu = {}, None, 0
    for solver in (pavg.PAVG_SOLVER_SUBDOMAIN, pavg.PAVG_SOLVER_MIXED, pavg.PAVG_SOLVER_FP64):
        g = _model(r, solver=solver)
        if U is None:
            U = np.random.default_rng(7).standard_normal(g.n)
            U[g.n_u:] *= 1e-2
        outs[solver] = g.linear(torch.from_numpy(U).cuda()).cpu().numpy()
        g.sync()
        nu = g.n_u
        g.close()
    ref = outs[pavg.PAVG_SOLVER_FP64]
    for solver in (pavg.PAVG_SOLVER_SUBDOMAIN, pavg.PAVG_SOLVER_MIXED):
        for sl in (slice(0, nu), slice(nu, None)):
            err = np.linalg.norm(outs[solver][sl] - ref[sl]) / np.linalg.norm(ref[sl])
            assert err <= 1e-12, (solver, err)


def test_repeatable_and_iteration_accounting():
    import torch
    g = _model(5)
    U = torch.from_numpy(np.random.default_rng(3).standard_normal(g.n)).cuda()
    a = g.linear(U).cpu().numpy()
    g.reset_stats()
    b = g.linear(U).cpu().numpy()
    g.sync()
    st = g.stats()
    assert np.array_equal(a, b)
    assert st["cg_solves"] == 1
    assert st["cg_iters_mean"] == st["cg_iters_max"] > 0
    # a fixed number of Chebyshev iterations per sweep
    assert st["cg_iters_mean"] % st["cg_sweeps_mean"] == 0
    g.close()


@pytest.mark.parametrize("mode", [1, 2])
def test_bounded_waits_run_out_and_the_context_recovers(mode):
    """A block that never arrives at a grid-wide sum (mode 1) or never
    publishes its shared contributions (mode 2) makes the other blocks' waits
    run out after the set bound (2 ms here): the launch ends, TIMEOUT is
    reported by pavg_sync, and after pavg_reset_stats the context is usable."""
    from paper_2103_07706_gb300 import pavg
    g, o = _model(4), orc(4)
    U = np.random.default_rng(44).standard_normal(o.n) * 10.0
    Ud = dev(U)
    g.linear(Ud)
    g.sync()
    g.test_stall(mode, part=3, wait_us=2000.0)
    g.linear(Ud)
    with pytest.raises(pavg.PavgError) as e:
        g.sync()
    assert e.value.code == -6  # PAVG_ERR_TIMEOUT
    assert g.stats()["error_flags"] & 2
    g.test_stall(0)
    g.reset_stats()
    assert_close(o, g.linear(Ud).cpu().numpy(), o.L(U), tol=1e-13)
    g.sync()
    assert g.stats()["error_flags"] == 0
    g.close()


def test_stall_hook_arguments():
    from paper_2103_07706_gb300 import pavg
    g = _model(3)
    for args in [(3, 0, 0.0), (1, -1, 0.0), (1, 10 ** 6, 0.0), (1, 0, -1.0)]:
        with pytest.raises(pavg.PavgError):
            g.test_stall(*args)
    g.close()
    h = _model(3, solver=pavg.PAVG_SOLVER_MIXED)
    with pytest.raises(pavg.PavgError):
        h.test_stall(1, 0, 100.0)
    h.close()


def test_large_mesh_after_small_mesh():
    """The kernel's dynamic shared-memory limit is one setting per device:
    configuring a small mesh after a large one must not make the large one's
    launches invalid (it did once, in the batched benchmark)."""
    import torch
    big = _model(6)
    small = _model(3)
    U = torch.from_numpy(np.random.default_rng(5).standard_normal(big.n)).cuda()
    big.linear(U)
    big.sync()
    assert big.stats()["solver_in_use"] == 2 and small.stats()["solver_in_use"] == 2
    small.close()
    big.close()
