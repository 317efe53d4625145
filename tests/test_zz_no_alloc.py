"""The allocation-free entry point pavg_linear_noalloc.

It serves callers that cannot call cudaMalloc where they apply L (inside a
global-mode stream capture, in real-time loops, under a capped external memory
pool): its scratch is a static device array of the library.  This file is
collected last so that a failure here never hides the other tests, and it
passes both alone in a fresh process and after them.
"""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_noalloc_matches_linear_two_calls_in_a_row():
    import torch

    from paper_2103_07706_gb300 import pavg
    m = pavg.Model(4, lambda_max=0.0057)
    rng = np.random.default_rng(44)
    U = rng.standard_normal(m.n) * 1e6
    U[m.n_u:] *= 1e-4
    Ud = torch.from_numpy(U).cuda()
    want = m.linear(Ud).cpu().numpy()
    for _ in range(2):
        got = m.linear_noalloc(Ud).cpu().numpy()
        m.sync()
        for sl in (slice(0, m.n_u), slice(m.n_u, m.n)):
            err = np.linalg.norm(got[sl] - want[sl]) / np.linalg.norm(want[sl])
            assert err <= 1e-12, err
    # a different state next: no stale scratch leaks into the result
    U2 = torch.from_numpy(rng.standard_normal(m.n) * 1e5).cuda()
    a = m.linear(U2).cpu().numpy()
    b = m.linear_noalloc(U2).cpu().numpy()
    m.sync()
    assert np.linalg.norm(a - b) <= 1e-12 * np.linalg.norm(a)
    m.close()


def test_noalloc_rejects_meshes_beyond_its_scratch():
    from paper_2103_07706_gb300 import pavg
    m = pavg.Model(6, lambda_max=0.02335)
    import torch
    U = torch.zeros(m.n, dtype=torch.float64, device="cuda")
    with pytest.raises(pavg.PavgError) as e:
        m.linear_noalloc(U)
    assert e.value.code == -1 and "exceed" in str(e.value)
    m.close()


def test_noalloc_mixed_precision_within_the_solve_tolerance():
    """Under PAVG_PRECISION_MIXED both pavg_linear and the allocation-free
    entry point stop their mass solves at a relative residual of 1e-5 (with
    different solvers: block-Jacobi FP32 refinement and FP64 Jacobi CG), so
    their results agree to about that level, not to rounding; pavg_linear
    also forms the K-hat products in FP32 in this mode (the allocation-free
    entry point in FP64), which the eta part (a cell-local solve on both
    paths) shows at the FP32 rounding level."""
    import torch

    from paper_2103_07706_gb300 import pavg
    m = pavg.Model(4, lambda_max=0.0057, precision=pavg.PAVG_PRECISION_MIXED)
    rng = np.random.default_rng(45)
    U = rng.standard_normal(m.n) * 1e6
    U[m.n_u:] *= 1e-4
    Ud = torch.from_numpy(U).cuda()
    want = m.linear(Ud).cpu().numpy()
    for _ in range(2):
        got = m.linear_noalloc(Ud).cpu().numpy()
        m.sync()
        eu = np.linalg.norm(got[: m.n_u] - want[: m.n_u]) / np.linalg.norm(want[: m.n_u])
        ee = np.linalg.norm(got[m.n_u:] - want[m.n_u:]) / np.linalg.norm(want[m.n_u:])
        print(f"noalloc vs linear, mixed precision: u {eu:.2e}, eta {ee:.2e}")
        assert eu <= 1e-4, eu
        assert ee <= 1e-6, ee   # FP32 against FP64 K-hat products, then the same cell-local solve
    m.close()


def test_noalloc_inside_a_global_mode_graph_capture():
    """The entry point's reason to exist: after one call outside capture, the
    call can be recorded in a global-mode stream capture (which fails any
    allocating or otherwise capture-unsafe call made meanwhile) and the
    graph replayed on new inputs copied into the captured buffer."""
    import torch

    from paper_2103_07706_gb300 import pavg
    m = pavg.Model(4, lambda_max=0.0057)
    rng = np.random.default_rng(46)
    Uin = torch.zeros(m.n, dtype=torch.float64, device="cuda")
    out = torch.empty_like(Uin)
    m.linear_noalloc(Uin, out)  # first call before any capture (device address lookup)
    m.sync()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, capture_error_mode="global"):
        m.linear_noalloc(Uin, out)
    for _ in range(2):
        U = rng.standard_normal(m.n) * 1e6
        U[m.n_u:] *= 1e-4
        Uin.copy_(torch.from_numpy(U).cuda())
        g.replay()
        torch.cuda.synchronize()
        m.sync()
        got = out.cpu().numpy()
        want = m.linear(Uin).cpu().numpy()
        m.sync()
        for sl in (slice(0, m.n_u), slice(m.n_u, m.n)):
            err = np.linalg.norm(got[sl] - want[sl]) / np.linalg.norm(want[sl])
            assert err <= 1e-12, err
    del g
    m.close()
