"""Batched evaluation (pavg_batch_*, one persistent launch per direction for
all instances) against the FP64 oracle and the single-instance GPU path.

Tolerance: the FP64 bound of the parity tests (relative L2 per field in the
finite element norms, 1e-12).  Results of two grid configurations differ only
by rounding (same bound); one configuration is bit-reproducible.
"""

import numpy as np
import pytest

from tests.test_gpu_parity import LAM, RTOL, assert_close, dev, orc, state

pytestmark = pytest.mark.gpu

# refinement, T, M: several levels and windows, T = 0 (N only), a window so
# short that the Chebyshev degree is 0, one shift, the closed-rule-free default
SPEC = [(2, 3600.0, 8), (3, 1800.0, 5), (3, 3600.0, 8), (4, 7200.0, 16), (2, 0.0, 4), (3, 1e-3, 3), (2, 900.0, 1)]


def _models(spec, **kw):
    from paper_2103_07706_gb300 import pavg
    return [pavg.Model(r, lambda_max=LAM[r], **kw) for r, _, _ in spec]


def _states(spec):
    return [dev(state(orc(r), seed=2103 + i, eta_noise=5.0)) for i, (r, _, _) in enumerate(spec)]


@pytest.fixture(scope="module")
def batch_case():
    from paper_2103_07706_gb300 import pavg
    ms = _models(SPEC)
    U = _states(SPEC)
    b = pavg.Batch(ms)
    yield ms, U, b
    b.close()
    for m in ms:
        m.close()


def test_batch_matches_oracle(batch_case):
    ms, U, b = batch_case
    T = [t for _, t, _ in SPEC]
    M = [m for _, _, m in SPEC]
    out = b.averaged_rhs(T, M, U)
    b.sync()
    cfg = b.config()
    assert cfg["threads"] in (128, 256) and cfg["blocks_per_sm"] >= 1
    for i, (r, t, m) in enumerate(SPEC):
        o = orc(r)
        assert_close(o, out[i].cpu().numpy(), o.averaged_rhs(t, m, U[i].cpu().numpy()))


def test_batch_matches_single_instance_and_is_reproducible(batch_case):
    ms, U, b = batch_case
    T = [t for _, t, _ in SPEC]
    M = [m for _, _, m in SPEC]
    a = [x.cpu().numpy() for x in b.averaged_rhs(T, M, U)]
    c = [x.cpu().numpy() for x in b.averaged_rhs(T, M, U)]
    b.sync()
    for i, (r, t, m) in enumerate(SPEC):
        assert np.array_equal(a[i], c[i])
        single = ms[i].averaged_rhs(t, m, U[i]).cpu().numpy()
        assert_close(orc(r), a[i], single)
    fwd, bwd = b.kernel_time()
    # one graph branch per instance times the whole evaluation as "forward"
    assert fwd > 0.0 and (bwd > 0.0 if b.config()["strategy"] == 0 else bwd >= 0.0)


@pytest.mark.parametrize("threads,bps,res,wt", [(128, 1, 0, 0), (256, 2, 1, 1), (128, 4, 1, 0), (256, 3, 0, 1)])
def test_batch_configurations_agree(batch_case, threads, bps, res, wt):
    ms, U, b = batch_case
    T = [t for _, t, _ in SPEC]
    M = [m for _, _, m in SPEC]
    ref = [x.cpu().numpy() for x in b.averaged_rhs(T, M, U)]
    keep = b.config()
    try:
        b.set_config(threads, bps, res, wt)
        got = [x.cpu().numpy() for x in b.averaged_rhs(T, M, U)]
        b.sync()
    finally:
        b.set_config(keep["threads"], keep["blocks_per_sm"], keep["resident"], keep["weighting"], keep["strategy"])
    for i, (r, _, _) in enumerate(SPEC):
        assert_close(orc(r), got[i], ref[i])


@pytest.mark.parametrize("part_cells", [0, 512])
def test_batch_strategies_agree(part_cells):
    """Persistent chain launches (strategy 0) and one graph branch per
    instance running its own solver (strategy 1), with the subdomain solver
    on all SMs or on parts of at least 512 cells: both match the
    single-instance path and the oracle; strategy 1 is bit-identical to the
    same contexts evaluated one at a time."""
    from paper_2103_07706_gb300 import pavg
    ms = _models(SPEC, sd_part_cells=part_cells)
    U = _states(SPEC)
    T = [t for _, t, _ in SPEC]
    M = [m for _, _, m in SPEC]
    b = pavg.Batch(ms)
    try:
        b.averaged_rhs(T, M, U)  # autotune and strategy choice
        keep = b.config()
        assert keep["strategy"] in (0, 1) and keep["predicted_ms"] > 0.0
        got = {}
        for k in (0, 1):
            b.set_config(keep["threads"], keep["blocks_per_sm"], keep["resident"], keep["weighting"], k)
            assert b.config()["strategy"] == k
            got[k] = [x.cpu().numpy() for x in b.averaged_rhs(T, M, U)]
            b.sync()
        with pytest.raises(pavg.PavgError):
            b.set_config(keep["threads"], keep["blocks_per_sm"], keep["resident"], keep["weighting"], 2)
        single = [m.averaged_rhs(t, mm, u).cpu().numpy() for m, t, mm, u in zip(ms, T, M, U)]
        for m in ms:
            m.sync()
        for i, (r, t, m) in enumerate(SPEC):
            assert np.array_equal(got[1][i], single[i])
            assert_close(orc(r), got[0][i], got[1][i])
            if i < 3:
                o = orc(r)
                assert_close(o, got[1][i], o.averaged_rhs(t, m, U[i].cpu().numpy()))
    finally:
        b.close()
        for m in ms:
            m.close()


def test_batch_survives_workspace_growth(batch_case):
    """A larger single-instance call moves a context's buffers; the batch
    re-captures its graph and stays correct."""
    ms, U, b = batch_case
    T = [t for _, t, _ in SPEC]
    M = [m for _, _, m in SPEC]
    ref = [x.cpu().numpy() for x in b.averaged_rhs(T, M, U)]
    ms[0].averaged_rhs(4 * 3600.0, 40, U[0])
    got = [x.cpu().numpy() for x in b.averaged_rhs(T, M, U)]
    b.sync()
    for i in range(len(SPEC)):
        assert np.array_equal(got[i], ref[i])


def test_batch_autotune_reports_a_launchable_configuration(batch_case):
    ms, U, b = batch_case
    T = [t for _, t, _ in SPEC]
    M = [m for _, _, m in SPEC]
    cfg = b.autotune(T, M, U)
    assert cfg["predicted_ms"] > 0.0
    assert cfg == b.config()
    out = b.averaged_rhs(T, M, U)
    b.sync()
    assert all(np.isfinite(x.cpu().numpy()).all() for x in out)


def test_batch_argument_errors():
    from paper_2103_07706_gb300 import pavg
    m = pavg.Model(2, lambda_max=LAM[2])
    with pytest.raises(pavg.PavgError):
        pavg.Batch([m, m])  # a context twice
    f = pavg.Model(2, lambda_max=LAM[2], solver=pavg.PAVG_SOLVER_FP64)
    with pytest.raises(pavg.PavgError):
        pavg.Batch([m, f])
    b = pavg.Batch([m])
    U = dev(state(orc(2)))
    with pytest.raises(pavg.PavgError):
        b.averaged_rhs([-1.0], [4], [U])
    with pytest.raises(pavg.PavgError):
        b.averaged_rhs([3600.0], [0], [U])
    with pytest.raises(pavg.PavgError):
        b.set_config(96, 1)
    b.close()
    m.close()
    f.close()


def test_batch_full_size_workload():
    """The batched workload at full size: 64 instances, refinements 4-6,
    T in [0.25, 4] h, M in {16, 32, 64, 128}, one persistent launch per
    direction.  Sampled instances (two per refinement) against the
    single-instance path; every instance finite, no device error."""
    from paper_2103_07706_gb300 import pavg
    from paper_2103_07706_gb300.inputs import batch_workload, harmonic_state, lambda_max_for
    work = batch_workload()
    ms, U = [], []
    for w in work:
        m = pavg.Model(w["refinement"], lambda_max=lambda_max_for(w["refinement"]))
        v, c = m.mesh()
        ms.append(m)
        U.append(dev(harmonic_state(v, c, w["state_seed"], 16)[0]))
    b = pavg.Batch(ms)
    out = b.averaged_rhs([w["T"] for w in work], [w["M"] for w in work], U)
    b.sync()
    sample = []
    for r in (4, 5, 6):
        sample += [i for i, w in enumerate(work) if w["refinement"] == r][:2]
    for i in sample:
        w = work[i]
        want = ms[i].averaged_rhs(w["T"], w["M"], U[i]).cpu().numpy()
        got = out[i].cpu().numpy()
        nu = ms[i].n_u
        du = np.linalg.norm(got[:nu] - want[:nu]) / np.linalg.norm(want[:nu])
        de = np.linalg.norm(got[nu:] - want[nu:]) / np.linalg.norm(want[nu:])
        assert du <= RTOL and de <= RTOL, (i, w, du, de)
    for i, m in enumerate(ms):
        x = out[i].cpu().numpy()
        assert np.isfinite(x).all()
        assert m.stats()["error_flags"] == 0
    b.close()
    for m in ms:
        m.close()


def test_contexts_share_the_mesh_but_not_topography():
    """Contexts of one refinement share mesh and operator data; each keeps its
    own topography and workspace, and destroying one leaves the other intact."""
    import torch
    from paper_2103_07706_gb300 import pavg
    a = pavg.Model(2, lambda_max=LAM[2])
    b = pavg.Model(2, lambda_max=LAM[2])
    o = orc(2)
    U = dev(state(o))
    ref = a.nonlinear(U).cpu().numpy()
    b.set_topography(dev(300.0 * np.random.default_rng(1).random(o.n_eta)))
    assert np.array_equal(a.nonlinear(U).cpu().numpy(), ref)
    assert not np.array_equal(b.nonlinear(U).cpu().numpy(), ref)
    b.close()
    assert np.array_equal(a.averaged_rhs(1800.0, 4, U).cpu().numpy(),
                          pavg.Model(2, lambda_max=LAM[2]).averaged_rhs(1800.0, 4, U).cpu().numpy())
    torch.cuda.synchronize()
    a.close()


def test_batch_timestep_matches_single_instance_and_oracle():
    """Two averaged Lawson RK4 steps of instances with their own dt, T, M."""
    from paper_2103_07706_gb300 import pavg
    spec = [(2, 900.0, 3600.0, 8), (3, 900.0, 3600.0, 8), (3, 600.0, 1800.0, 5), (2, 1200.0, 0.0, 1)]
    ms = [pavg.Model(r, lambda_max=LAM[r]) for r, _, _, _ in spec]
    U0 = [state(orc(r), seed=70 + i) for i, (r, _, _, _) in enumerate(spec)]
    Ub = [dev(u) for u in U0]
    b = pavg.Batch(ms)
    b.timestep([d for _, d, _, _ in spec], [t for _, _, t, _ in spec], [m for _, _, _, m in spec], Ub, 2)
    b.sync()
    for i, (r, d, t, m) in enumerate(spec):
        Us = dev(U0[i])
        ms[i].timestep(d, t, m, Us, 2)
        assert_close(orc(r), Ub[i].cpu().numpy(), Us.cpu().numpy())
    o = orc(3)
    assert_close(o, Ub[1].cpu().numpy(), o.timestep(900.0, 3600.0, 8, U0[1], 2))
    b.close()
    for m_ in ms:
        m_.close()


def test_batch_instance_with_topography():
    """Each instance keeps its own topography inside a batch."""
    from paper_2103_07706_gb300 import pavg
    o = orc(2)
    b0 = 300.0 * np.random.default_rng(8).random(o.n_eta)
    ms = [pavg.Model(2, lambda_max=LAM[2]) for _ in range(2)]
    ms[1].set_topography(dev(b0))
    U = [dev(state(o, seed=31)), dev(state(o, seed=32))]
    b = pavg.Batch(ms)
    out = b.averaged_rhs([3600.0, 3600.0], [6, 6], U)
    b.sync()
    assert_close(o, out[0].cpu().numpy(), o.averaged_rhs(3600.0, 6, U[0].cpu().numpy()))
    o.ops.set_topography(b0)
    try:
        assert_close(o, out[1].cpu().numpy(), o.averaged_rhs(3600.0, 6, U[1].cpu().numpy()))
    finally:
        o.ops.set_topography(np.zeros(o.n_eta))
    b.close()
    for m in ms:
        m.close()
