"""Learned surrogate (pavg_surrogate_*): its kernels against the FP64 oracle
(oracle/surrogate.py), training, the Riemann-sum fallback, and what the
trained network gains over the cheap average it corrects.

Tolerances: features are FP32 copies of FP64 values (relative 1e-6); the MLP,
its gradient and Adam run in FP32 against the oracle's FP64 (relative 1e-4 in
the max norm of each parameter block, 1e-5 for the forward output).
"""

import numpy as np
import pytest

from oracle import surrogate as S
from tests.test_gpu_parity import LAM, dev, orc, state

pytestmark = pytest.mark.gpu


def _model(r):
    from paper_2103_07706_gb300 import pavg
    return pavg.Model(r, lambda_max=LAM[r])


def _blocks(vec, hidden):
    return S.unflatten(np.asarray(vec, dtype=np.float64), hidden=hidden)


def _rel_max(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-30))


def test_features_match_oracle():
    from paper_2103_07706_gb300 import pavg
    m, o = _model(2), orc(2)
    U = state(o, seed=1, eta_noise=5.0)
    V = state(o, seed=2, eta_noise=3.0)
    sur = pavg.Surrogate(hidden=16)
    X = sur.features(m, dev(U), dev(V)).cpu().numpy()
    want = S.features(o.ops.asm, U, V)
    assert X.shape == want.shape
    assert np.allclose(X, want, rtol=1e-6, atol=1e-6 * np.abs(want).max(axis=0))
    sur.close()
    m.close()


@pytest.mark.parametrize("B,hidden", [(300, 128), (64, 32), (1, 7)])
def test_gradient_matches_oracle(B, hidden):
    """Forward and backward kernels on standardised rows (B not a multiple of the 64-row tile)."""
    import torch
    from paper_2103_07706_gb300 import pavg
    rng = np.random.default_rng(B)
    sur = pavg.Surrogate(hidden=hidden, seed=B + 1)
    p = _blocks(sur.params(), hidden)
    for k in ("b1", "b2", "b3"):  # nonzero biases exercise the bias paths
        p[k] = rng.standard_normal(p[k].shape) * 0.2
    sur.set_params(S.flatten(p).astype(np.float32))
    p = _blocks(sur.params(), hidden)  # the FP32 values the kernels see
    X = rng.standard_normal((B, S.N_IN)).astype(np.float32)
    Z = rng.standard_normal((B, S.N_OUT)).astype(np.float32)
    loss, g = sur.gradient(torch.from_numpy(X).cuda(), torch.from_numpy(Z).cuda())
    want_loss, want = S.loss_and_grads(p, X.astype(np.float64), Z.astype(np.float64))
    assert loss == pytest.approx(want_loss, rel=1e-5)
    got = _blocks(g.cpu().numpy(), hidden)
    for k in S.PARAM_ORDER:
        assert _rel_max(got[k], want[k]) <= 1e-4, k
    sur.close()


def test_adam_step_matches_oracle():
    import torch
    from paper_2103_07706_gb300 import pavg
    rng = np.random.default_rng(4)
    sur = pavg.Surrogate(hidden=32, seed=9)
    p = _blocks(sur.params(), 32)
    m = {k: np.zeros_like(v) for k, v in p.items()}
    v = {k: np.zeros_like(x) for k, x in p.items()}
    for t in (1, 2, 3):
        g = {k: rng.standard_normal(x.shape) for k, x in p.items()}
        gf = S.flatten(g).astype(np.float32)
        sur.adam_step(torch.from_numpy(gf).cuda(), 1e-2)
        S.adam_step(p, _blocks(gf, 32), m, v, t, 1e-2)
    got = _blocks(sur.params(), 32)
    for k in S.PARAM_ORDER:
        assert _rel_max(got[k], p[k]) <= 1e-5, k
    sur.close()


def test_apply_matches_oracle_and_bf16_is_close():
    """Features, forward pass, de-standardisation and edge-averaging scatter."""
    from paper_2103_07706_gb300 import pavg
    m, o = _model(2), orc(2)
    rng = np.random.default_rng(8)
    U = state(o, seed=3, eta_noise=5.0)
    V = state(o, seed=4, eta_noise=2.0)
    sur = pavg.Surrogate(hidden=32, seed=5)
    X = S.features(o.ops.asm, U, V)
    mx, sx = X.mean(axis=0).astype(np.float32), (X.std(axis=0) + 1e-3).astype(np.float32)
    my = rng.standard_normal(S.N_OUT).astype(np.float32)
    sy = (0.5 + rng.random(S.N_OUT)).astype(np.float32)
    sur.set_scaling(mx, sx, my, sy)
    p = _blocks(sur.params(), 32)
    got = sur.apply(m, dev(U), dev(V)).cpu().numpy()
    want = S.apply(o.ops.asm, p, (mx.astype(np.float64), sx.astype(np.float64), my.astype(np.float64),
                                  sy.astype(np.float64)), U, V)
    corr_want = want - V
    assert np.abs((got - V) - corr_want).max() <= 1e-5 * np.abs(corr_want).max()
    bf = sur.apply(m, dev(U), dev(V), bf16=True).cpu().numpy()
    assert np.abs((bf - V) - corr_want).max() <= 3e-2 * np.abs(corr_want).max()
    sur.close()
    m.close()


def _pairs(m, o, seeds, T, Mc, Mf, lmax=8):
    import torch
    U, Vc, Vf = [], [], []
    for sd in seeds:
        u = dev(state(o, seed=sd, lmax=lmax))
        U.append(u)
        Vc.append(m.averaged_rhs(T, Mc, u))
        Vf.append(m.averaged_rhs(T, Mf, u))
    torch.cuda.synchronize()
    return U, Vc, Vf


def test_training_gain_and_fallback():
    """Refinement 3, T = 4 h: the network trained on 48 (state, average)
    pairs generated by the method corrects the M = 8 average towards the
    M = 128 average on states it never saw; the M = 128 sum judges the error
    and replaces the surrogate above the threshold."""
    from paper_2103_07706_gb300 import pavg
    m, o = _model(3), orc(3)
    T, Mc, Mf = 4 * 3600.0, 8, 128
    U, Vc, Vf = _pairs(m, o, range(100, 148), T, Mc, Mf)
    sur = pavg.Surrogate(hidden=128, seed=2103)
    sur.add_pairs(m, U, Vc, Vf)
    assert sur.rows() == 48 * m.n_cells
    sur.fit_scaling()
    loss = sur.train(epochs=40, batch=2048, lr=2e-3)
    assert loss[-1] < 0.5 * loss[0]
    # held-out states: error of the cheap average alone (a network that outputs 0)
    zero = pavg.Surrogate(hidden=8)
    zero.set_params(np.zeros(zero.nparams, dtype=np.float32))
    errs_cheap, errs_sur = [], []
    for sd in range(900, 906):
        u = dev(state(o, seed=sd, lmax=8))
        _, _, e0 = zero.averaged_rhs(m, T, Mc, Mf, u, threshold=1.0)
        out, fb, e1 = sur.averaged_rhs(m, T, Mc, Mf, u, threshold=1.0)
        assert not fb
        errs_cheap.append(e0)
        errs_sur.append(e1)
    gain = np.mean(errs_cheap) / np.mean(errs_sur)
    print(f"surrogate r3 T=4h: error of M=8 {np.mean(errs_cheap):.3e}, "
          f"M=8 + network {np.mean(errs_sur):.3e}, gain {gain:.2f}x")
    assert gain >= 1.5
    # fallback: a threshold below the error hands back the M = 128 sum
    u = dev(state(o, seed=950, lmax=8))
    out, fb, e = sur.averaged_rhs(m, T, Mc, Mf, u, threshold=1e-12)
    assert fb and e > 1e-12
    assert np.array_equal(out.cpu().numpy(), m.averaged_rhs(T, Mf, u).cpu().numpy())
    out, fb, e = sur.averaged_rhs(m, T, Mc, Mf, u, check=False)
    assert not fb and e == -1.0
    zero.close()
    sur.close()
    m.close()


def test_surrogate_argument_errors():
    import torch
    from paper_2103_07706_gb300 import pavg
    sur = pavg.Surrogate(hidden=8)
    with pytest.raises(pavg.PavgError):
        sur.fit_scaling()  # no rows
    with pytest.raises(pavg.PavgError):
        sur.train(1)  # not scaled
    with pytest.raises(ValueError):
        sur.set_params(np.zeros(3, dtype=np.float32))
    with pytest.raises(pavg.PavgError):
        sur.set_scaling(np.zeros(124), np.zeros(124), np.zeros(15), np.ones(15))
    sur.close()
    del torch


def test_features_and_apply_at_refinement6():
    """The benchmark's inference size: GPU features of every cell and the
    applied correction on every DOF against the oracle at refinement 6."""
    from oracle.assembly import Assembly
    from oracle.mesh import build_mesh
    from paper_2103_07706_gb300 import pavg
    from paper_2103_07706_gb300.inputs import harmonic_state, lambda_max_for
    m = pavg.Model(6, lambda_max=lambda_max_for(6))
    mesh = build_mesh(6, 6.37122e6)
    asm = Assembly(mesh, 7.292e-5, 6.37122e6)
    U, _ = harmonic_state(mesh.verts, mesh.cells, 11, 16)
    V, _ = harmonic_state(mesh.verts, mesh.cells, 12, 16)
    sur = pavg.Surrogate(hidden=32, seed=6)
    X = sur.features(m, dev(U), dev(V)).cpu().numpy()
    want = S.features(asm, U, V)
    assert np.allclose(X, want, rtol=1e-6, atol=1e-6 * np.abs(want).max(axis=0))
    rng = np.random.default_rng(6)
    mx, sx = want.mean(axis=0).astype(np.float32), (want.std(axis=0) + 1e-3).astype(np.float32)
    my, sy = rng.standard_normal(S.N_OUT).astype(np.float32), (0.5 + rng.random(S.N_OUT)).astype(np.float32)
    sur.set_scaling(mx, sx, my, sy)
    p = _blocks(sur.params(), 32)
    got = sur.apply(m, dev(U), dev(V)).cpu().numpy() - V
    corr = S.apply(asm, p, tuple(a.astype(np.float64) for a in (mx, sx, my, sy)), U, V) - V
    assert np.abs(got - corr).max() <= 1e-5 * np.abs(corr).max()
    sur.close()
    m.close()


def test_scratch_follows_the_context_not_its_address():
    """A context created after another was destroyed may reuse its address;
    the surrogate's per-context scratch must follow the new context's mesh."""
    from paper_2103_07706_gb300 import pavg
    sur = pavg.Surrogate(hidden=8)
    o2, o3 = orc(2), orc(3)
    for r, o in ((2, o2), (3, o3), (2, o2)):
        m = pavg.Model(r, lambda_max=LAM[r])
        U = state(o, seed=5)
        X = sur.features(m, dev(U), dev(U)).cpu().numpy()
        assert X.shape == (m.n_cells, S.N_IN)
        assert np.allclose(X, S.features(o.ops.asm, U, U), rtol=1e-6, atol=1e-6)
        m.close()
    sur.close()


def _bf16(x):
    """Round float32 values to bfloat16 (nearest, ties to even), kept as float32."""
    b = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32)


def test_bf16_tensor_core_inference_matches_bf16_arithmetic():
    """BF16 inference (tensor cores, FP32 accumulation) against the same
    network evaluated in numpy with every GEMM operand rounded to BF16."""
    from paper_2103_07706_gb300 import pavg
    m, o = _model(2), orc(2)
    U = state(o, seed=13, eta_noise=5.0)
    V = state(o, seed=14, eta_noise=2.0)
    sur = pavg.Surrogate(hidden=64, seed=15)
    X = S.features(o.ops.asm, U, V)
    mx, sx = X.mean(axis=0).astype(np.float32), (X.std(axis=0) + 1e-3).astype(np.float32)
    my, sy = np.zeros(S.N_OUT, np.float32), np.ones(S.N_OUT, np.float32)
    sur.set_scaling(mx, sx, my, sy)
    p = {k: v.astype(np.float32) for k, v in _blocks(sur.params(), 64).items()}
    Xs = sur.features(m, dev(U), dev(V), standardised=True).cpu().numpy()
    H1 = np.tanh(_bf16(Xs) @ _bf16(p["W1"]).T + p["b1"]).astype(np.float32)
    H2 = np.tanh(_bf16(H1) @ _bf16(p["W2"]).T + p["b2"]).astype(np.float32)
    Y = (_bf16(H2) @ _bf16(p["W3"]).T + p["b3"]).astype(np.float64)
    want = S.scatter(o.ops.asm, Y)
    got = sur.apply(m, dev(U), dev(V), bf16=True).cpu().numpy() - V
    # the hidden activations are rounded to BF16 too, so FP32 summation-order
    # differences occasionally flip a rounding by one BF16 step (2^-8); a
    # wrong fragment layout would give O(1) errors
    assert np.linalg.norm(got - want) <= 1e-3 * np.linalg.norm(want)
    assert np.abs(got - want).max() <= 1e-2 * np.abs(want).max()
    sur.close()
    m.close()
