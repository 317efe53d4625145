"""Mixed-precision mode (PAVG_PRECISION_MIXED) against FP64 references.

The mode computes N, the forward shift contraction and the K-hat products of
L in FP32 arithmetic (with FP64 sums over the quadrature points and an FP64
cell divergence; the recurrences add the FP32 products in FP64), solves with
M1 by FP32 CG inside FP64 residual refinement stopped at a relative residual
of 1e-5, and keeps the Chebyshev recurrences, the weighted sum over shifts and
the timestep update in FP64.  Stated bounds, relative L2 per field in the
finite element norms (measured values in brackets):
  N, refinement 3               u, eta <= 1e-5     [2.9e-6, 2.0e-7]
  e^{tL}, refinement 3, 1 h     u, eta <= 1e-6     [2.5e-7, 2.0e-7]
  averaged_rhs, r4, M 16        u, eta <= 1e-5     [3.7e-6, 2.0e-6]
  two timesteps, r3, M 8        u, eta <= 1e-6     [1.3e-7, 9.2e-8]
  averaged_rhs, r6, M 64, 1 h   u <= 1e-5, eta <= 5e-4   [6.1e-6, 3.2e-4]
(with the K-hat products in FP64 the r6 errors were 3.3e-6 and 1.3e-4).
The refinement-6 eta bound is wider because the seeded state is geostrophic:
u is tangent to the contours of eta and divergence-free, so the exact eta
part of N is zero and what the FP64 path returns is discretisation residue,
small next to the individual flux terms that cancel to give it.  The sum over
shifts cancels a further factor of about 12 in eta (sum of w_m times the
shift norms over the norm of the sum).  FP32 rounding of those flux terms is
therefore large relative to the result while small relative to its parts.
"""

import numpy as np
import pytest

from tests.test_gpu_parity import LAM, dev, gpu, orc, rel, state

pytestmark = pytest.mark.gpu

MIXED = 1


def check(m, got, want, tol, what):
    ru, re = rel(m, got, want)
    print(f"mixed precision {what}: rel L2 u {ru:.2e} eta {re:.2e}")
    assert ru <= tol and re <= tol, (what, ru, re)


def test_mixed_nonlinear_and_exponential():
    g, o = gpu(3, precision=MIXED), orc(3)
    U = state(o, eta_noise=20.0)
    check(o, g.nonlinear(dev(U)).cpu().numpy(), o.N(U), 1e-5, "N r3")
    check(o, g.expL(3600.0, dev(U)).cpu().numpy(), o.expL(3600.0, U), 1e-6, "expL r3 t=1h")
    g.sync()


def test_mixed_averaged_rhs_vs_oracle():
    g, o = gpu(4, precision=MIXED), orc(4)
    U = state(o, eta_noise=5.0)
    check(o, g.averaged_rhs(3600.0, 16, dev(U)).cpu().numpy(), o.averaged_rhs(3600.0, 16, U), 1e-5,
          "averaged_rhs r4 M16 T1h")
    g.sync()


def test_mixed_timestep_vs_oracle():
    g, o = gpu(3, precision=MIXED), orc(3)
    U = state(o)
    want = o.timestep(900.0, 3600.0, 8, U, 2)
    Ud = dev(U)
    g.timestep(900.0, 3600.0, 8, Ud, 2)
    check(o, Ud.cpu().numpy(), want, 1e-6, "2 timesteps r3 M8 T1h")


def test_mixed_full_size_vs_fp64_gpu():
    """Refinement 6, M = 64, T = 1 h: the benchmark configuration."""
    from paper_2103_07706_gb300 import pavg
    from paper_2103_07706_gb300.inputs import harmonic_state
    g64 = pavg.Model(6, lambda_max=0.02335)
    gmx = pavg.Model(6, lambda_max=0.02335, precision=MIXED)
    v, c = g64.mesh()
    U, _ = harmonic_state(v, c, 2103, 16)
    Ud = dev(U)
    a = g64.averaged_rhs(3600.0, 64, Ud).cpu().numpy()
    b = gmx.averaged_rhs(3600.0, 64, Ud).cpu().numpy()
    g64.sync()
    gmx.sync()
    nu = g64.n_u
    du = np.linalg.norm(a[:nu] - b[:nu]) / np.linalg.norm(a[:nu])
    de = np.linalg.norm(a[nu:] - b[nu:]) / np.linalg.norm(a[nu:])
    print(f"mixed precision averaged_rhs r6 M64 vs FP64 GPU: rel l2 u {du:.2e} eta {de:.2e}")
    assert du <= 1e-5 and de <= 5e-4, (du, de)
    g64.close()
    gmx.close()


def test_mixed_at_rossby_0p1():
    """Mixed precision on a Rossby-0.1 state (refinement 4, M = 16, T = 1 h)
    against the oracle: the measured error is printed; bounds u <= 1e-5,
    eta <= 1e-4."""
    from paper_2103_07706_gb300.inputs import harmonic_state
    g, o = gpu(4, precision=MIXED), orc(4)
    U, _ = harmonic_state(o.mesh.verts, o.mesh.cells, 2103, 16, rossby=0.1)
    ru, re = rel(o, g.averaged_rhs(3600.0, 16, dev(U)).cpu().numpy(), o.averaged_rhs(3600.0, 16, U))
    print(f"mixed precision averaged_rhs r4 M16 T1h, Rossby 0.1: rel L2 u {ru:.2e} eta {re:.2e}")
    assert ru <= 1e-5 and re <= 1e-4, (ru, re)
    g.sync()
