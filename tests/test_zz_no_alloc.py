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
