"""Shift groups of the phase average (Sec. 2.5: the independent Riemann terms
are split over process groups whose partial sums are reduced once), emulated
on one GPU: each group's partial sum through pavg_averaged_rhs_group against
the oracle's literal partial sum, and the fixed-order sum of a partition
against the whole average."""

import numpy as np
import pytest

from tests.test_gpu_parity import assert_close, dev, gpu, orc, state

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("r,T,M,m0,m1", [(2, 3600.0, 8, 0, 3), (2, 3600.0, 8, 3, 5), (3, 1800.0, 6, 5, 6),
                                          (3, 7200.0, 16, 4, 12)])
def test_group_parity(r, T, M, m0, m1):
    from oracle import averaging
    g, o = gpu(r), orc(r)
    U = state(o, eta_noise=5.0)
    want = averaging.averaged_rhs_group(o, T, M, m0, m1, U)
    assert_close(o, g.averaged_rhs_group(T, M, m0, m1, dev(U)).cpu().numpy(), want)
    g.sync()


@pytest.mark.parametrize("r,T,M,G", [(3, 3600.0, 8, 2), (3, 3600.0, 16, 3), (4, 7200.0, 16, 4), (3, 0.0, 4, 2)])
def test_partition_sums_to_the_whole_average(r, T, M, G):
    import torch

    from paper_2103_07706_gb300 import shift_groups
    g, o = gpu(r), orc(r)
    Ud = dev(state(o))
    full = g.averaged_rhs(T, M, Ud).cpu().numpy()
    tot = torch.zeros_like(Ud)
    for m0, m1 in shift_groups.groups(M, G):
        tot += g.averaged_rhs_group(T, M, m0, m1, Ud)
    g.sync()
    assert_close(o, tot.cpu().numpy(), full, tol=1e-13)


def test_group_arguments_are_checked():
    from paper_2103_07706_gb300 import pavg
    g = gpu(2)
    Ud = dev(np.zeros(g.n))
    for m0, m1 in [(-1, 2), (3, 3), (2, 9), (5, 4)]:
        with pytest.raises(pavg.PavgError):
            g.averaged_rhs_group(3600.0, 8, m0, m1, Ud)
