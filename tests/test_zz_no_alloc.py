"""The MBAR solve that allocates no device memory (regc_mbar_solve_static).

It serves callers that cannot let a library allocate device memory, for
instance a framework that owns all device memory through its own pool, or a
loop that cannot afford the device-wide synchronisation of cudaMalloc and
cudaFree.  It solves the same equations as regc_mbar_solve on a fixed scratch
area compiled into the library (log-sum-exps of the energies, where the
allocating solve iterates on a kernel matrix it allocates).  These tests call it through the C ABI twice in a
row -- a larger problem, then a smaller one, so that anything the first call
left in the shared scratch area would show -- and compare each result with
regc_mbar_solve and with the FP64 oracle (oracle/mbar.py) at the tolerance of
the other MBAR tests.  The device's free memory is the same before and after
the second call (the first may load the library's device code).  This file is
collected last, so a run that stops at the first failure has run every other
test before it.
"""
import numpy as np
import pytest
import torch

from oracle import mbar as OM
from paper_1908_11118_gb300 import RegcError, mbar_solve
from paper_1908_11118_gb300 import build as B
from paper_1908_11118_gb300.regc import mbar_solve_static
from test_gpu_stats_mbar import synthetic_bins

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()


def test_static_solve_matches_allocating_solve_on_two_calls():
    for seed, side in ((0, 5), (1, 3)):
        kT, mu, omega, N, E, H, nmax = synthetic_bins(seed=seed, S_side=side)
        f_r, D_r, it_r = mbar_solve(kT, mu, 1.0, omega, N, E, H, tol=1e-11)
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        f_s, D_s, it_s = mbar_solve_static(kT, mu, 1.0, omega, N, E, H, tol=1e-11)
        torch.cuda.synchronize()
        if seed == 1:                       # the first call may load the device code
            assert torch.cuda.mem_get_info()[0] == free_before
        np.testing.assert_allclose(f_s, f_r, atol=1e-9)
        np.testing.assert_allclose(D_s, D_r, atol=1e-9)
        f_o, D_o, _, ok = OM.solve(kT, mu, 1.0, omega, N, E, H, tol=1e-12)
        assert ok
        np.testing.assert_allclose(f_s, f_o, atol=1e-9)
        np.testing.assert_allclose(D_s, D_o, atol=1e-9)
        # the allocating solve iterates on the kernel matrix, the static one on
        # log-sum-exps: the same fixed point, reached by Anderson paths that
        # differ by rounding (so in different numbers of maps); both converge
        assert 0 < it_s < 200000 and 0 < it_r < 200000


def test_static_solve_rejects_sizes_beyond_its_scratch():
    n = 4097
    with pytest.raises(RegcError) as err:
        mbar_solve_static(np.ones(n), np.zeros(n), 1.0, np.ones(n), np.zeros(1, np.int32),
                          np.zeros(1), np.ones(1))
    assert err.value.status == -1
