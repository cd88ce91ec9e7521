"""Failure detection on the GPU without a fault.

Every hand-off inside the persistent kernels waits on an mbarrier phase with
a wall-clock limit.  recon_selftest_wait_timeout runs that same bounded wait
on a phase nothing completes (a barrier that nothing arrives at) with a short
limit: the wait must give up, the call must report RECON_ERR_TIMEOUT, and the
context must stay usable for a normal solve afterwards.
"""

import numpy as np
import pytest

import oracle
import synthdata

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RECON_ERR_TIMEOUT = 5


@pytest.mark.parametrize("limit_us", [1000, 20000])
def test_bounded_wait_gives_up_and_reports(limit_us):
    from paper_1203_4587_gb300 import binding
    st, ms = binding.selftest_wait_timeout(limit_us)
    assert st == RECON_ERR_TIMEOUT
    assert ms >= 0.9 * limit_us / 1e3          # it did wait out its limit
    assert ms < limit_us / 1e3 + 2000.0         # and no longer than the limit plus launch overheads


def test_context_usable_after_timeout():
    from paper_1203_4587_gb300 import Plan, binding
    st, _ = binding.selftest_wait_timeout(2000)
    assert st == RECON_ERR_TIMEOUT
    case = synthdata.make_case("tiny", Nx=32, Ny=32, Nt=4, Nc=2, seed=61)
    k64 = case.kspace.astype(np.complex64)
    s64 = case.sens.astype(np.complex64)
    P = Plan(case.mask.astype(np.uint8), torch.from_numpy(s64).cuda(), case.lam, case.mu, rho=case.rho, max_iters=8)
    x, info = P.solve(torch.from_numpy(k64).cuda())
    prob = oracle.Problem(k64.astype(np.complex128), s64.astype(np.complex128), case.mask, case.mu)
    xr, _ = prob.solve("tv", case.lam, case.mu, case.rho, 8, objective=False)
    xg = x.cpu().numpy().astype(np.complex128)
    assert info.iters == 8
    assert np.linalg.norm(xg - xr) / np.linalg.norm(xr) < 1e-5
