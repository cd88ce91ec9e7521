"""GPU checks of the plan phase: recon_plan_set_mu (a new mu on an existing
plan, Eq. eigen_mu) and the inversion's agreement with the oracle at the new
mu.

set_mu recomputes the inverses with the same kernel from the same device
inputs as recon_plan_create, so a plan moved to mu' equals a plan created at
mu', bit for bit (inverses and solves).
"""

import numpy as np
import pytest

import oracle
import synthdata

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def gpu(x):
    return torch.from_numpy(np.asarray(x, dtype=np.complex64)).cuda()


def plan(case, mu, prior="tv", **opts):
    from paper_1203_4587_gb300 import Plan
    opts.setdefault("max_iters", 12)
    return Plan(case.mask.astype(np.uint8), gpu(case.sens), case.lam, mu, prior=prior, rho=case.rho, **opts)


@pytest.mark.parametrize("prior", ["tv", "dft", "stv"])
@pytest.mark.parametrize("storage", ["fp32", "fp16"])
def test_set_mu_equals_fresh_plan(prior, storage):
    case = synthdata.make_case("tiny", Nx=40, Ny=48, Nt=6, Nc=3, seed=51)
    mu_new = 0.37
    P = plan(case, case.mu, prior, storage=storage)
    k = gpu(case.kspace)
    P.solve(k)                                   # used at the old mu first
    P.set_mu(mu_new)
    Q = plan(case, mu_new, prior, storage=storage)
    for i, t in ((0, 0), (17, 3), (39, 5)):
        np.testing.assert_array_equal(P.export_inverse(i, t).cpu().numpy(), Q.export_inverse(i, t).cpu().numpy())
    xp, ip = P.solve(k)
    xq, iq = Q.solve(k)
    np.testing.assert_array_equal(xp.cpu().numpy(), xq.cpu().numpy())
    assert abs(ip.J - iq.J) <= 1e-12 * abs(iq.J)   # J's FP64 sums are added across CTAs in any order


def test_set_mu_matches_oracle_inverse():
    case = synthdata.make_case("tiny", Nx=32, Ny=64, Nt=4, Nc=4, seed=52)
    P = plan(case, case.mu)
    mu_new = 0.05
    P.set_mu(mu_new)
    mu32 = float(np.float32(mu_new))
    sens = np.asarray(case.sens, dtype=np.complex64).astype(np.complex128)
    for i, t in ((3, 1), (30, 2)):
        Aref = oracle.inverse_blocks(oracle.gram_blocks(sens, case.mask, [i])[t, 0], mu32)
        A = P.export_inverse(i, t).cpu().numpy().astype(np.complex128)
        assert np.linalg.norm(A - Aref) / np.linalg.norm(Aref) < 2e-7


def test_batches_and_gradients_built_before_refuse():
    from paper_1203_4587_gb300 import Batch, Grad, ReconError
    case = synthdata.make_case("tiny", Nx=24, Ny=32, Nt=4, Nc=2, seed=53)
    P = plan(case, case.mu)
    b = Batch([P])
    g = Grad([P], checkpoint_every=4)
    k = gpu(case.kspace)
    b.solve([k])
    g.forward([k])
    P.set_mu(0.2)
    with pytest.raises(ReconError):
        b.solve([k])
    with pytest.raises(ReconError):
        g.forward([k])
    b2 = Batch([P])                               # rebuilt: runs, and agrees with the plan's own solve
    x_b = b2.solve([k])[0].cpu().numpy()
    x_p = P.solve(k)[0].cpu().numpy()
    np.testing.assert_array_equal(x_b, x_p)


def test_invalid_mu_leaves_plan_intact():
    from paper_1203_4587_gb300 import ReconError
    case = synthdata.make_case("tiny", Nx=16, Ny=32, Nt=3, Nc=2, seed=54)
    P = plan(case, case.mu)
    k = gpu(case.kspace)
    x0 = P.solve(k)[0].cpu().numpy()
    for bad in (0.0, -1.0, float("inf"), float("nan")):
        with pytest.raises(ReconError):
            P.set_mu(bad)
    np.testing.assert_array_equal(P.solve(k)[0].cpu().numpy(), x0)
