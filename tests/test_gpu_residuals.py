"""GPU parity of the ADMM residuals recon_info reports, against the FP64 oracle
on its own iterates (every prior: temporal TV, the spatio-temporal R and
volumes, the DFT and the Haar frame).

Algorithm 2 (temporal TV, oracle.tv_residuals): primal sqrt(||v - D_t m||^2 +
||m - x||^2) and dual sqrt(mu1^2 ||D_t dm||^2 + mu2^2 ||dm||^2), dm = m_K -
m_{K-1}.  Algorithm 1 (temporal DFT or the Haar frame,
oracle.synthesis_residuals): primal ||w - v|| and dual mu ||w_K - w_{K-1}||.

Bound: the GPU state matches the oracle's to 1e-5 relative (the parity bar),
and each residual is a norm of differences of state fields, so it may differ
by a few times 1e-5 of the fields' norms: |r - r_ref| <= 4e-5 (sum of the
fields' norms) + 1e-4 r_ref, the field term scaled by the residual's weight.
"""

import numpy as np
import pytest

import oracle
import synthdata

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def gpu(x):
    return torch.from_numpy(np.asarray(x, dtype=np.complex64)).cuda()


def case64(name="tiny", **over):
    c = synthdata.make_case(name, **over)
    c.kspace = np.asarray(c.kspace, dtype=np.complex64).astype(np.complex128)
    c.sens = np.asarray(c.sens, dtype=np.complex64).astype(np.complex128)
    return c


def check(info, oinfo, xr, mu):
    _, m, _, _ = oinfo["state"]
    scale = np.linalg.norm(xr) + np.linalg.norm(m)
    for got, ref, w in ((info.primal_res, oinfo["primal_res"], 1.0), (info.dual_res, oinfo["dual_res"], mu)):
        assert np.isfinite(got)
        assert abs(got - ref) <= 4e-5 * w * 4 * scale + 1e-4 * ref, (got, ref)


@pytest.mark.parametrize("iters", [1, 2, 50])
def test_tv_residuals_match_oracle(iters):
    from paper_1203_4587_gb300 import Plan
    c = case64("tiny")
    P = Plan(c.mask.astype(np.uint8), gpu(c.sens), c.lam, c.mu, prior="tv", rho=c.rho, max_iters=iters)
    _, info = P.solve(gpu(c.kspace))
    prob = oracle.Problem(c.kspace, c.sens, c.mask, c.mu)
    xr, oinfo = prob.solve("tv", c.lam, c.mu, c.rho, iters, objective=False)
    check(info, oinfo, xr, c.mu / c.rho)


def test_batched_tv_residuals_per_slice():
    from paper_1203_4587_gb300 import Batch, Plan
    cases = [case64("tiny", Nx=24, Ny=32, Nt=4, Nc=2, seed=81), case64("tiny", Nx=40, Ny=48, Nt=6, Nc=3, seed=82)]
    plans = [Plan(c.mask.astype(np.uint8), gpu(c.sens), c.lam, c.mu, prior="tv", rho=c.rho, max_iters=10)
             for c in cases]
    b = Batch(plans)
    b.solve([gpu(c.kspace) for c in cases])
    for c, info in zip(cases, b.info()):
        prob = oracle.Problem(c.kspace, c.sens, c.mask, c.mu)
        xr, oinfo = prob.solve("tv", c.lam, c.mu, c.rho, 10, objective=False)
        check(info, oinfo, xr, c.mu / c.rho)


def check_dft(info, oinfo, xr, mu):
    w, d = oinfo["state"]
    scale = np.linalg.norm(xr) + np.linalg.norm(w) + np.linalg.norm(d)
    for got, ref, wt in ((info.primal_res, oinfo["primal_res"], 1.0), (info.dual_res, oinfo["dual_res"], mu)):
        assert np.isfinite(got)
        assert abs(got - ref) <= 4e-5 * wt * 4 * scale + 1e-4 * ref, (got, ref)


@pytest.mark.parametrize("iters", [1, 2, 30])
def test_dft_residuals_match_oracle(iters):
    from paper_1203_4587_gb300 import Plan
    c = case64("tiny")
    P = Plan(c.mask.astype(np.uint8), gpu(c.sens), c.lam, c.mu, prior="dft", max_iters=iters)
    _, info = P.solve(gpu(c.kspace))
    prob = oracle.Problem(c.kspace, c.sens, c.mask, c.mu)
    xr, oinfo = prob.solve("dft", c.lam, c.mu, iters=iters, objective=False)
    check_dft(info, oinfo, xr, c.mu)


def test_batched_dft_residuals_per_slice_and_odd_frames():
    """Slices of different sizes in one launch, Nt = 5 and 6 (radix-5 and mixed
    stages), and a pixel count that is not a multiple of the 16-pixel tile."""
    from paper_1203_4587_gb300 import Batch, Plan
    cases = [case64("tiny", Nx=24, Ny=33, Nt=5, Nc=2, seed=84), case64("tiny", Nx=40, Ny=48, Nt=6, Nc=3, seed=85)]
    plans = [Plan(c.mask.astype(np.uint8), gpu(c.sens), c.lam, c.mu, prior="dft", max_iters=7) for c in cases]
    b = Batch(plans)
    b.solve([gpu(c.kspace) for c in cases])
    for c, info in zip(cases, b.info()):
        prob = oracle.Problem(c.kspace, c.sens, c.mask, c.mu)
        xr, oinfo = prob.solve("dft", c.lam, c.mu, iters=7, objective=False)
        check_dft(info, oinfo, xr, c.mu)


@pytest.mark.parametrize("iters,levels", [(1, 2), (2, 1), (20, 3)])
def test_haar_residuals_match_oracle(iters, levels):
    """The redundant Haar frame: w is not stored, the residuals come from u,
    s = Psi'u and xhat of the last two iterations (Psi'Psi = I)."""
    from paper_1203_4587_gb300 import Plan
    c = case64("tiny", Nx=24, Ny=40, Nt=6, Nc=3, seed=86)
    P = Plan(c.mask.astype(np.uint8), gpu(c.sens), c.lam, c.mu, prior="haar", frame_levels=levels, max_iters=iters)
    _, info = P.solve(gpu(c.kspace))
    prob = oracle.Problem(c.kspace, c.sens, c.mask, c.mu)
    xr, oinfo = prob.solve("haar", c.lam, c.mu, iters=iters, objective=False, levels=levels)
    check_dft(info, oinfo, xr, c.mu)


def check_stv(info, oinfo, xr, mu1):
    _, m, d1, _ = oinfo["state"]
    scale = np.linalg.norm(xr) + np.linalg.norm(m) + sum(np.linalg.norm(c) for c in d1)
    for got, ref, w in ((info.primal_res, oinfo["primal_res"], 1.0), (info.dual_res, oinfo["dual_res"], mu1)):
        assert np.isfinite(got)
        assert abs(got - ref) <= 4e-5 * w * 4 * scale + 1e-4 * ref, (got, ref)


@pytest.mark.parametrize("iters,ws", [(1, 1.0), (2, 0.5), (12, 1.0)])
def test_stv_residuals_match_oracle(iters, ws):
    """Algorithm 2 with the spatio-temporal R (oracle.stacked_residuals): the
    finishing kernels of iterations K-1 and K keep d1 and sum its change
    (v_K - R m_K = d1_{K-1} - d1_K), and a pass after the loop sums
    ||m_K - x_K||^2, ||dm||^2 and ||R dm||^2 from m_{K-1} copied aside."""
    from paper_1203_4587_gb300 import Plan
    c = case64("tiny", Nx=24, Ny=32, Nt=5, Nc=2, seed=87)
    P = Plan(c.mask.astype(np.uint8), gpu(c.sens), c.lam, c.mu, prior="stv", rho=c.rho, max_iters=iters,
             spatial_weight=ws, cg_steps=4)
    _, info = P.solve(gpu(c.kspace))
    prob = oracle.Problem(c.kspace, c.sens, c.mask, c.mu)
    xr, oinfo = prob.solve("stv", c.lam, c.mu, c.rho, iters, objective=False, ws=ws, cg=4)
    check_stv(info, oinfo, xr, c.mu / c.rho)


def test_volume_residuals_match_oracle():
    """A volume of 3 slices: every slice reports the volume's residuals (sums
    over all slices, z-differences included)."""
    from paper_1203_4587_gb300 import Plan, Volume
    cases = [case64("tiny", Nx=24, Ny=32, Nt=4, Nc=2, R=2, seed=70 + z) for z in range(3)]
    iters, ws, wz, cg = 8, 0.8, 0.6, 4
    plans = [Plan(c.mask.astype(np.uint8), gpu(c.sens), c.lam, c.mu, prior="stv", rho=c.rho, max_iters=iters,
                  spatial_weight=ws, cg_steps=cg) for c in cases]
    V = Volume(plans, wz)
    V.solve([gpu(c.kspace) for c in cases])
    probs = [oracle.Problem(c.kspace, c.sens, c.mask, c.mu) for c in cases]
    c0 = cases[0]
    xr, oinfo = oracle.admm_analysis_stv_volume([p.b for p in probs], [p.inv for p in probs], c0.lam, c0.mu, c0.rho,
                                                iters, ws=ws, wz=wz, cg=cg)
    for info in V.info():
        check_stv(info, oinfo, xr, c0.mu / c0.rho)


def test_residuals_nan_where_not_defined():
    from paper_1203_4587_gb300 import Plan
    c = case64("tiny", Nx=24, Ny=32, Nt=4, Nc=2, seed=83)
    Q = Plan(c.mask.astype(np.uint8), gpu(c.sens), c.lam, c.mu, prior="tv", rho=c.rho, max_iters=200, tol=1e-2)
    _, info = Q.solve(gpu(c.kspace))
    assert info.stopped == 1 and np.isnan(info.primal_res) and np.isnan(info.dual_res)
    S = Plan(c.mask.astype(np.uint8), gpu(c.sens), c.lam, c.mu, prior="stv", rho=c.rho, max_iters=200, tol=1e-2)
    _, info = S.solve(gpu(c.kspace))
    assert info.stopped == 1 and np.isnan(info.primal_res) and np.isnan(info.dual_res)
