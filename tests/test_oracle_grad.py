"""Pins of the oracle gradient of unrolled Algorithm 2 by central finite differences (FP64)."""

import numpy as np
import pytest

import oracle
import synthdata


def _case(seed=3, Nx=6, Ny=8, Nt=4, Nc=2):
    return synthdata.make_case("tiny", Nx=Nx, Ny=Ny, Nt=Nt, Nc=Nc, R=2, seed=seed, lam=0.05, mu=0.2, noise=0.05)


def _loss(case, y, lam, mu, iters):
    inv = oracle.ColumnInverse(case.sens, case.mask, mu)
    b = oracle.adjoint_op(y, case.sens, case.mask)
    xK = oracle.unrolled_tv_forward(b, inv, lam, mu, case.rho, iters)[-1][0]
    return float(np.vdot(xK - case.x_true, xK - case.x_true).real)


def test_soft_threshold_adjoint_matches_fd():
    rng = np.random.default_rng(0)
    tau = 0.3
    a = (rng.standard_normal(50) + 1j * rng.standard_normal(50))
    a = a[np.abs(np.abs(a) - tau) > 0.05]          # keep clear of the kink
    vb = rng.standard_normal(a.shape) + 1j * rng.standard_normal(a.shape)
    ab, tb = oracle.grad._soft_adjoint(a, vb, tau)
    h = 1e-7
    for comp in (1.0, 1j):                          # derivative along Re and Im of a
        d = (oracle.soft(a + h * comp, tau) - oracle.soft(a - h * comp, tau)) / (2 * h)
        fd = np.real(np.conj(vb) * d)               # <vbar, dv/da_comp>
        an = np.real(ab) if comp == 1.0 else np.imag(ab)
        np.testing.assert_allclose(an, fd, rtol=1e-6, atol=1e-8)
    dt = (oracle.soft(a, tau + h) - oracle.soft(a, tau - h)) / (2 * h)
    assert abs(tb - float(np.sum(np.real(np.conj(vb) * dt)))) < 1e-6 * max(1.0, abs(tb))


@pytest.mark.parametrize("iters", [1, 5])
def test_unrolled_gradient_matches_central_differences(iters):
    case = _case()
    lam, mu = case.lam, case.mu
    L, gy, gl, gm, _ = oracle.unrolled_tv_loss_and_grad(case.kspace, case.sens, case.mask, case.x_true, lam, mu,
                                                        case.rho, iters)
    assert abs(L - _loss(case, case.kspace, lam, mu, iters)) < 1e-12 * L
    rng = np.random.default_rng(1)
    sel = np.broadcast_to(case.mask[:, None, :, None], case.kspace.shape)
    assert np.all(gy[~sel] == 0)                    # unsampled entries do not reach the loss
    h = 1e-6
    for _ in range(3):
        dy = (rng.standard_normal(gy.shape) + 1j * rng.standard_normal(gy.shape)) * sel
        fd = (_loss(case, case.kspace + h * dy, lam, mu, iters) - _loss(case, case.kspace - h * dy, lam, mu, iters)) / (2 * h)
        an = float(np.vdot(gy, dy).real)            # dL = Re <grad, dy>
        assert abs(an - fd) <= 1e-6 * max(abs(fd), 1e-3), (an, fd)
    fdl = (_loss(case, case.kspace, lam + h, mu, iters) - _loss(case, case.kspace, lam - h, mu, iters)) / (2 * h)
    assert abs(gl - fdl) <= 1e-6 * max(abs(fdl), 1e-3), (gl, fdl)
    fdm = (_loss(case, case.kspace, lam, mu + h, iters) - _loss(case, case.kspace, lam, mu - h, iters)) / (2 * h)
    assert abs(gm - fdm) <= 1e-6 * max(abs(fdm), 1e-3), (gm, fdm)


def test_gradient_separates_over_columns():
    """Loss and gradients are sums over columns: two disjoint column sets add up to the full run."""
    case = _case(Nx=6)
    L, _, gl, gm, bb = oracle.unrolled_tv_loss_and_grad(case.kspace, case.sens, case.mask, case.x_true, case.lam,
                                                        case.mu, case.rho, 3)
    parts = []
    for cols in (np.array([0, 2, 5]), np.array([1, 3, 4])):
        P = oracle.Problem(case.kspace, case.sens, case.mask, case.mu, cols)
        parts.append((cols, oracle.unrolled_tv_adjoint(P.b, P.inv, case.x_true[:, :, cols], case.lam, case.mu,
                                                       case.rho, 3)))
    assert abs(sum(p[1][0] for p in parts) - L) < 1e-12 * L
    assert abs(sum(p[1][2] for p in parts) - gl) < 1e-10 * max(1.0, abs(gl))
    assert abs(sum(p[1][3] for p in parts) - gm) < 1e-10 * max(1.0, abs(gm))
    for cols, (_, bbc, _, _) in parts:
        np.testing.assert_allclose(bbc, bb[:, :, cols], atol=1e-12)


@pytest.mark.parametrize("iters", [1, 4])
def test_forward_is_algorithm_2(iters):
    """The unrolled forward runs Algorithm 2 exactly: after K steps its state
    (x, m, d1, d2) is that of oracle.admm_analysis_tv, which the KKT and
    closed-form pins fix independently."""
    case = _case()
    P = oracle.Problem(case.kspace, case.sens, case.mask, case.mu)
    states = oracle.unrolled_tv_forward(P.b, P.inv, case.lam, case.mu, case.rho, iters)
    _, info = oracle.admm_analysis_tv(P.b, P.inv, case.lam, case.mu, case.rho, iters)
    for a, b in zip(states[-1], info["state"]):
        np.testing.assert_allclose(a, b, atol=1e-12 * max(1.0, np.abs(b).max()))
