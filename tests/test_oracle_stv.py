"""Pins of the oracle's spatio-temporal analysis operator, its CG m-update and
Algorithm 2 with it (CPU, no GPU).

None of these re-derive the code under test:
* R and R' are adjoint (inner products on random fields, several shapes,
  including length-1 axes);
* (rho I + R'R) equals a dense matrix assembled from Kronecker products of
  one-dimensional difference matrices;
* CG reaches the dense solve once it has taken as many steps as the system
  has unknowns, and converges to the closed form given by the DCT-II, which
  diagonalises every non-circular difference Laplacian D'D (eigenvalues
  2 - 2 cos(pi k / n));
* CG's error in the energy norm never grows from step to step;
* with w = 0 and enough CG steps, Algorithm 2 reduces to the temporal-TV
  oracle (Thomas / dense m-update);
* the converged ADMM point satisfies the KKT conditions of
  lambda ||R x||_1 + ||y - H x||^2 on a tiny problem.
"""

import functools

import numpy as np
import pytest
import scipy.fft

import oracle
from test_oracle_pins import _small_case


def _rand(rng, shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def _D(n):
    D = np.zeros((max(n - 1, 0), n))
    for k in range(n - 1):
        D[k, k], D[k, k + 1] = -1.0, 1.0
    return D


def _dense_M(shape, rho, ws):
    """rho I + R'R for x[t, j, i] flattened C-order, from Kronecker products."""
    Nt, Ny, Nx = shape
    It, Iy, Ix = np.eye(Nt), np.eye(Ny), np.eye(Nx)
    Lt, Ly, Lx = (_D(n).T @ _D(n) for n in (Nt, Ny, Nx))
    L = np.kron(np.kron(Lt, Iy), Ix) + ws ** 2 * (np.kron(np.kron(It, Ly), Ix) + np.kron(np.kron(It, Iy), Lx))
    return rho * np.eye(Nt * Ny * Nx) + L


@pytest.mark.parametrize("shape", [(4, 5, 6), (1, 3, 4), (5, 1, 3), (3, 4, 1), (2, 2, 2)])
@pytest.mark.parametrize("ws", [1.0, 0.37])
def test_R_adjoint(shape, ws):
    rng = np.random.default_rng(sum(shape))
    x = _rand(rng, shape)
    Rx = oracle.stv_R(x, ws)
    u = tuple(_rand(rng, c.shape) for c in Rx)
    lhs = sum(np.vdot(a, b) for a, b in zip(Rx, u))
    rhs = np.vdot(x, oracle.stv_Radj(u, ws, shape))
    assert abs(lhs - rhs) < 1e-12 * max(1.0, abs(lhs))


@pytest.mark.parametrize("shape", [(3, 4, 5), (1, 3, 2), (4, 1, 3)])
@pytest.mark.parametrize("ws", [1.0, 0.5, 0.0])
def test_M_equals_kronecker_assembly(shape, ws):
    rho = 0.5
    n = int(np.prod(shape))
    cols = []
    for k in range(n):
        e = np.zeros(n, complex)
        e[k] = 1.0
        cols.append(oracle.stv_M(e.reshape(shape), rho, ws).ravel())
    np.testing.assert_allclose(np.stack(cols, axis=1), _dense_M(shape, rho, ws), atol=1e-14)


def test_cg_exact_after_n_steps():
    shape, rho, ws = (2, 3, 4), 0.5, 1.0
    rng = np.random.default_rng(3)
    rhs, m0 = _rand(rng, shape), _rand(rng, shape)
    exact = np.linalg.solve(_dense_M(shape, rho, ws), rhs.ravel()).reshape(shape)
    m = oracle.cg_steps(lambda a: oracle.stv_M(a, rho, ws), rhs, m0, int(np.prod(shape)))
    np.testing.assert_allclose(m, exact, atol=1e-10 * np.abs(exact).max())


def _dct_solve(rhs, rho, ws):
    """(rho I + R'R)^{-1} rhs by the DCT-II diagonalisation of each D'D."""
    Nt, Ny, Nx = rhs.shape
    lam = [2.0 - 2.0 * np.cos(np.pi * np.arange(n) / n) for n in (Nt, Ny, Nx)]
    den = rho + lam[0][:, None, None] + ws ** 2 * (lam[1][None, :, None] + lam[2][None, None, :])
    c = scipy.fft.dctn(rhs, type=2, norm="ortho")
    return scipy.fft.idctn(c / den, type=2, norm="ortho")


@pytest.mark.parametrize("ws", [1.0, 0.3])
def test_cg_converges_to_dct_closed_form(ws):
    shape, rho = (7, 6, 9), 0.5
    rng = np.random.default_rng(4)
    rhs = _rand(rng, shape)
    m = oracle.cg_steps(lambda a: oracle.stv_M(a, rho, ws), rhs, np.zeros(shape, complex), 120)
    exact = _dct_solve(rhs, rho, ws)
    np.testing.assert_allclose(m, exact, atol=1e-9 * np.abs(exact).max())


def test_cg_energy_error_never_grows():
    shape, rho, ws = (6, 8, 8), 0.5, 1.0
    rng = np.random.default_rng(5)
    rhs, m0 = _rand(rng, shape), _rand(rng, shape)
    exact = _dct_solve(rhs, rho, ws)

    def energy(m):
        e = m - exact
        return np.vdot(e, oracle.stv_M(e, rho, ws)).real

    errs = [energy(oracle.cg_steps(lambda a: oracle.stv_M(a, rho, ws), rhs, m0, s)) for s in range(0, 12)]
    assert all(b <= a * (1 + 1e-12) for a, b in zip(errs, errs[1:]))
    assert errs[-1] < 1e-3 * errs[0]


def test_zero_spatial_weight_is_temporal_tv():
    x, sens, mask, y = _small_case(Nx=5, Ny=6, Nt=5, Nc=2, R=2, noise=0.02, seed=21)
    lam, mu, rho, iters = 0.02, 0.1, 0.5, 15
    P = oracle.Problem(y, sens, mask, mu)
    xt, it = oracle.admm_analysis_tv(P.b, P.inv, lam, mu, rho, iters, fid=P.fid)
    # global CG on a system that decouples per pixel: at most Nt distinct eigenvalues
    xs, is_ = oracle.admm_analysis_stv(P.b, P.inv, lam, mu, rho, iters, ws=0.0, cg=x.shape[0] + 1, fid=P.fid)
    np.testing.assert_allclose(xs, xt, atol=1e-10 * np.abs(xt).max())
    np.testing.assert_allclose(is_["J"], it["J"], rtol=1e-10)
    # R = (D_t, 0, 0): the stacked residuals are the temporal-TV ones
    for key in ("primal_res", "dual_res"):
        assert abs(is_[key] - it[key]) <= 1e-9 * it[key]


@functools.lru_cache(maxsize=1)
def _stv_converged():
    x, sens, mask, y = _small_case(Nx=4, Ny=4, Nt=4, Nc=2, R=2, noise=0.05, seed=18)
    lam, mu, rho, ws = 0.05, 0.1, 0.5, 0.8
    P = oracle.Problem(y, sens, mask, mu)
    xr, info = oracle.admm_analysis_stv(P.b, P.inv, lam, mu, rho, 3000, ws=ws, cg=70)
    return x, sens, mask, y, lam, mu, rho, ws, xr, info


def test_kkt_stv_on_tiny_problem():
    """2 H'(Hx - y) + lambda R' g = 0, g = 2 mu1 d1 / lambda in the subdifferential of ||.||_1 at R x."""
    x, sens, mask, y, lam, mu, rho, ws, xr, info = _stv_converged()
    _, m, d1, d2 = info["state"]
    np.testing.assert_allclose(m, xr, atol=1e-9)                      # the split is tight at convergence
    mu1 = mu / rho
    g = tuple(2 * mu1 * d / lam for d in d1)
    Rx = oracle.stv_R(xr, ws)
    for gc, rc in zip(g, Rx):
        assert np.abs(gc).max() <= 1 + 1e-8
        # the sign condition on the clearly nonzero differences (the zeros sit at
        # |R x| ~ 1e-10; a few small ones near 1e-3 converge more slowly)
        big = np.abs(rc) > 1e-3
        assert big.sum() > 20
        np.testing.assert_allclose(gc[big], rc[big] / np.abs(rc[big]), atol=1e-6)
    grad = 2 * oracle.adjoint_op(oracle.forward_op(xr, sens, mask) - y, sens, mask)
    stat = grad + lam * oracle.stv_Radj(g, ws, xr.shape)
    assert np.linalg.norm(stat) < 1e-8 * max(1.0, np.linalg.norm(grad))


def test_stv_residuals_follow_the_duals_and_vanish():
    """Stacked residuals of Algorithm 2 with R = (D_t, w D_x, w D_y): the v - R m
    part equals the change of d1 in the last iteration (the d1-update), both are
    positive early on, and both decay towards the fixed point."""
    x, sens, mask, y = _small_case(Nx=4, Ny=5, Nt=4, Nc=2, R=2, noise=0.05, seed=23)
    lam, mu, rho, ws = 0.05, 0.1, 0.5, 0.8
    P = oracle.Problem(y, sens, mask, mu)
    _, i4 = oracle.admm_analysis_stv(P.b, P.inv, lam, mu, rho, 4, ws=ws, cg=3)
    _, i5 = oracle.admm_analysis_stv(P.b, P.inv, lam, mu, rho, 5, ws=ws, cg=3)
    assert i5["primal_res"] > 1e-6 and i5["dual_res"] > 1e-6
    x5, m5, d1_5, _ = i5["state"]
    d1_4 = i4["state"][2]
    part = np.sqrt(sum(np.vdot(a - b, a - b).real for a, b in zip(d1_4, d1_5)) + np.vdot(m5 - x5, m5 - x5).real)
    assert abs(part - i5["primal_res"]) <= 1e-12 * part
    # the converged run of the KKT test: a million-fold drop from iteration 5
    _, sens, mask, y, lam, mu, rho, ws, _, info = _stv_converged()
    P = oracle.Problem(y, sens, mask, mu)
    _, early = oracle.admm_analysis_stv(P.b, P.inv, lam, mu, rho, 5, ws=ws, cg=70)
    for key in ("primal_res", "dual_res"):
        assert info[key] < 1e-6 * early[key]


def test_volume_residuals_of_one_slice_are_the_2d_ones():
    x, sens, mask, y = _small_case(Nx=4, Ny=5, Nt=4, Nc=2, R=2, noise=0.05, seed=24)
    lam, mu, rho, ws = 0.05, 0.1, 0.5, 0.7
    P = oracle.Problem(y, sens, mask, mu)
    _, i2 = oracle.admm_analysis_stv(P.b, P.inv, lam, mu, rho, 6, ws=ws, cg=4)
    _, iv = oracle.admm_analysis_stv_volume([P.b], [P.inv], lam, mu, rho, 6, ws=ws, wz=1.3, cg=4)
    for key in ("primal_res", "dual_res"):
        assert abs(iv[key] - i2[key]) <= 1e-12 * i2[key]


def test_objective_is_lambda_l1_plus_fidelity():
    x, sens, mask, y = _small_case(Nx=3, Ny=4, Nt=3, Nc=2, R=2, seed=22)
    P = oracle.Problem(y, sens, mask, 0.1)
    ws = 0.6
    J = oracle.objective_stv(x, 0.3, ws, P.fid)
    l1 = 0.0
    for t in range(3):                                   # element by element, every difference
        for j in range(4):
            for i in range(3):
                if t + 1 < 3:
                    l1 += abs(x[t + 1, j, i] - x[t, j, i])
                if i + 1 < 3:
                    l1 += ws * abs(x[t, j, i + 1] - x[t, j, i])
                if j + 1 < 4:
                    l1 += ws * abs(x[t, j + 1, i] - x[t, j, i])
    assert abs(J - (0.3 * l1 + oracle.data_residual(x, y, sens, mask))) < 1e-10 * J


def test_column_subset_refused():
    x, sens, mask, y = _small_case(Nx=4, Ny=4, Nt=2, Nc=2, R=2, seed=23)
    P = oracle.Problem(y, sens, mask, 0.1, cols=[0, 2])
    with pytest.raises(ValueError):
        P.solve("stv", 0.01, 0.1, iters=2)


# --- 3D volumes: slices coupled by a z-difference --------------------------------------------

def _dense_M_vol(shape, rho, ws, wz):
    Nz, Nt, Ny, Nx = shape
    I = [np.eye(n) for n in shape]
    Lz, Lt, Ly, Lx = (_D(n).T @ _D(n) for n in shape)

    def k4(a, b, c, d):
        return np.kron(np.kron(np.kron(a, b), c), d)
    L = (k4(I[0], Lt, I[2], I[3]) + ws ** 2 * (k4(I[0], I[1], Ly, I[3]) + k4(I[0], I[1], I[2], Lx))
         + wz ** 2 * k4(Lz, I[1], I[2], I[3]))
    return rho * np.eye(int(np.prod(shape))) + L


@pytest.mark.parametrize("shape", [(3, 2, 4, 5), (1, 3, 2, 2), (4, 1, 3, 1)])
def test_volume_R_adjoint(shape):
    rng = np.random.default_rng(sum(shape) + 7)
    x = _rand(rng, shape)
    Rx = oracle.stv_R_vol(x, 0.7, 1.3)
    u = tuple(_rand(rng, c.shape) for c in Rx)
    lhs = sum(np.vdot(a, b) for a, b in zip(Rx, u))
    rhs = np.vdot(x, oracle.stv_Radj_vol(u, 0.7, 1.3, shape))
    assert abs(lhs - rhs) < 1e-12 * max(1.0, abs(lhs))


@pytest.mark.parametrize("wz", [1.0, 0.4, 0.0])
def test_volume_M_equals_kronecker_assembly(wz):
    shape, rho, ws = (3, 2, 3, 2), 0.5, 0.8
    n = int(np.prod(shape))
    cols = []
    for k in range(n):
        e = np.zeros(n, complex)
        e[k] = 1.0
        cols.append(oracle.stv_M_vol(e.reshape(shape), rho, ws, wz).ravel())
    np.testing.assert_allclose(np.stack(cols, axis=1), _dense_M_vol(shape, rho, ws, wz), atol=1e-14)


def test_volume_cg_converges_to_dct_closed_form():
    shape, rho, ws, wz = (4, 5, 6, 7), 0.5, 1.0, 0.6
    rng = np.random.default_rng(9)
    rhs = _rand(rng, shape)
    m = oracle.cg_steps(lambda a: oracle.stv_M_vol(a, rho, ws, wz), rhs, np.zeros(shape, complex), 150)
    lam = [2.0 - 2.0 * np.cos(np.pi * np.arange(n) / n) for n in shape]
    den = (rho + wz ** 2 * lam[0][:, None, None, None] + lam[1][None, :, None, None]
           + ws ** 2 * (lam[2][None, None, :, None] + lam[3][None, None, None, :]))
    exact = scipy.fft.idctn(scipy.fft.dctn(rhs, type=2, norm="ortho") / den, type=2, norm="ortho")
    np.testing.assert_allclose(m, exact, atol=1e-9 * np.abs(exact).max())


def test_volume_of_one_slice_is_the_2d_algorithm():
    x, sens, mask, y = _small_case(Nx=5, Ny=6, Nt=4, Nc=2, R=2, noise=0.02, seed=24)
    lam, mu, rho, iters = 0.02, 0.1, 0.5, 10
    P = oracle.Problem(y, sens, mask, mu)
    x2, i2 = oracle.admm_analysis_stv(P.b, P.inv, lam, mu, rho, iters, ws=0.9, cg=4, fid=P.fid)
    xv, iv = oracle.admm_analysis_stv_volume([P.b], [P.inv], lam, mu, rho, iters, ws=0.9, wz=2.0, cg=4,
                                             fids=[P.fid])
    np.testing.assert_allclose(xv[0], x2, atol=1e-12 * np.abs(x2).max())
    np.testing.assert_allclose(iv["J"], i2["J"], rtol=1e-12)


def test_kkt_volume_on_tiny_problem():
    """sum_z 2 H_z'(H_z x_z - y_z) + lambda R' g = 0 at the converged volume."""
    cases = [_small_case(Nx=3, Ny=4, Nt=3, Nc=2, R=2, noise=0.05, seed=s) for s in (31, 32)]
    lam, mu, rho, ws, wz = 0.05, 0.1, 0.5, 0.8, 1.2
    probs = [oracle.Problem(y, sens, mask, mu) for (_, sens, mask, y) in cases]
    xv, info = oracle.admm_analysis_stv_volume([p.b for p in probs], [p.inv for p in probs], lam, mu, rho, 3000,
                                               ws=ws, wz=wz, cg=80)
    _, m, d1, _ = info["state"]
    np.testing.assert_allclose(m, xv, atol=1e-9)
    g = tuple(2 * (mu / rho) * d / lam for d in d1)
    for gc in g:
        assert np.abs(gc).max() <= 1 + 1e-8
    grad = np.stack([2 * oracle.adjoint_op(oracle.forward_op(xz, sens, mask) - y, sens, mask)
                     for xz, (_, sens, mask, y) in zip(xv, cases)])
    stat = grad + lam * oracle.stv_Radj_vol(g, ws, wz, xv.shape)
    assert np.linalg.norm(stat) < 1e-8 * max(1.0, np.linalg.norm(grad))
