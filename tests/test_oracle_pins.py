"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: a closed
form, a brute-force computation on a tiny input, an invariant, or a textbook
special case.  Together they make a plausible slip anywhere in the oracle
(a dropped term, a wrong sign or conjugation, a transposed operand, a wrong
index) fail at least one test.
"""

import json
import os

import numpy as np
import pytest

import oracle
import synthdata

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rand_c(rng, shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def _small_case(Nx=6, Ny=8, Nt=3, Nc=2, R=2, seed=0, full=False, noise=0.0):
    rng = np.random.default_rng(seed)
    x = synthdata.make_phantom(Nx, Ny, Nt, rng, moving=1) + 0.05 * _rand_c(rng, (Nt, Ny, Nx))
    sens = synthdata.make_sens(Nx, Ny, Nc)
    if full:
        mask = np.ones((Nt, Ny), bool)
    else:
        mask = np.zeros((Nt, Ny), bool)
        for t in range(Nt):
            mask[t, rng.choice(Ny, size=max(1, Ny // R), replace=False)] = True
    y = synthdata.simulate_kspace(x, sens, mask, rng, noise=noise)
    return x, sens, mask, y


def _dense_H(sens, mask):
    """Brute force: the forward operator as an explicit matrix (columns H e_n)."""
    Nc, Ny, Nx = sens.shape
    Nt = mask.shape[0]
    n = Nt * Ny * Nx
    cols = []
    for idx in range(n):
        e = np.zeros(n, complex)
        e[idx] = 1.0
        cols.append(oracle.forward_op(e.reshape(Nt, Ny, Nx), sens, mask).ravel())
    return np.stack(cols, axis=1)


# --- Section III: soft threshold --------------------------------------------
def test_soft_threshold_special_values():
    tau = 0.3
    a = np.array([0.0, 0.3, -0.3j, 0.2 + 0.2j, 0.3 * np.exp(0.7j)])
    out = oracle.soft(a, tau)
    # |a| <= tau -> exactly 0 (including a = 0 and |a| = tau)
    assert np.all(out == 0)
    b = np.array([1.0, -2.0j, 3 * np.exp(1.1j)])
    ob = oracle.soft(b, tau)
    np.testing.assert_allclose(np.abs(ob), np.abs(b) - tau, rtol=0, atol=1e-15)
    np.testing.assert_allclose(np.angle(ob), np.angle(b), atol=1e-15)


def test_soft_threshold_is_the_prox_by_grid_search():
    """S(a, tau) minimises tau|v| + 1/2 |v - a|^2 (checked by brute force)."""
    rng = np.random.default_rng(3)
    tau = 0.4
    g = np.linspace(-2.5, 2.5, 1001)
    V = g[None, :] + 1j * g[:, None]
    for a in list(_rand_c(rng, 6) * 0.8) + [0.35 + 0.2j, 0.0]:
        f = tau * np.abs(V) + 0.5 * np.abs(V - a) ** 2
        vbest = V.flat[np.argmin(f)]
        assert abs(vbest - oracle.soft(np.array([a]), tau)[0]) < 1.5 * (g[1] - g[0])


# --- Section II-A: operators ------------------------------------------------
def test_adjoint_identity():
    rng = np.random.default_rng(1)
    _, sens, mask, _ = _small_case(Nx=10, Ny=12, Nt=4, Nc=3)
    x = _rand_c(rng, (4, 12, 10))
    y = _rand_c(rng, (4, 3, 12, 10))
    lhs = np.vdot(oracle.forward_op(x, sens, mask), y)
    rhs = np.vdot(x, oracle.adjoint_op(y, sens, mask))
    assert abs(lhs - rhs) <= 1e-13 * abs(lhs)


def test_unitary_parseval_and_impulse():
    """Full sampling, one coil with s = 1: H is the unitary 2D DFT."""
    rng = np.random.default_rng(2)
    Nt, Ny, Nx = 2, 15, 10          # radix 3 and 5 lengths
    sens = np.ones((1, Ny, Nx), complex)
    mask = np.ones((Nt, Ny), bool)
    x = _rand_c(rng, (Nt, Ny, Nx))
    k = oracle.forward_op(x, sens, mask)
    assert abs(np.linalg.norm(k) - np.linalg.norm(x)) <= 1e-13 * np.linalg.norm(x)
    imp = np.zeros((1, Ny, Nx), complex)
    imp[0, 0, 0] = 1.0
    k = oracle.forward_op(imp, sens, mask[:1])
    np.testing.assert_allclose(k[0, 0], np.full((Ny, Nx), 1 / np.sqrt(Ny * Nx)), atol=1e-15)
    # sign convention: a plane wave exp(+2 pi i j q / Ny) lands on row ky = q
    q = 4
    j = np.arange(Ny)[:, None] * np.ones((1, Nx))
    wave = np.exp(2j * np.pi * q * j / Ny)[None]
    k = oracle.forward_op(wave, sens, mask[:1])[0, 0]
    assert abs(abs(k[q, 0]) - np.sqrt(Ny * Nx)) < 1e-10
    assert np.abs(k).sum() - abs(k[q, 0]) < 1e-9


def test_forward_matches_acquisition_simulator_noise_free():
    """The oracle's H reproduces the noise-free data of the input generator."""
    x, sens, mask, y = _small_case(noise=0.0)
    np.testing.assert_allclose(oracle.forward_op(x, sens, mask), y, atol=1e-13)


def test_hybrid_residual_equals_full_residual():
    rng = np.random.default_rng(4)
    x0, sens, mask, y = _small_case(Nx=8, Ny=10, Nt=3, Nc=2, noise=0.05)
    x = x0 + 0.1 * _rand_c(rng, x0.shape)
    full = oracle.data_residual(x, y, sens, mask)
    yhat = oracle.hybrid_data(y, mask)
    cols = np.arange(8)
    part = oracle.data_residual_columns(x, yhat, sens, mask, cols)
    assert abs(full - part) <= 1e-12 * full
    # columns add up
    a = oracle.data_residual_columns(x[:, :, :3], yhat, sens, mask, cols[:3])
    b = oracle.data_residual_columns(x[:, :, 3:], yhat, sens, mask, cols[3:])
    assert abs(a + b - full) <= 1e-12 * full


# --- Section IV-C: Gram blocks and inverse ----------------------------------
@pytest.mark.parametrize("phase_y", [0.0, 1.5])
def test_gram_blocks_equal_dense_HtH(phase_y):
    """C_t (.) K_i equals the (i,t) block of H'H built column by column.  With a
    coil phase that varies along y, K_i is complex and not symmetric, so the
    side of the conjugation in Eq. HconjH matters."""
    _, sens, mask, _ = _small_case(Nx=3, Ny=6, Nt=2, Nc=3, R=2, seed=5)
    sens = synthdata.make_sens(3, 6, 3, phase_y=phase_y)
    if phase_y:
        K = np.einsum("cj,ck->jk", np.conj(sens[:, :, 1]), sens[:, :, 1])
        assert np.abs(K - K.T).max() > 0.1
    Nc, Ny, Nx = sens.shape
    Nt = mask.shape[0]
    Hd = _dense_H(sens, mask)
    HtH = Hd.conj().T @ Hd
    G = oracle.gram_blocks(sens, mask)
    for t in range(Nt):
        for i in range(Nx):
            idx = [(t * Ny + j) * Nx + i for j in range(Ny)]
            np.testing.assert_allclose(G[t, i], HtH[np.ix_(idx, idx)], atol=1e-13)
    # H'H has no coupling between different columns or frames
    blk = np.zeros_like(HtH, dtype=bool)
    for t in range(Nt):
        for i in range(Nx):
            idx = [(t * Ny + j) * Nx + i for j in range(Ny)]
            blk[np.ix_(idx, idx)] = True
    assert np.abs(HtH[~blk]).max() < 1e-13


def test_gram_full_sampling_is_identity_and_circulant():
    _, sens, mask, _ = _small_case(Nx=4, Ny=8, Nt=2, Nc=3, full=True)
    G = oracle.gram_blocks(sens, mask)
    np.testing.assert_allclose(G, np.broadcast_to(np.eye(8), G.shape), atol=1e-13)
    # partial sampling: F~'F~ is circulant (one coil, s = 1 gives C_t itself)
    _, _, mask2, _ = _small_case(Nx=4, Ny=8, Nt=2, Nc=1, seed=9)
    C = oracle.gram_blocks(np.ones((1, 8, 4), complex), mask2)[:, 0]
    for t in range(2):
        for j in range(8):
            np.testing.assert_allclose(C[t, j], np.roll(C[t, 0], j), atol=1e-14)
    # eigenvalues of C_t (.) K_i lie in [0, max_j K_jj] = [0, 1] (Schur product)
    _, sens3, mask3, _ = _small_case(Nx=4, Ny=8, Nt=3, Nc=2, seed=11)
    e = np.linalg.eigvalsh(oracle.gram_blocks(sens3, mask3))
    assert e.min() > -1e-12 and e.max() < 1 + 1e-12


def test_inverse_blocks_identity():
    _, sens, mask, _ = _small_case(Nx=5, Ny=12, Nt=3, Nc=2, seed=6)
    mu = 0.1
    G = oracle.gram_blocks(sens, mask)
    A = oracle.inverse_blocks(G, mu)
    eye = np.eye(12)
    res = np.einsum("tijk,tikl->tijl", A, mu * eye + G) - eye
    assert np.abs(res).max() < 1e-12
    np.testing.assert_allclose(A, np.conj(np.swapaxes(A, -1, -2)), atol=1e-14)


def test_inverse_single_coil_is_pointwise_kspace_inverse():
    """Nc = 1, s = 1: (mu I + F'PF)^{-1} = F' diag(1/(mu + P)) F (textbook)."""
    Ny, Nt, mu = 10, 2, 0.07
    rng = np.random.default_rng(7)
    mask = rng.random((Nt, Ny)) < 0.4
    A = oracle.inverse_blocks(oracle.gram_blocks(np.ones((1, Ny, 1), complex), mask), mu)
    F = np.fft.fft(np.eye(Ny), axis=0, norm="ortho")
    for t in range(Nt):
        ref = F.conj().T @ np.diag(1.0 / (mu + mask[t])) @ F
        np.testing.assert_allclose(A[t, 0], ref, atol=1e-13)


def test_synthesis_inversion_lemma_with_overcomplete_frame():
    """(mu I + Psi H'H Psi')^{-1} = (1/mu)(I - Psi Psi') + Psi (mu I + H'H)^{-1} Psi'.

    Checked with a dense tight frame Psi (Psi'Psi = I, Psi Psi' != I), the last
    line of the lemma in Section IV-A.
    """
    rng = np.random.default_rng(8)
    n, mu = 6, 0.3
    B = _rand_c(rng, (4, n))
    HtH = B.conj().T @ B
    Q, _ = np.linalg.qr(_rand_c(rng, (2 * n, 2 * n)))
    Psi = Q[:, :n]                              # 2n x n, Psi'Psi = I
    assert np.allclose(Psi.conj().T @ Psi, np.eye(n))
    lhs = np.linalg.inv(mu * np.eye(2 * n) + Psi @ HtH @ Psi.conj().T)
    rhs = (np.eye(2 * n) - Psi @ Psi.conj().T) / mu + Psi @ np.linalg.inv(mu * np.eye(n) + HtH) @ Psi.conj().T
    np.testing.assert_allclose(lhs, rhs, atol=1e-12)


# --- Eq. TV and the m-update ------------------------------------------------
def test_tv_difference_and_adjoint():
    rng = np.random.default_rng(9)
    Nt = 5
    x = _rand_c(rng, (Nt, 3, 2))
    u = _rand_c(rng, (Nt - 1, 3, 2))
    D = np.diff(np.eye(Nt), axis=0)           # rows e_{t+1} - e_t
    np.testing.assert_allclose(oracle.tv_D(x), np.tensordot(D, x, axes=(1, 0)), atol=1e-15)
    assert abs(np.vdot(oracle.tv_D(x), u) - np.vdot(x, oracle.tv_Dadj(u, Nt))) < 1e-13


def test_tv_m_matrix_matches_dct_eigen_closed_form():
    """rho I + D'D has eigenvalues rho + 2 - 2cos(pi k / Nt), DCT-II eigenvectors."""
    for Nt in (1, 2, 7, 32):
        rho = 0.5
        Minv = oracle.tv_m_matrix(Nt, rho)
        ev = np.sort(1.0 / np.linalg.eigvalsh(Minv))
        ref = np.sort(rho + 2 - 2 * np.cos(np.pi * np.arange(Nt) / Nt))
        np.testing.assert_allclose(ev, ref, atol=1e-12)
        if Nt > 1:
            k = 1
            vec = np.cos(np.pi * k * (np.arange(Nt) + 0.5) / Nt)
            np.testing.assert_allclose(np.linalg.solve(Minv, vec),
                                       (rho + 2 - 2 * np.cos(np.pi * k / Nt)) * vec, atol=1e-12)


# --- Algorithms 1 and 2: closed forms and optimality ------------------------
def test_alg1_full_sampling_reaches_soft_threshold_closed_form():
    """H'H = I makes the minimiser w* = S(Psi H'y, lambda/2) (closed form)."""
    x, sens, mask, y = _small_case(Nx=6, Ny=8, Nt=4, Nc=2, full=True, noise=0.02, seed=12)
    lam, mu = 0.05, 0.2
    P = oracle.Problem(y, sens, mask, mu)
    xr, info = oracle.admm_synthesis_dft(P.b, P.inv, lam, mu, 200, fid=P.fid)
    w_star = oracle.soft(oracle.psi_dft(P.b), lam / 2)
    np.testing.assert_allclose(oracle.psi_dft(xr), w_star, atol=1e-12)


def test_alg2_full_sampling_lambda0_is_exact_sense():
    x, sens, mask, y = _small_case(Nx=6, Ny=8, Nt=3, Nc=3, full=True, noise=0.0, seed=13)
    P = oracle.Problem(y, sens, mask, 0.1)
    xr, _ = oracle.admm_analysis_tv(P.b, P.inv, 0.0, 0.1, 0.5, 300)
    np.testing.assert_allclose(xr, x, atol=1e-10)
    np.testing.assert_allclose(P.b, x, atol=1e-12)       # H'H = I: H'y = x


def test_alg2_two_frames_closed_form():
    """Nt = 2, full sampling: per pixel min lam|x2-x1| + |x1-b1|^2 + |x2-b2|^2."""
    x, sens, mask, y = _small_case(Nx=5, Ny=6, Nt=2, Nc=2, full=True, noise=0.3, seed=14)
    lam = 0.25
    P = oracle.Problem(y, sens, mask, 0.1)
    xr, _ = oracle.admm_analysis_tv(P.b, P.inv, lam, 0.1, 0.5, 3000)
    b1, b2 = P.b[0], P.b[1]
    dl = b2 - b1
    mag = np.abs(dl)
    ph = np.where(mag > 0, dl / np.where(mag > 0, mag, 1), 0)
    small = mag <= lam
    x1 = np.where(small, (b1 + b2) / 2, b1 + lam / 2 * ph)
    x2 = np.where(small, (b1 + b2) / 2, b2 - lam / 2 * ph)
    assert (~small).any() and small.any()
    np.testing.assert_allclose(xr[0], x1, atol=1e-8)
    np.testing.assert_allclose(xr[1], x2, atol=1e-8)


def _tv_converged(seed=15, iters=4000):
    # 3 coils, half the rows: H'H is non-singular, so the minimiser is unique
    x, sens, mask, y = _small_case(Nx=4, Ny=4, Nt=3, Nc=3, R=2, noise=0.05, seed=seed)
    lam, mu, rho = 0.05, 0.1, 0.5
    P = oracle.Problem(y, sens, mask, mu)
    xr, info = oracle.admm_analysis_tv(P.b, P.inv, lam, mu, rho, iters, fid=P.fid)
    return x, sens, mask, y, lam, mu, rho, P, xr, info


def test_kkt_tv_on_tiny_problem():
    """2 H'(Hx - y) + lambda D_t' g = 0 with g = 2 mu1 d1 / lambda in the subdifferential."""
    x, sens, mask, y, lam, mu, rho, P, xr, info = _tv_converged()
    _, m, d1, d2 = info["state"]
    mu1 = mu / rho
    g = 2 * mu1 * d1 / lam
    assert np.abs(g).max() <= 1 + 1e-8
    Dx = oracle.tv_D(xr)
    big = np.abs(Dx) > 1e-6
    np.testing.assert_allclose(g[big], Dx[big] / np.abs(Dx[big]), atol=1e-6)
    grad = 2 * oracle.adjoint_op(oracle.forward_op(xr, sens, mask) - y, sens, mask)
    stat = grad + lam * oracle.tv_Dadj(g, xr.shape[0])
    assert np.linalg.norm(stat) < 1e-8 * max(1.0, np.linalg.norm(grad))


def test_kkt_dft_on_tiny_problem():
    x, sens, mask, y = _small_case(Nx=4, Ny=4, Nt=4, Nc=2, R=2, noise=0.05, seed=16)
    lam, mu = 0.05, 0.1
    P = oracle.Problem(y, sens, mask, mu)
    xr, info = oracle.admm_synthesis_dft(P.b, P.inv, lam, mu, 4000, fid=P.fid)
    w, d = info["state"]
    g = -2 * mu * d / lam
    assert np.abs(g).max() <= 1 + 1e-8
    big = np.abs(w) > 1e-6
    np.testing.assert_allclose(g[big], w[big] / np.abs(w[big]), atol=1e-6)
    grad = 2 * oracle.psi_dft(oracle.adjoint_op(oracle.forward_op(oracle.psi_dft_adj(w), sens, mask) - y, sens, mask))
    assert np.linalg.norm(grad + lam * g) < 1e-8 * max(1.0, np.linalg.norm(grad))


def test_dense_p1_reaches_same_minimiser():
    """A different splitting (P1 of Section III) with a dense direct inverse."""
    x, sens, mask, y, lam, mu, rho, P, xr, info = _tv_converged()
    Nt, Ny, Nx = xr.shape
    Hd = _dense_H(sens, mask)
    n = Nt * Ny * Nx
    D = np.zeros(((Nt - 1) * Ny * Nx, n))
    for t in range(Nt - 1):
        for p in range(Ny * Nx):
            D[t * Ny * Nx + p, t * Ny * Nx + p] = -1
            D[t * Ny * Nx + p, (t + 1) * Ny * Nx + p] = 1
    yv = y.ravel()
    mup = 0.2
    Minv = np.linalg.inv(mup * D.T @ D + Hd.conj().T @ Hd)
    Hty = Hd.conj().T @ yv
    xv = Hty.copy()
    dv = np.zeros(D.shape[0], complex)
    for _ in range(6000):
        v = oracle.soft(D @ xv - dv, lam / (2 * mup))
        xv = Minv @ (Hty + mup * D.T @ (v + dv))
        dv = dv - (D @ xv - v)
    assert np.linalg.cond(Hd.conj().T @ Hd) < 1e6
    J = lambda z: lam * np.abs(D @ z).sum() + np.linalg.norm(yv - Hd @ z) ** 2
    assert abs(J(xv) - J(xr.ravel())) < 1e-12 * J(xv)
    np.testing.assert_allclose(xv.reshape(Nt, Ny, Nx), xr, atol=1e-7)


def test_random_perturbations_never_lower_J():
    x, sens, mask, y, lam, mu, rho, P, xr, info = _tv_converged()
    rng = np.random.default_rng(0)
    J0 = oracle.objective_tv(xr, lam, P.fid)
    for _ in range(200):
        dx = 1e-4 * _rand_c(rng, xr.shape)
        assert oracle.objective_tv(xr + dx, lam, P.fid) >= J0 - 1e-12


def test_objective_and_delta_definitions():
    assert oracle.delta_ratio(2.0, 1.0) == 1.0
    assert oracle.delta_ratio(1.0, 1.0) == 0.0
    # J(0) is the objective at the initial point x = H'y
    case = synthdata.make_case("tiny", Nx=16, Ny=16, Nt=4, Nc=2)
    P = oracle.make_problem(case)
    _, info = P.solve("tv", case.lam, case.mu, iters=3)
    assert abs(info["J"][0] - oracle.objective_tv(P.b, case.lam, P.fid)) < 1e-12
    full = oracle.data_residual(P.b, case.kspace, case.sens, case.mask)
    assert abs(P.fid(P.b) - full) <= 1e-12 * full


def test_objectives_closed_forms():
    """J on inputs whose terms are known in closed form (Eqs. L1an_pri,
    L1unconst): noise-free data of x_t = x0 + t c gives a zero data term and
    ||D_t x||_1 = (Nt - 1) sum |c|; a single temporal frequency x_t = a
    exp(2 pi i f t / Nt) has one nonzero DFT bin per pixel, of modulus
    sqrt(Nt) |a|; at x = 0 (w = 0) the data term is ||y||^2."""
    rng = np.random.default_rng(7)
    Nt, Ny, Nx, lam = 5, 6, 4, 0.3
    sens = synthdata.make_sens(Nx, Ny, 2, phase_y=1.0)
    mask = np.zeros((Nt, Ny), bool)
    mask[:, ::2] = True
    x0, c, a = (_rand_c(rng, (Ny, Nx)) for _ in range(3))
    ramp = x0[None] + np.arange(Nt)[:, None, None] * c[None]
    y = oracle.forward_op(ramp, sens, mask)
    fid = lambda z: oracle.data_residual(z, y, sens, mask)
    ref = lam * (Nt - 1) * np.abs(c).sum()
    assert abs(oracle.objective_tv(ramp, lam, fid) - ref) <= 1e-12 * ref
    yy = float(np.vdot(y, y).real)
    assert abs(oracle.objective_tv(np.zeros_like(ramp), lam, fid) - yy) <= 1e-12 * yy
    f = 2
    tone = a[None] * np.exp(2j * np.pi * f * np.arange(Nt) / Nt)[:, None, None]
    y = oracle.forward_op(tone, sens, mask)
    fid = lambda z: oracle.data_residual(z, y, sens, mask)
    ref = lam * np.sqrt(Nt) * np.abs(a).sum()
    assert abs(oracle.objective_dft(oracle.psi_dft(tone), lam, fid) - ref) <= 1e-12 * ref
    yy = float(np.vdot(y, y).real)
    assert abs(oracle.objective_dft(np.zeros_like(tone), lam, fid) - yy) <= 1e-12 * yy


def test_column_subset_is_exact():
    """Columns are independent (Section IV-C): a subset run equals the full run."""
    case = synthdata.make_case("tiny", Nx=16, Ny=16, Nt=4, Nc=2)
    P = oracle.make_problem(case)
    cols = np.array([1, 5, 11])
    S = oracle.make_problem(case, cols)
    for prior in ("tv", "dft"):
        xf, _ = P.solve(prior, case.lam, case.mu, iters=10, objective=False)
        xs, _ = S.solve(prior, case.lam, case.mu, iters=10, objective=False)
        np.testing.assert_allclose(xs, xf[:, :, cols], atol=1e-13)


def test_golden_tiny_trajectory():
    """Regression fixture written by tests/golden/make_golden.py (oracle only)."""
    path = os.path.join(GOLDEN, "tiny_oracle.json")
    if not os.path.exists(path):
        pytest.skip("golden fixture not generated")
    g = json.load(open(path))
    case = synthdata.make_case("tiny", Nx=g["Nx"], Ny=g["Ny"], Nt=g["Nt"], Nc=g["Nc"])
    P = oracle.make_problem(case)
    for prior in ("tv", "dft"):
        x, info = P.solve(prior, case.lam, case.mu, iters=g["iters"])
        np.testing.assert_allclose(info["J"], g[prior]["J"], rtol=1e-12)
        assert abs(np.linalg.norm(x) - g[prior]["xnorm"]) < 1e-10 * g[prior]["xnorm"]
        for key in ("primal_res", "dual_res"):
            assert abs(info[key] - g[prior][key]) <= 1e-10 * g[prior][key]


# --- the input generator ----------------------------------------------------
def test_synthdata_structure():
    case = synthdata.make_case("tiny")
    Nt, Nc, Ny, Nx = case.kspace.shape
    assert (Nt, Nc, Ny, Nx) == (8, 4, 64, 64)
    assert np.allclose(np.sum(np.abs(case.sens) ** 2, axis=0), 1.0)
    assert abs(np.abs(case.x_true).max() - 1.0) < 1e-12
    assert np.all(case.mask.sum(1) == 16)                      # round(64/4)
    central = np.mod(np.arange(-4, 4), Ny)
    assert case.mask[:, central].all()
    assert np.all(case.kspace[~np.broadcast_to(case.mask[:, None, :, None], case.kspace.shape)] == 0)
    assert len({tuple(np.nonzero(case.mask[t])[0]) for t in range(Nt)}) > 1


def test_tv_residuals_vanish_at_convergence_and_follow_the_duals():
    """Algorithm 2's residuals: v - D_t m equals d1_prev - d1 (the d1-update), both
    residuals shrink to ~0 at the ADMM fixed point, and they are positive early on."""
    x, sens, mask, y = _small_case(Nx=4, Ny=4, Nt=4, Nc=2, R=2, noise=0.05, seed=19)
    lam, mu, rho = 0.05, 0.1, 0.5
    P = oracle.Problem(y, sens, mask, mu)
    _, early = oracle.admm_analysis_tv(P.b, P.inv, lam, mu, rho, 3)
    assert early["primal_res"] > 1e-6 and early["dual_res"] > 1e-6
    # the v - D_t m part equals the change of d1 in the last iteration
    _, i4 = oracle.admm_analysis_tv(P.b, P.inv, lam, mu, rho, 4)
    _, i5 = oracle.admm_analysis_tv(P.b, P.inv, lam, mu, rho, 5)
    x5, m5, d1_5, _ = i5["state"]
    d1_4 = i4["state"][2]
    part = np.sqrt(np.vdot(d1_4 - d1_5, d1_4 - d1_5).real + np.vdot(m5 - x5, m5 - x5).real)
    assert abs(part - i5["primal_res"]) <= 1e-12 * max(part, 1e-30)
    _, late = oracle.admm_analysis_tv(P.b, P.inv, lam, mu, rho, 3000)
    assert late["primal_res"] < 1e-8 and late["dual_res"] < 1e-8


@pytest.mark.parametrize("prior", ["dft", "haar"])
def test_synthesis_residuals_vanish_at_convergence_and_follow_the_dual(prior):
    """Algorithm 1's residuals: w - v equals d_prev - d (the d-update), both shrink
    to ~0 at the ADMM fixed point and are positive early on; for the unitary DFT
    the dual mu ||w - w_prev|| equals mu ||x - x_prev|| in the image domain
    (Parseval), the form a GPU path can evaluate without the coefficients."""
    x, sens, mask, y = _small_case(Nx=4, Ny=4, Nt=4, Nc=2, R=2, noise=0.05, seed=21)
    lam, mu = 0.05, 0.1
    P = oracle.Problem(y, sens, mask, mu)
    kw = {} if prior == "dft" else dict(psi=lambda a: oracle.psi_haar(a, 1), psi_adj=lambda a: oracle.psi_haar_adj(a, 1))
    _, early = oracle.admm_synthesis_dft(P.b, P.inv, lam, mu, 3, **kw)
    assert early["primal_res"] > 1e-6 and early["dual_res"] > 1e-6
    x4, i4 = oracle.admm_synthesis_dft(P.b, P.inv, lam, mu, 4, **kw)
    x5, i5 = oracle.admm_synthesis_dft(P.b, P.inv, lam, mu, 5, **kw)
    (w4, d4), (w5, d5) = i4["state"], i5["state"]
    assert abs(np.linalg.norm(d4 - d5) - i5["primal_res"]) <= 1e-12 * i5["primal_res"]
    assert abs(mu * np.linalg.norm(w5 - w4) - i5["dual_res"]) <= 1e-12 * i5["dual_res"]
    if prior == "dft":
        assert abs(mu * np.linalg.norm(x5 - x4) - i5["dual_res"]) <= 1e-10 * i5["dual_res"]
    # one iteration: w_0 = Psi H'y, d_0 = 0, so the primal is ||w_1 - v_1|| = ||d_1||
    _, i1 = oracle.admm_synthesis_dft(P.b, P.inv, lam, mu, 1, **kw)
    assert abs(np.linalg.norm(i1["state"][1]) - i1["primal_res"]) <= 1e-12 * i1["primal_res"]
    # the redundant Haar frame converges far more slowly than the unitary DFT
    _, late = oracle.admm_synthesis_dft(P.b, P.inv, lam, mu, 3000 if prior == "dft" else 12000, **kw)
    for key in ("primal_res", "dual_res"):
        assert late[key] < (1e-8 if prior == "dft" else 1e-4 * early[key])
