"""Pins of the oracle's redundant temporal frame and of Algorithm 1 with it (CPU).

``psi_haar`` is the undecimated temporal Haar frame with circular shifts.
Its pins do not re-derive the code:
* the frequency response of each channel on complex exponentials, in closed form;
* the tight-frame identity Psi'Psi = I together with Psi Psi' != I (redundancy);
* adjointness; constants pass to the approximation channel untouched.
Algorithm 1 with this frame (the lemma of Section IV-A with its
(1/mu)(I - Psi Psi') term active) is pinned by the KKT conditions of the
synthesis problem on a tiny case.
"""

import numpy as np
import pytest

import oracle
from test_oracle_pins import _small_case


def _dense(levels, Nt):
    """Psi as a dense ((levels+1) Nt) x Nt matrix, column by column."""
    cols = [oracle.psi_haar(np.eye(Nt)[:, k], levels).reshape(-1) for k in range(Nt)]
    return np.stack(cols, axis=1)


@pytest.mark.parametrize("Nt", [7, 8, 12, 32])
@pytest.mark.parametrize("levels", [1, 2, 3, 4])
def test_channel_frequency_response_closed_form(Nt, levels):
    t = np.arange(Nt)
    for k in range(Nt):
        x = np.exp(2j * np.pi * k * t / Nt)
        w = oracle.psi_haar(x, levels)
        low = 1.0 + 0j
        for j in range(1, levels + 1):
            z = np.exp(2j * np.pi * k * (2 ** (j - 1)) / Nt)
            np.testing.assert_allclose(w[j - 1], x * low * (1 - z) / 2, atol=1e-12)
            low = low * (1 + z) / 2
        np.testing.assert_allclose(w[levels], x * low, atol=1e-12)


@pytest.mark.parametrize("Nt,levels", [(8, 1), (8, 3), (12, 2), (5, 3)])
def test_tight_and_redundant(Nt, levels):
    F = _dense(levels, Nt)
    np.testing.assert_allclose(F.conj().T @ F, np.eye(Nt), atol=1e-13)       # Psi'Psi = I
    G = F @ F.conj().T
    assert np.linalg.matrix_rank(G) == Nt < G.shape[0]                         # Psi Psi' != I
    rng = np.random.default_rng(levels)
    x = rng.standard_normal((Nt, 2, 3)) + 1j * rng.standard_normal((Nt, 2, 3))
    w = rng.standard_normal((levels + 1, Nt, 2, 3)) + 1j * rng.standard_normal((levels + 1, Nt, 2, 3))
    lhs = np.vdot(oracle.psi_haar(x, levels), w)
    rhs = np.vdot(x, oracle.psi_haar_adj(w, levels))
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)
    np.testing.assert_allclose(oracle.psi_haar_adj(oracle.psi_haar(x, levels), levels), x, atol=1e-13)


def test_constant_goes_to_approximation():
    c = (0.3 - 1.2j) * np.ones((8, 2))
    w = oracle.psi_haar(c, 3)
    assert np.abs(w[:3]).max() == 0
    np.testing.assert_allclose(w[3], c, atol=1e-15)


def test_kkt_alg1_with_redundant_haar_frame():
    x, sens, mask, y = _small_case(Nx=4, Ny=4, Nt=4, Nc=2, R=2, noise=0.05, seed=17)
    lam, mu, L = 0.05, 0.03, 2          # ADMM with a redundant frame converges slowly; small mu is fastest here
    P = oracle.Problem(y, sens, mask, mu)
    psi = lambda z: oracle.psi_haar(z, L)
    psi_adj = lambda z: oracle.psi_haar_adj(z, L)
    xr, info = oracle.admm_synthesis_dft(P.b, P.inv, lam, mu, 8000, psi=psi, psi_adj=psi_adj)
    w, d = info["state"]
    np.testing.assert_allclose(xr, psi_adj(w), atol=1e-14)
    g = -2 * mu * d / lam
    assert np.abs(g).max() <= 1 + 1e-5
    big = np.abs(w) > 1e-6
    np.testing.assert_allclose(g[big], w[big] / np.abs(w[big]), atol=1e-5)
    grad = 2 * psi(oracle.adjoint_op(oracle.forward_op(psi_adj(w), sens, mask) - y, sens, mask))
    assert np.linalg.norm(grad + lam * g) < 1e-7 * max(1.0, np.linalg.norm(grad))
