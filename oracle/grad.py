"""FP64 oracle gradient of unrolled Algorithm 2 (test infrastructure only).

The paper gives no derivative; this is the reverse-mode (adjoint) of the K
steps of Algorithm 2 exactly as ``admm.admm_analysis_tv`` runs them, derived
by hand.  Parameters: mu2 = mu, mu1 = mu / rho with rho fixed, so the
threshold is tau1 = lambda rho / (2 mu).  One iteration, from the state
(x, m, d1, d2):

    a   = D_t m + d1;            v  = S(a, tau1)
    rhs = D_t'(v - d1) + rho (x + d2);   m' = M^{-1} rhs,  M = rho I + D_t'D_t
    r   = b + mu (m' - d2);      x' = A(mu) r,  A(mu) = (mu I + H'H)^{-1}
    d1' = d1 - v + D_t m';       d2' = d2 - m' + x'

with b = H'y and x0 = m0 = b, d1 = d2 = 0.  Loss L = ||x_K - x_true||^2.
Gradients follow the PyTorch convention for complex inputs
(dL/dRe + i dL/dIm), so a complex-linear map W contributes W' to the
reverse pass.  Special rules:

    dA/dmu = -A^2           ->  mu_bar += -Re<A xbar', x'>
    S(a, tau) for |a|>tau   ->  abar = vbar - (tau/|a|)(vbar - n Re(conj(n) vbar)),  n = a/|a|
                                tau_bar += -Re(conj(n) vbar)
    |a| <= tau              ->  abar = 0, no tau_bar
    y                       ->  ybar = H bbar   (b = H'y)

Parity status: pinned by central finite differences in FP64
(tests/test_oracle_grad.py).
"""

from __future__ import annotations

import numpy as np

from .admm import (ColumnInverse, adjoint_op, forward_op, soft, tv_D, tv_Dadj, tv_m_matrix)

__all__ = ["unrolled_tv_forward", "unrolled_tv_adjoint", "unrolled_tv_loss_and_grad"]


def unrolled_tv_forward(b, inv, lam, mu, rho, iters):
    """K steps of Algorithm 2 keeping every state (x, m, d1, d2)."""
    Nt = b.shape[0]
    tau1 = lam * rho / (2.0 * mu)
    Minv = tv_m_matrix(Nt, rho)
    x, m = b.copy(), b.copy()
    d1 = np.zeros((max(Nt - 1, 0),) + b.shape[1:], dtype=np.complex128)
    d2 = np.zeros_like(b)
    states = [(x, m, d1, d2)]
    for _ in range(iters):
        v = soft(tv_D(m) + d1, tau1)
        rhs = tv_Dadj(v - d1, Nt) + rho * (x + d2)
        m_new = np.tensordot(Minv, rhs, axes=(1, 0))
        x_new = inv.apply(b + mu * (m_new - d2))
        d1 = d1 - v + tv_D(m_new)
        d2 = d2 - m_new + x_new
        x, m = x_new, m_new
        states.append((x, m, d1, d2))
    return states


def _soft_adjoint(a, vbar, tau):
    """J^T vbar of v = S(a, tau) (J symmetric as a real 2x2 map) and tau_bar."""
    mag = np.abs(a)
    on = mag > tau
    n = np.zeros_like(a)
    n[on] = a[on] / mag[on]
    proj = np.real(np.conj(n) * vbar)
    abar = np.zeros_like(vbar)
    abar[on] = vbar[on] - (tau / mag[on]) * (vbar[on] - n[on] * proj[on])
    tau_bar = -float(np.sum(proj[on]))
    return abar, tau_bar


def unrolled_tv_adjoint(b, inv, x_true, lam, mu, rho, iters):
    """Loss and reverse pass on given columns: (L, bbar, dL/dlambda, dL/dmu).

    ``b`` = H'y and ``x_true`` restricted to the columns of ``inv``; the loss
    and every gradient are sums over columns, since columns are independent.
    """
    Nt = b.shape[0]
    tau1 = lam * rho / (2.0 * mu)
    Minv = tv_m_matrix(Nt, rho)
    S = unrolled_tv_forward(b, inv, lam, mu, rho, iters)
    xK = S[-1][0]
    L = float(np.vdot(xK - x_true, xK - x_true).real)
    xb = 2.0 * (xK - x_true)
    mb = np.zeros_like(b)
    d1b = np.zeros_like(S[0][2])
    d2b = np.zeros_like(b)
    bb = np.zeros_like(b)
    mu_bar = 0.0
    tau_bar = 0.0
    for k in range(iters, 0, -1):
        x0, m0, d10, d20 = S[k - 1]
        x1, m1, _, _ = S[k]
        # d2' = d2 - m' + x';  d1' = d1 - v + D m'
        d2_acc = d2b.copy()
        mb_t = mb - d2b + tv_Dadj(d1b, Nt)
        xb_t = xb + d2b
        vb = -d1b
        d1_acc = d1b.copy()
        # x' = A r
        rb = inv.apply(xb_t)
        mu_bar += -float(np.vdot(rb, x1).real)
        # r = b + mu (m' - d2)
        bb += rb
        mb_t = mb_t + mu * rb
        d2_acc = d2_acc - mu * rb
        mu_bar += float(np.vdot(rb, m1 - d20).real)
        # m' = M^{-1} rhs;  rhs = D'(v - d1) + rho (x + d2)
        rhsb = np.tensordot(Minv, mb_t, axes=(1, 0))
        ub = tv_D(rhsb)
        xb_new = rho * rhsb
        d2_acc = d2_acc + rho * rhsb
        vb = vb + ub
        d1_acc = d1_acc - ub
        # v = S(D m + d1, tau1)
        ab, tb = _soft_adjoint(tv_D(m0) + d10, vb, tau1)
        tau_bar += tb
        mb = tv_Dadj(ab, Nt)
        d1_acc = d1_acc + ab
        xb, d1b, d2b = xb_new, d1_acc, d2_acc
    bb += xb + mb            # x0 = m0 = b
    grad_lam = tau_bar * rho / (2.0 * mu)
    grad_mu = mu_bar - tau_bar * tau1 / mu
    return L, bb, grad_lam, grad_mu


def unrolled_tv_loss_and_grad(kspace, sens, mask, x_true, lam, mu, rho, iters):
    """L = ||x_K - x_true||^2 and (dL/dy, dL/dlambda, dL/dmu, bbar) of unrolled Algorithm 2."""
    inv = ColumnInverse(sens, mask, mu)
    b = adjoint_op(kspace, sens, mask)
    L, bb, grad_lam, grad_mu = unrolled_tv_adjoint(b, inv, x_true, lam, mu, rho, iters)
    grad_y = forward_op(bb, sens, mask)
    return L, grad_y, grad_lam, grad_mu, bb
