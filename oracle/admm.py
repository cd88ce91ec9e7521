"""FP64 oracle of the paper's ADMM reconstruction (test infrastructure only).

Parity status: every function below is pinned by a test in
``tests/test_oracle_pins.py`` (closed forms, brute force, invariants).  No
function here is "parity unpinned".

Array conventions (NumPy, complex128):
  image      x[t, j, i]        frame t, vertical (ky / Ny) j, horizontal (kx / Nx) i
  k-space    y[t, c, ky, kx]   unsampled rows are ignored (treated as 0)
  coils      s[c, j, i]
  mask       mask[t, ky]       bool row mask in FFT order; kx always sampled
The paper's "column" x_{v,i,t} (Eq. x_def) is x[t, :, i].

Readings of the paper used here (where it is garbled, silent or ambiguous):
  * Eq. HconjH prints sum_c s_c s_c'.  From S_c' F~' F~ S_c the (j,k) entry is
    conj(s_j) s_k, i.e. the elementwise conjugate of the printed form; the
    operator form is used (Section IV-C).
  * The matrix-inversion lemma of Section IV-A: the first printed line lacks a
    1/mu; the last line, (1/mu)(I - Psi Psi') + Psi (mu I + H'H)^{-1} Psi', is
    used.
  * "SVD" of the Hermitian PSD block H'H is its eigendecomposition (eigh).
  * All Fourier transforms are unitary: forward exp(-2 pi i k n / N)/sqrt(N).
  * Algorithm 2 with one mu in the workload: mu2 = mu, mu1 = mu / rho,
    rho = mu2/mu1 (0.5 by default, Section V).
  * Temporal TV is non-circular: D_t is (Nt-1) x Nt (Eq. TV).
  * Soft threshold: |a| <= tau gives exactly 0; |a| is the complex modulus and
    the l1 norm is sum |a_i|.
  * Objective without 1/2: lambda ||.||_1 + ||y - H.||^2 (Eqs. L1unconst,
    L1an_pri); J(0) is evaluated at the initial point, J(k) at the new x (TV)
    or new w (DFT) of iteration k; stop when 0 <= Delta(k) < tol.
"""

from __future__ import annotations

import numpy as np

__all__ = [
    "soft", "unitary_dft_matrix", "forward_op", "adjoint_op", "hybrid_data",
    "gram_blocks", "inverse_blocks", "ColumnInverse", "tv_D", "tv_Dadj",
    "tv_m_matrix", "data_residual", "data_residual_columns", "objective_tv",
    "objective_dft", "delta_ratio", "admm_analysis_tv", "admm_synthesis_dft", "tv_residuals",
    "synthesis_residuals",
    "psi_dft", "psi_dft_adj", "psi_haar", "psi_haar_adj", "Problem", "make_problem",
]


# ---------------------------------------------------------------------------
# Section III: complex soft threshold S(a, tau) = (|a|-tau) a/|a| if |a|>tau else 0
# ---------------------------------------------------------------------------
def soft(a, tau):
    """Element-wise complex soft threshold (Section III, definition of S)."""
    a = np.asarray(a)
    mag = np.abs(a)
    out = np.zeros_like(a)
    keep = mag > tau
    out[keep] = (mag[keep] - tau) * a[keep] / mag[keep]
    return out


# ---------------------------------------------------------------------------
# Section II-A: Cartesian multi-coil forward model and its adjoint
# ---------------------------------------------------------------------------
def unitary_dft_matrix(n):
    """Explicit unitary DFT matrix F[q, j] = exp(-2 pi i q j / n) / sqrt(n)."""
    q = np.arange(n)
    return np.exp(-2j * np.pi * np.outer(q, q) / n) / np.sqrt(n)


def forward_op(x, sens, mask):
    """H x: y[t,c] = M_{v,t} F_h F_v (s_c . x_t)  (Eqs. mri_csmcoill, H_1, S, F).

    F_h, F_v are unitary 1D DFTs along the horizontal / vertical axes; M_{v,t}
    keeps the sampled rows of frame t (others are returned as 0).
    """
    coil = sens[None, :, :, :] * x[:, None, :, :]               # S x
    k = np.fft.fft(coil, axis=-2, norm="ortho")                 # F_v
    k = np.fft.fft(k, axis=-1, norm="ortho")                    # F_h
    return k * mask[:, None, :, None]                           # M_{v,t}


def adjoint_op(y, sens, mask):
    """H' y = sum_c conj(s_c) . F_v' M' F_h' y_{t,c}  (adjoint of ``forward_op``)."""
    k = y * mask[:, None, :, None]
    img = np.fft.ifft(k, axis=-1, norm="ortho")                 # F_h'
    img = np.fft.ifft(img, axis=-2, norm="ortho")               # F_v'
    return np.sum(np.conj(sens)[None] * img, axis=1)


def hybrid_data(y, mask):
    """F_h' y on the sampled rows: yhat[t, c, ky, i] (0 on unsampled rows).

    Since F_h is unitary along each k-space row, ||y - Hx||^2 equals
    sum over sampled rows of |yhat - F_v(s_c x_t)|^2 (Section IV-C uses
    F_h'F_h = I the same way).
    """
    return np.fft.ifft(y * mask[:, None, :, None], axis=-1, norm="ortho")


# ---------------------------------------------------------------------------
# Section IV-C: separable Gram blocks and the exact inverse
# ---------------------------------------------------------------------------
def gram_blocks(sens, mask, cols=None):
    """G[t, ci] = (F~_{v,t}' F~_{v,t}) (.) sum_c conj(s_{v,i,c}) s_{v,i,c}^T  (Eq. HconjH).

    ``F~_{v,t} = M_{v,t} F_v`` is built explicitly as the sampled rows of the
    unitary DFT matrix.  Returns an array [Nt, ncols, Ny, Ny].
    """
    Nc, Ny, Nx = sens.shape
    Nt = mask.shape[0]
    cols = np.arange(Nx) if cols is None else np.asarray(cols)
    F = unitary_dft_matrix(Ny)
    FtF = np.empty((Nt, Ny, Ny), dtype=np.complex128)
    for t in range(Nt):
        Ft = F[mask[t], :]                                      # M_{v,t} F_v
        FtF[t] = Ft.conj().T @ Ft
    S = sens[:, :, cols]                                        # [Nc, Ny, ncols]
    # K[ci, j, k] = sum_c conj(s[c, j, i]) s[c, k, i]
    K = np.einsum("cji,cki->ijk", np.conj(S), S)
    return FtF[:, None, :, :] * K[None, :, :, :]


def inverse_blocks(G, mu):
    """(mu I + G)^{-1} = U diag(1/(e_k + mu)) U'  per block (Eq. eigen_mu)."""
    e, U = np.linalg.eigh(G)
    return np.einsum("...jk,...k,...lk->...jl", U, 1.0 / (e + mu), np.conj(U))


class ColumnInverse:
    """Applies (mu I + H'H)^{-1} column by column (Eq. separate_x, eigen_mu).

    H'H is block diagonal over frames t and columns i, so the inverse acts on
    each column x[t, :, i] with its own dense Ny x Ny matrix A[t, i].
    """

    def __init__(self, sens, mask, mu, cols=None):
        self.cols = np.arange(sens.shape[2]) if cols is None else np.asarray(cols)
        self.G = gram_blocks(sens, mask, self.cols)
        self.A = inverse_blocks(self.G, mu)
        self.mu = mu

    def apply(self, r):
        """r[t, j, ci] -> x[t, j, ci] = A[t, ci] r[t, :, ci]."""
        return np.einsum("tijk,tki->tji", self.A, r)


# ---------------------------------------------------------------------------
# Section II-A, Eq. TV: temporal difference D_t and the m-update matrix
# ---------------------------------------------------------------------------
def tv_D(x):
    """(D_t x)_t = x_{t+1} - x_t for t = 0..Nt-2 (non-circular, Eq. TV)."""
    return x[1:] - x[:-1]


def tv_Dadj(u, Nt):
    """D_t' u: (D_t' u)_s = u_{s-1} - u_s with u_{-1} = u_{Nt-1} = 0."""
    out = np.zeros((Nt,) + u.shape[1:], dtype=np.result_type(u, np.complex128))
    out[:-1] -= u
    out[1:] += u
    return out


def _D_matrix(Nt):
    D = np.zeros((max(Nt - 1, 0), Nt))
    for t in range(Nt - 1):
        D[t, t] = -1.0
        D[t, t + 1] = 1.0
    return D


def tv_m_matrix(Nt, rho):
    """(rho I + D_t' D_t)^{-1} as a dense Nt x Nt matrix (Algorithm 2, m-update)."""
    D = _D_matrix(Nt)
    return np.linalg.inv(rho * np.eye(Nt) + D.T @ D)


# ---------------------------------------------------------------------------
# Objective (Eqs. L1unconst, L1an_pri) and convergence ratio (Eq. r_ratio)
# ---------------------------------------------------------------------------
def data_residual(x, y, sens, mask):
    """||y - H x||^2 over the sampled entries (full grid)."""
    r = (y * mask[:, None, :, None]) - forward_op(x, sens, mask)
    return float(np.vdot(r, r).real)


def data_residual_columns(x_cols, yhat, sens, mask, cols):
    """||y - H x||^2 restricted to columns ``cols`` via hybrid data F_h'y.

    x_cols[t, j, ci]; yhat from ``hybrid_data``.  Summed over all columns this
    equals ``data_residual`` (F_h unitary per row).
    """
    S = sens[:, :, cols]
    z = np.fft.fft(S[None] * x_cols[:, None], axis=-2, norm="ortho")   # F_v(s_c x)
    r = (yhat[:, :, :, cols] - z) * mask[:, None, :, None]
    return float(np.vdot(r, r).real)


def objective_tv(x, lam, fid):
    """J = lambda ||D_t x||_1 + ||y - H x||^2  (Eq. L1an_pri with R = TV_t)."""
    return lam * float(np.abs(tv_D(x)).sum()) + fid(x)


def objective_dft(w, lam, fid):
    """J = lambda ||w||_1 + ||y - H Psi' w||^2  (Eq. L1unconst)."""
    return lam * float(np.abs(w).sum()) + fid(psi_dft_adj(w))


def delta_ratio(J_prev, J):
    """Delta(k) = (J(k-1) - J(k)) / J(k)  (Eq. r_ratio)."""
    return (J_prev - J) / J


# ---------------------------------------------------------------------------
# Psi: unitary temporal DFT (orthonormal, Psi'Psi = Psi Psi' = I)
# ---------------------------------------------------------------------------
def psi_dft(x):
    return np.fft.fft(x, axis=0, norm="ortho")


def psi_dft_adj(w):
    return np.fft.ifft(w, axis=0, norm="ortho")


def psi_haar(x, levels):
    """Undecimated temporal Haar frame (a redundant tight frame, Psi'Psi = I).

    Along t with circular shifts: a_0 = x and, for level j = 1..levels with
    shift s = 2^(j-1) (mod Nt),
        a_j[t] = (a_{j-1}[t] + a_{j-1}[t+s]) / 2,   d_j[t] = (a_{j-1}[t] - a_{j-1}[t+s]) / 2.
    Coefficients stacked as [d_1, ..., d_levels, a_levels] on a new axis 0.
    Section IV-A allows any tight frame for Psi; this is one with
    Psi Psi' != I, so the (1/mu)(I - Psi Psi') term of the lemma is active.
    """
    a = np.asarray(x, dtype=np.complex128)
    Nt = a.shape[0]
    out = []
    for j in range(1, levels + 1):
        sh = (2 ** (j - 1)) % Nt
        nxt = np.roll(a, -sh, axis=0)              # nxt[t] = a[t + s]
        out.append((a - nxt) / 2.0)
        a = (a + nxt) / 2.0
    out.append(a)
    return np.stack(out)


def psi_haar_adj(w, levels):
    """Synthesis Psi' of ``psi_haar`` (its adjoint; psi_haar_adj(psi_haar(x)) = x)."""
    w = np.asarray(w, dtype=np.complex128)
    Nt = w.shape[1]
    a = w[levels].copy()
    for j in range(levels, 0, -1):
        sh = (2 ** (j - 1)) % Nt
        d = w[j - 1]
        # adjoint of a -> ((a + S a)/2, (a - S a)/2) with (S a)[t] = a[t + s]
        a = (a + np.roll(a, sh, axis=0)) / 2.0 + (d - np.roll(d, sh, axis=0)) / 2.0
    return a


# ---------------------------------------------------------------------------
# Algorithm 2: ADMM for the analysis prior (R = D_t, temporal TV)
# ---------------------------------------------------------------------------
def admm_analysis_tv(b, inv, lam, mu, rho, iters, fid=None, tol=0.0, state=None):
    """Algorithm 2 (ADMM_Analysis) with R = D_t.

    b = H'y restricted to the columns of ``inv``; mu2 = mu, mu1 = mu/rho.
    Returns (x, info) with info["J"] = [J(0), ..., J(k)] when ``fid`` is given.
    ``state`` = (x, m, d1, d2) resumes from a previous call.
    """
    Nt = b.shape[0]
    mu2 = mu
    mu1 = mu / rho
    Minv = tv_m_matrix(Nt, mu2 / mu1)
    m_prev = None
    if state is None:
        x = b.copy()                                            # x = H'y
        m = x.copy()                                            # m = x
        d1 = np.zeros((max(Nt - 1, 0),) + b.shape[1:], dtype=np.complex128)
        d2 = np.zeros_like(b)
    else:
        x, m, d1, d2 = (np.array(a, dtype=np.complex128) for a in state)
    J = [objective_tv(x, lam, fid)] if fid is not None else []
    k_done = 0
    for k in range(1, iters + 1):
        m_prev = m
        # v <- S(R m + d1, lambda / (2 mu1))
        v = soft(tv_D(m) + d1, lam / (2.0 * mu1))
        # m <- (mu2/mu1 I + R'R)^{-1} [R'(v - d1) + mu2/mu1 (x + d2)]
        rhs = tv_Dadj(v - d1, Nt) + (mu2 / mu1) * (x + d2)
        m = np.tensordot(Minv, rhs, axes=(1, 0))
        # x <- (mu2 I + H'H)^{-1} [H'y + mu2 (m - d2)]
        x = inv.apply(b + mu2 * (m - d2))
        # d1 <- d1 - (v - R m);  d2 <- d2 - (m - x)
        d1 = d1 - (v - tv_D(m))
        d2 = d2 - (m - x)
        k_done = k
        if fid is not None:
            J.append(objective_tv(x, lam, fid))
            if tol > 0:
                dk = delta_ratio(J[-2], J[-1])
                if 0.0 <= dk < tol:
                    break
    info = dict(J=J, iters=k_done, state=(x, m, d1, d2))
    if m_prev is not None:
        info["primal_res"], info["dual_res"] = tv_residuals(x, m, v, m_prev, mu1, mu2)
    return x, info


def tv_residuals(x, m, v, m_prev, mu1, mu2):
    """ADMM residuals of Algorithm 2 after an iteration, in the stacked form of
    Boyd et al. (Distributed Optimization and Statistical Learning via ADMM,
    2011, Sec. 3.3) for its two splits, v = D_t m (penalty mu1) and m = x
    (penalty mu2), with m the variable updated second:
      primal = sqrt(||v - D_t m||^2 + ||m - x||^2)
      dual   = sqrt(mu1^2 ||D_t (m - m_prev)||^2 + mu2^2 ||m - m_prev||^2)."""
    rp = np.vdot(v - tv_D(m), v - tv_D(m)).real + np.vdot(m - x, m - x).real
    dm = m - m_prev
    rd = mu1 ** 2 * np.vdot(tv_D(dm), tv_D(dm)).real + mu2 ** 2 * np.vdot(dm, dm).real
    return float(np.sqrt(rp)), float(np.sqrt(rd))


# ---------------------------------------------------------------------------
# Algorithm 1: ADMM for the synthesis prior (Psi = unitary temporal DFT)
# ---------------------------------------------------------------------------
def admm_synthesis_dft(b, inv, lam, mu, iters, fid=None, tol=0.0, state=None,
                       psi=psi_dft, psi_adj=psi_dft_adj):
    """Algorithm 1 (ADMM_Synthesis) with a tight frame Psi (default temporal DFT).

    Returns (x = Psi' w, info); info["J"] = [J(0), ..., J(k)] when ``fid``
    is given.  ``state`` = (w, d) resumes from a previous call.
    """
    Psi_b = psi(b)
    if state is None:
        d = np.zeros_like(Psi_b)                                # d = 0
        w = Psi_b.copy()                                        # w = Psi H'y
    else:
        w, d = (np.array(a, dtype=np.complex128) for a in state)
    J = [lam * float(np.abs(w).sum()) + fid(psi_adj(w))] if fid is not None else []
    k_done = 0
    w_prev = v = None
    for k in range(1, iters + 1):
        w_prev = w
        # v <- S(w - d, lambda / (2 mu))
        v = soft(w - d, lam / (2.0 * mu))
        # w <- (1/mu)(I - Psi Psi')[Psi H'y + mu(v + d)]
        #      + Psi (mu I + H'H)^{-1} [H'y + mu Psi'(v + d)]
        u = Psi_b + mu * (v + d)
        w = (u - psi(psi_adj(u))) / mu + psi(inv.apply(b + mu * psi_adj(v + d)))
        # d <- d - (w - v)
        d = d - (w - v)
        k_done = k
        if fid is not None:
            J.append(lam * float(np.abs(w).sum()) + fid(psi_adj(w)))
            if tol > 0:
                dk = delta_ratio(J[-2], J[-1])
                if 0.0 <= dk < tol:
                    break
    info = dict(J=J, iters=k_done, state=(w, d))
    if w_prev is not None:
        info["primal_res"], info["dual_res"] = synthesis_residuals(w, v, w_prev, mu)
    return psi_adj(w), info


def synthesis_residuals(w, v, w_prev, mu):
    """ADMM residuals of Algorithm 1 after an iteration (Boyd et al. 2011,
    Sec. 3.3) for its one split v = w (penalty mu), w the variable updated
    second:
      primal = ||w - v||,   dual = mu ||w - w_prev||.
    As for Algorithm 2, the paper's penalty weight mu stands where Boyd's
    scaled form has rho/2."""
    rp = np.vdot(w - v, w - v).real
    dw = w - w_prev
    return float(np.sqrt(rp)), float(mu * np.sqrt(np.vdot(dw, dw).real))


# ---------------------------------------------------------------------------
# Convenience: one problem restricted to a set of columns
# ---------------------------------------------------------------------------
class Problem:
    """Oracle view of one reconstruction restricted to columns ``cols``."""

    def __init__(self, kspace, sens, mask, mu, cols=None):
        self.kspace = np.asarray(kspace, dtype=np.complex128)
        self.sens = np.asarray(sens, dtype=np.complex128)
        self.mask = np.asarray(mask, dtype=bool)
        Nx = self.sens.shape[2]
        self.cols = np.arange(Nx) if cols is None else np.asarray(cols)
        self.inv = ColumnInverse(self.sens, self.mask, mu, self.cols)
        self.b_full = adjoint_op(self.kspace, self.sens, self.mask)
        self.b = self.b_full[:, :, self.cols]
        self.yhat = hybrid_data(self.kspace, self.mask)

    def fid(self, x_cols):
        return data_residual_columns(x_cols, self.yhat, self.sens, self.mask, self.cols)

    def solve(self, prior, lam, mu, rho=0.5, iters=50, tol=0.0, objective=True, levels=2, ws=1.0, cg=5):
        """prior: "tv" (Algorithm 2), "dft" (Algorithm 1, unitary temporal DFT),
        "haar" (Algorithm 1, undecimated temporal Haar frame of ``levels`` levels)
        or "stv" (Algorithm 2 with spatio-temporal differences of spatial weight
        ``ws`` and a ``cg``-step CG m-update; needs every column)."""
        fid = self.fid if objective else None
        if prior == "stv":
            from .stv import admm_analysis_stv
            if len(self.cols) != self.sens.shape[2]:
                raise ValueError("the spatio-temporal prior couples columns: solve on all of them")
            return admm_analysis_stv(self.b, self.inv, lam, mu, rho, iters, ws=ws, cg=cg, fid=fid, tol=tol)
        if prior == "tv":
            return admm_analysis_tv(self.b, self.inv, lam, mu, rho, iters, fid=fid, tol=tol)
        if prior == "dft":
            return admm_synthesis_dft(self.b, self.inv, lam, mu, iters, fid=fid, tol=tol)
        if prior == "haar":
            return admm_synthesis_dft(self.b, self.inv, lam, mu, iters, fid=fid, tol=tol,
                                      psi=lambda z: psi_haar(z, levels), psi_adj=lambda z: psi_haar_adj(z, levels))
        raise ValueError(prior)


def make_problem(case, cols=None):
    """Oracle ``Problem`` for a ``synthdata.Case``."""
    return Problem(case.kspace, case.sens, case.mask, case.mu, cols)
