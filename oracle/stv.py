"""FP64 oracle: Algorithm 2 with a spatio-temporal analysis operator whose
m-update is solved by conjugate gradients (test infrastructure only).

Section IV-B notes that (mu2/mu1 I + R'R)^{-1} has a closed form for many
common R and can otherwise be computed with a few conjugate-gradient (CG)
iterations.  Here R stacks non-circular finite differences along time and
both image axes,

    R x = ( D_t x,  w D_x x,  w D_y x ),

with D_t as in Eq. TV, D_x along the horizontal index i and D_y along the
vertical index j (x[t, j, i], as in ``admm.py``), and a spatial weight w >= 0.
The l1 term is anisotropic: ||R x||_1 sums the complex moduli of all three
components, and the soft threshold acts element by element (Section III).

The m-update of Algorithm 2 takes ``cg_steps`` CG steps on the Hermitian
positive definite system (rho I + R'R) m = rhs (rho = mu2/mu1), started
from the previous m (m = x = H'y at the first iteration).  The CG steps are
the textbook recurrence (Hestenes-Stiefel):

    r = rhs - M m,  p = r,  gamma = <r, r>
    repeat: q = M p,  alpha = gamma / <p, q>,  m += alpha p,  r -= alpha q,
            gamma' = <r, r>,  p = r + (gamma'/gamma) p,  gamma = gamma'

stopping early only when gamma = 0 (then m solves the system exactly).

Parity status: pinned in ``tests/test_oracle_stv.py`` (adjointness of R,
R'R against a dense brute-force matrix, CG against an exact solve and
against the DCT-II diagonalisation of the non-circular Laplacians, w = 0
against the temporal-TV oracle, KKT optimality of the ADMM fixed point; the
stacked residuals against the d1 change, the temporal-TV residuals at w = 0,
a volume of one slice and their decay at the fixed point).
"""

from __future__ import annotations

import numpy as np

from .admm import delta_ratio, soft

__all__ = ["stv_R", "stv_Radj", "stv_M", "cg_steps", "objective_stv", "admm_analysis_stv",
           "stv_R_vol", "stv_Radj_vol", "stv_M_vol", "objective_stv_vol", "admm_analysis_stv_volume",
           "stacked_residuals"]


def stv_R(x, ws):
    """R x = (D_t x, w D_x x, w D_y x); shapes (Nt-1, Ny, Nx), (Nt, Ny, Nx-1),
    (Nt, Ny-1, Nx)."""
    x = np.asarray(x)
    return (x[1:] - x[:-1], ws * (x[:, :, 1:] - x[:, :, :-1]), ws * (x[:, 1:, :] - x[:, :-1, :]))


def _diff_adj(u, axis, n):
    """Adjoint of the forward difference along ``axis`` (length n): for
    (D a)_k = a_{k+1} - a_k, k < n-1, (D' u)_s = u_{s-1} - u_s with
    u_{-1} = u_{n-1} = 0."""
    shape = list(u.shape)
    shape[axis] = n
    out = np.zeros(shape, dtype=np.result_type(u, np.complex128))
    lo = [slice(None)] * u.ndim
    hi = [slice(None)] * u.ndim
    lo[axis] = slice(0, n - 1)
    hi[axis] = slice(1, n)
    out[tuple(lo)] -= u
    out[tuple(hi)] += u
    return out


def stv_Radj(u, ws, shape):
    """R' (ut, ux, uy) = D_t' ut + w D_x' ux + w D_y' uy, image of ``shape``."""
    ut, ux, uy = u
    Nt, Ny, Nx = shape
    return _diff_adj(ut, 0, Nt) + ws * _diff_adj(ux, 2, Nx) + ws * _diff_adj(uy, 1, Ny)


def stv_M(m, rho, ws):
    """(rho I + R'R) m."""
    return rho * m + stv_Radj(stv_R(m, ws), ws, m.shape)


def _dot(a, b):
    """<a, b> = sum conj(a) b."""
    return np.vdot(a, b)


def cg_steps(apply_M, rhs, m0, steps):
    """``steps`` CG steps on M m = rhs from m0 (M Hermitian positive definite)."""
    m = np.array(m0, dtype=np.complex128)
    r = rhs - apply_M(m)
    p = r.copy()
    gamma = _dot(r, r).real
    for _ in range(steps):
        if gamma == 0.0:
            break
        q = apply_M(p)
        alpha = gamma / _dot(p, q).real
        m = m + alpha * p
        r = r - alpha * q
        gamma_new = _dot(r, r).real
        p = r + (gamma_new / gamma) * p
        gamma = gamma_new
    return m


def objective_stv(x, lam, ws, fid):
    """J = lambda ||R x||_1 + ||y - H x||^2 (Eq. L1an_pri with R above)."""
    return lam * float(sum(np.abs(c).sum() for c in stv_R(x, ws))) + fid(x)


def admm_analysis_stv(b, inv, lam, mu, rho, iters, ws=1.0, cg=5, fid=None, tol=0.0, state=None):
    """Algorithm 2 (ADMM_Analysis) with R = (D_t, w D_x, w D_y) and a CG
    m-update of ``cg`` steps.  b = H'y on the full image grid; mu2 = mu,
    mu1 = mu/rho.  Returns (x, info) like ``admm.admm_analysis_tv``;
    ``state`` = (x, m, d1, d2) with d1 a tuple of the three components."""
    shape = b.shape
    mu2 = mu
    mu1 = mu / rho
    r2 = mu2 / mu1

    def M(a):
        return stv_M(a, r2, ws)

    if state is None:
        x = b.copy()                                            # x = H'y
        m = x.copy()                                            # m = x
        d1 = tuple(np.zeros_like(c) for c in stv_R(x, ws))
        d2 = np.zeros_like(b)
    else:
        x, m, d1, d2 = state
        x, m, d2 = (np.array(a, dtype=np.complex128) for a in (x, m, d2))
        d1 = tuple(np.array(a, dtype=np.complex128) for a in d1)
    J = [objective_stv(x, lam, ws, fid)] if fid is not None else []
    k_done = 0
    m_prev = v = None
    for k in range(1, iters + 1):
        m_prev = m
        # v <- S(R m + d1, lambda / (2 mu1))
        Rm = stv_R(m, ws)
        v = tuple(soft(a + d, lam / (2.0 * mu1)) for a, d in zip(Rm, d1))
        # m <- (mu2/mu1 I + R'R)^{-1} [R'(v - d1) + mu2/mu1 (x + d2)]   (CG)
        rhs = stv_Radj(tuple(a - d for a, d in zip(v, d1)), ws, shape) + r2 * (x + d2)
        m = cg_steps(M, rhs, m, cg)
        # x <- (mu2 I + H'H)^{-1} [H'y + mu2 (m - d2)]
        x = inv.apply(b + mu2 * (m - d2))
        # d1 <- d1 - (v - R m);  d2 <- d2 - (m - x)
        Rm = stv_R(m, ws)
        d1 = tuple(d - (a - c) for d, a, c in zip(d1, v, Rm))
        d2 = d2 - (m - x)
        k_done = k
        if fid is not None:
            J.append(objective_stv(x, lam, ws, fid))
            if tol > 0:
                dk = delta_ratio(J[-2], J[-1])
                if 0.0 <= dk < tol:
                    break
    info = dict(J=J, iters=k_done, state=(x, m, d1, d2))
    if m_prev is not None:
        info["primal_res"], info["dual_res"] = stacked_residuals(x, m, v, m_prev, mu1, mu2,
                                                                 lambda a: stv_R(a, ws))
    return x, info


def stacked_residuals(x, m, v, m_prev, mu1, mu2, R):
    """ADMM residuals of Algorithm 2 with a stacked analysis operator R (a tuple
    of components), in the stacked form of Boyd et al. (2011, Sec. 3.3) for the
    splits v = R m (mu1) and m = x (mu2), m updated second:
      primal = sqrt(sum_c ||v_c - (R m)_c||^2 + ||m - x||^2)
      dual   = sqrt(mu1^2 sum_c ||(R (m - m_prev))_c||^2 + mu2^2 ||m - m_prev||^2)."""
    rp = sum(np.vdot(a - b, a - b).real for a, b in zip(v, R(m))) + np.vdot(m - x, m - x).real
    dm = m - m_prev
    rd = mu1 ** 2 * sum(np.vdot(c, c).real for c in R(dm)) + mu2 ** 2 * np.vdot(dm, dm).real
    return float(np.sqrt(rp)), float(np.sqrt(rd))


# ---------------------------------------------------------------------------
# 3D volumes (Section II-A: the model extends from 2D slices to volumes).
# With kz fully sampled, an inverse FFT along z separates the volume into
# slices, each with its own ky-t mask, coil profiles and per-column inverses
# (Section IV-C holds slice by slice).  The slices are then coupled only by a
# z-difference in R:
#     R x = (D_t x, w D_x x, w D_y x, w_z D_z x),   x[z, t, j, i],
# and the m-update's CG runs on the whole volume (inner products over every
# slice).  A volume of one slice is the 2D algorithm above.
# ---------------------------------------------------------------------------
def stv_R_vol(x, ws, wz):
    """R x for x[z, t, j, i]: (D_t, w D_x, w D_y, w_z D_z), non-circular."""
    x = np.asarray(x)
    return (x[:, 1:] - x[:, :-1], ws * (x[:, :, :, 1:] - x[:, :, :, :-1]), ws * (x[:, :, 1:, :] - x[:, :, :-1, :]),
            wz * (x[1:] - x[:-1]))


def stv_Radj_vol(u, ws, wz, shape):
    ut, ux, uy, uz = u
    Nz, Nt, Ny, Nx = shape
    return (_diff_adj(ut, 1, Nt) + ws * _diff_adj(ux, 3, Nx) + ws * _diff_adj(uy, 2, Ny)
            + wz * _diff_adj(uz, 0, Nz))


def stv_M_vol(m, rho, ws, wz):
    return rho * m + stv_Radj_vol(stv_R_vol(m, ws, wz), ws, wz, m.shape)


def objective_stv_vol(x, lam, ws, wz, fids):
    """J = lambda ||R x||_1 + sum_z ||y_z - H_z x_z||^2."""
    return lam * float(sum(np.abs(c).sum() for c in stv_R_vol(x, ws, wz))) + sum(f(xz) for f, xz in zip(fids, x))


def admm_analysis_stv_volume(bs, invs, lam, mu, rho, iters, ws=1.0, wz=1.0, cg=5, fids=None):
    """Algorithm 2 on a volume of slices: bs[z] = H_z'y_z, invs[z] the slice's
    column inverses; the same steps as ``admm_analysis_stv`` with the 4-component
    R above and one CG over the volume.  Returns (x[z, t, j, i], info)."""
    b = np.stack([np.asarray(v, dtype=np.complex128) for v in bs])
    shape = b.shape
    mu2 = mu
    mu1 = mu / rho
    r2 = mu2 / mu1

    def M(a):
        return stv_M_vol(a, r2, ws, wz)

    def inverse(r):
        return np.stack([inv.apply(rz) for inv, rz in zip(invs, r)])

    x = b.copy()
    m = x.copy()
    d1 = tuple(np.zeros_like(c) for c in stv_R_vol(x, ws, wz))
    d2 = np.zeros_like(b)
    J = [objective_stv_vol(x, lam, ws, wz, fids)] if fids is not None else []
    m_prev = v = None
    for _ in range(iters):
        m_prev = m
        Rm = stv_R_vol(m, ws, wz)
        v = tuple(soft(a + d, lam / (2.0 * mu1)) for a, d in zip(Rm, d1))
        rhs = stv_Radj_vol(tuple(a - d for a, d in zip(v, d1)), ws, wz, shape) + r2 * (x + d2)
        m = cg_steps(M, rhs, m, cg)
        x = inverse(b + mu2 * (m - d2))
        Rm = stv_R_vol(m, ws, wz)
        d1 = tuple(d - (a - c) for d, a, c in zip(d1, v, Rm))
        d2 = d2 - (m - x)
        if fids is not None:
            J.append(objective_stv_vol(x, lam, ws, wz, fids))
    info = dict(J=J, iters=iters, state=(x, m, d1, d2))
    if m_prev is not None:
        info["primal_res"], info["dual_res"] = stacked_residuals(x, m, v, m_prev, mu1, mu2,
                                                                 lambda a: stv_R_vol(a, ws, wz))
    return x, info
