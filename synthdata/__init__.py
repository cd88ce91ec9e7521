"""Seeded synthetic inputs for dynamic parallel MRI (cardiac-like cine).

This module is the only code shared by the FP64 oracle, the tests and the
benchmark.  It draws the random inputs and simulates the acquisition; it holds
none of the reconstruction method (no ADMM step, no Gram matrix, no inverse,
no prior).

What it produces (all NumPy, complex128 / bool / float64):

* ``x_true``  image series ``[Nt, Ny, Nx]`` (frame t, vertical j, horizontal i),
  max |x| = 1.  Sum of filled ellipses; some move periodically over t.  A
  smooth low-order phase makes the imaginary part non-trivial.
* ``sens``    coil sensitivities ``[Nc, Ny, Nx]``: complex Gaussian bumps on a
  circle of radius 1.2 around the field of view, each with a linear phase
  ramp, normalised so that sum_c |s_c|^2 = 1 at every pixel.
* ``mask``    Cartesian ky-t row mask ``[Nt, Ny]`` (bool, FFT order): kx is
  fully sampled, the same rows for every column and coil, a new random
  variable-density draw per frame, the 8 central ky lines always kept
  (Section II-A, Fig. 1: sub-sampling along the vertical axis only, changing
  with t).
* ``kspace``  ``[Nt, Nc, Ny, Nx]``: the acquisition ``M_t F_h F_v (s_c . x_t)``
  with unitary 2D FFTs (Eq. mri_csmcoill), plus circular complex Gaussian noise
  of standard deviation sigma = 0.01 * max|k| on sampled entries; unsampled
  entries are exactly 0.

The shapes and parameters of the five workloads are in ``CONFIGS``.  The
paper's own data set (a 32-coil 3T cardiac cine, Section V) is not available;
these inputs stand in for it with the same structure.
"""

from __future__ import annotations

import dataclasses
import numpy as np

__all__ = ["Case", "CONFIGS", "make_case", "make_mask", "make_sens",
           "make_phantom", "simulate_kspace", "batched_shapes"]


@dataclasses.dataclass
class Case:
    """One synthetic reconstruction problem."""
    x_true: np.ndarray      # [Nt, Ny, Nx] complex128
    sens: np.ndarray        # [Nc, Ny, Nx] complex128
    mask: np.ndarray        # [Nt, Ny] bool
    kspace: np.ndarray      # [Nt, Nc, Ny, Nx] complex128
    lam: float
    mu: float
    rho: float
    iters: int
    prior: str              # "tv" or "dft"
    seed: int

    @property
    def shape(self):
        Nt, Nc, Ny, Nx = self.kspace.shape
        return dict(Nx=Nx, Ny=Ny, Nt=Nt, Nc=Nc)


# name -> parameters.  mu is mu for the synthesis prior and mu2 for the
# analysis prior; rho = mu2/mu1.
CONFIGS = {
    "tiny": dict(Nx=64, Ny=64, Nt=8, Nc=4, R=4, lam=0.01, mu=0.1, rho=0.5,
                 iters=50, prior="tv", seed=1, moving=1),
    "cardiac": dict(Nx=256, Ny=256, Nt=32, Nc=12, R=8, lam=0.005, mu=0.1,
                    rho=0.5, iters=100, prior="tv", seed=2, moving=3),
    "precision": dict(Nx=384, Ny=384, Nt=48, Nc=16, R=6, lam=0.005, mu=0.1,
                      rho=0.5, iters=100, prior="tv", seed=3, moving=3),
    "diff": dict(Nx=192, Ny=192, Nt=24, Nc=8, R=8, lam=0.005, mu=0.1,
                 rho=0.5, iters=20, prior="tv", seed=0, moving=3),
}


def _grid(Ny, Nx):
    """Pixel-centre coordinates on [-1, 1]^2: (yy, xx) each [Ny, Nx]."""
    y = -1.0 + (2.0 * np.arange(Ny) + 1.0) / Ny
    x = -1.0 + (2.0 * np.arange(Nx) + 1.0) / Nx
    return np.meshgrid(y, x, indexing="ij")


def _ellipse(yy, xx, cy, cx, ry, rx, ang):
    ca, sa = np.cos(ang), np.sin(ang)
    u = (xx - cx) * ca + (yy - cy) * sa
    v = -(xx - cx) * sa + (yy - cy) * ca
    return (u / rx) ** 2 + (v / ry) ** 2 <= 1.0


def make_phantom(Nx, Ny, Nt, rng, moving=3):
    """Cardiac-like cine phantom [Nt, Ny, Nx], complex128, max |x| = 1.

    Static: a body ellipse (0.3) and 3-4 ellipses with intensities U(0.1,0.6).
    Dynamic: ``moving`` ellipses whose radius and intensity vary sinusoidally.
    With one moving structure the period is 8 frames; with three the periods
    are Nt/2, Nt and Nt/4 frames.
    """
    yy, xx = _grid(Ny, Nx)
    static = np.zeros((Ny, Nx))
    static[_ellipse(yy, xx, 0.0, 0.0, 0.85, 0.7, 0.0)] = 0.3
    for _ in range(int(rng.integers(3, 5))):
        cy, cx = rng.uniform(-0.5, 0.5, size=2)
        ry, rx = rng.uniform(0.08, 0.25, size=2)
        ang = rng.uniform(0, np.pi)
        static[_ellipse(yy, xx, cy, cx, ry, rx, ang)] += rng.uniform(0.1, 0.6)
    if moving == 1:
        periods = [8.0]
    else:
        periods = [Nt / 2.0, float(Nt), Nt / 4.0][:moving]
    movers = []
    for per in periods:
        movers.append(dict(cy=rng.uniform(-0.35, 0.35), cx=rng.uniform(-0.35, 0.35),
                           r0=rng.uniform(0.1, 0.2), I0=rng.uniform(0.3, 0.6),
                           per=max(per, 1.0), ph=rng.uniform(0, 2 * np.pi)))
    x = np.empty((Nt, Ny, Nx))
    for t in range(Nt):
        f = static.copy()
        for mv in movers:
            s = np.sin(2 * np.pi * t / mv["per"] + mv["ph"])
            r = mv["r0"] * (1.0 + 0.25 * s)
            f[_ellipse(yy, xx, mv["cy"], mv["cx"], r, 1.2 * r, 0.3)] += mv["I0"] * (1.0 + 0.3 * s)
        x[t] = f
    x = np.clip(x, 0.0, None)
    x /= x.max()
    phase = np.exp(1j * 0.3 * np.pi * (xx + yy) / 2.0)
    return x * phase[None]


def make_sens(Nx, Ny, Nc, rng=None, phase_y=0.0):
    """Smooth coil sensitivities [Nc, Ny, Nx], normalised sum_c |s_c|^2 = 1.

    The phase of coil c is th_c + 0.5 x (+ phase_y cos(th_c) y).  With
    phase_y = 0 it is constant along every image column, so each column's coil
    Gram sum_c conj(s_j) s_k is real; phase_y != 0 makes it complex, which is
    what distinguishes conj(s_j) s_k from s_j conj(s_k) (Eq. HconjH)."""
    yy, xx = _grid(Ny, Nx)
    s = np.empty((Nc, Ny, Nx), dtype=np.complex128)
    for c in range(Nc):
        th = 2 * np.pi * c / Nc
        cy, cx = 1.2 * np.sin(th), 1.2 * np.cos(th)
        mag = np.exp(-((xx - cx) ** 2 + (yy - cy) ** 2) / (2 * 0.8 ** 2))
        s[c] = mag * np.exp(1j * (th + 0.5 * xx + phase_y * np.cos(th) * yy))
    s /= np.sqrt(np.sum(np.abs(s) ** 2, axis=0, keepdims=True))
    return s


def make_mask(Ny, Nt, R, rng, ncentre=8):
    """Variable-density random Cartesian ky-t mask [Nt, Ny] (bool, FFT order).

    Per frame ``round(Ny/R)`` rows: the ``ncentre`` central rows (centred
    ky in [-ncentre/2, ncentre/2 - 1]) plus rows drawn without replacement
    with probability proportional to (1 - |ky|/(Ny/2))^2 + 0.01.
    """
    m = int(round(Ny / R))
    m = max(1, min(m, Ny))
    kyc = np.arange(Ny) - Ny // 2                 # centred coordinate
    idx = np.mod(kyc, Ny)                         # FFT-order index of each kyc
    mask = np.zeros((Nt, Ny), dtype=bool)
    central = (kyc >= -(ncentre // 2)) & (kyc <= ncentre // 2 - 1)
    ncen = int(min(central.sum(), m))
    cen_pos = np.nonzero(central)[0][:ncen]
    rest = np.setdiff1d(np.arange(Ny), cen_pos)
    p = (1.0 - np.abs(kyc[rest]) / (Ny / 2.0)) ** 2 + 0.01
    p = p / p.sum()
    for t in range(Nt):
        pick = rng.choice(rest, size=m - ncen, replace=False, p=p) if m > ncen else []
        rows = np.concatenate([cen_pos, np.asarray(pick, dtype=int)])
        mask[t, idx[rows]] = True
    return mask


def simulate_kspace(x, sens, mask, rng, noise=0.01):
    """Acquisition y = M_t F (s_c . x_t) + n (unitary 2D FFT), [Nt, Nc, Ny, Nx].

    Noise: circular complex Gaussian, E|n|^2 = sigma^2 with
    sigma = noise * max|k| over the noiseless sampled entries; unsampled
    entries are exactly zero.
    """
    k = np.fft.fft2(sens[None, :, :, :] * x[:, None, :, :], axes=(-2, -1), norm="ortho")
    sel = mask[:, None, :, None]
    k = np.where(sel, k, 0.0)
    if noise > 0:
        sigma = noise * np.abs(k).max()
        n = (rng.standard_normal(k.shape) + 1j * rng.standard_normal(k.shape)) * (sigma / np.sqrt(2.0))
        k = np.where(sel, k + n, 0.0)
    return k


def make_case(name="tiny", seed=None, **over) -> Case:
    """Build one seeded problem of the named workload (parameters overridable)."""
    cfg = dict(CONFIGS[name]) if name in CONFIGS else {}
    cfg.update(over)
    if seed is not None:
        cfg["seed"] = seed
    rng = np.random.default_rng(cfg["seed"])
    Nx, Ny, Nt, Nc = cfg["Nx"], cfg["Ny"], cfg["Nt"], cfg["Nc"]
    x = make_phantom(Nx, Ny, Nt, rng, moving=cfg.get("moving", 3))
    sens = make_sens(Nx, Ny, Nc, phase_y=cfg.get("phase_y", 0.0))
    mask = cfg.get("mask")
    if mask is None:
        mask = make_mask(Ny, Nt, cfg["R"], rng)
    k = simulate_kspace(x, sens, mask, rng, noise=cfg.get("noise", 0.01))
    return Case(x_true=x, sens=sens, mask=np.asarray(mask, bool), kspace=k,
                lam=float(cfg["lam"]), mu=float(cfg["mu"]), rho=float(cfg.get("rho", 0.5)),
                iters=int(cfg["iters"]), prior=cfg.get("prior", "tv"), seed=int(cfg["seed"]))


def batched_shapes(n=64, seed=64):
    """Uneven slice shapes of the batched workload: list of dicts.

    Nx, Ny drawn from {128,160,192,256}, Nt from {16,24,32,40}, Nc from
    {8,12,16}, R from {4,6,8}; each slice gets its own seed.
    """
    rng = np.random.default_rng(seed)
    out = []
    for s in range(n):
        out.append(dict(Nx=int(rng.choice([128, 160, 192, 256])),
                        Ny=int(rng.choice([128, 160, 192, 256])),
                        Nt=int(rng.choice([16, 24, 32, 40])),
                        Nc=int(rng.choice([8, 12, 16])),
                        R=int(rng.choice([4, 6, 8])),
                        lam=0.005, mu=0.1, rho=0.5, iters=80, prior="tv",
                        seed=1000 + s, moving=3))
    return out
