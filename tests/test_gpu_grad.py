"""GPU parity of the differentiable unrolled Algorithm 2 (recon_grad_*).

The reverse pass on the GPU is compared with the FP64 oracle gradient
(``oracle.grad``, itself pinned by finite differences on the CPU) for
L = ||x_K - x_true||^2.  The GPU's backward is fed the oracle's
dL/dx_K = 2 (x_K - x_true), so only the reverse pass is under test (the
forward image is checked separately at the solver tolerance TOL).

The gradient is only piecewise smooth: the soft threshold's Jacobian jumps
where |a| = tau (the threshold gives exactly 0 for |a| <= tau and its
derivative there is taken from that zero side).  The GPU decides |a| > tau on its FP32 states,
the oracle on its FP64 states, and the two trajectories differ by ~1e-6
relative, so any |a| within about 1e-5 relative of tau may take opposite
branches on the two sides.  Hence two bounds:

* kink-free inputs (lambda = 3e-4: the oracle checks that no |a| of any step
  lies within 1e-3 relative of tau, while some values stay below it):
  GTOL = 2e-5 on dL/dy and STOL = 1e-4 on dL/dlambda, dL/dmu.  An FP32
  emulation of these reverse steps in NumPy lands within 7e-6 (b_bar) and
  3e-6 (dL/dy) of FP64; the bounds allow ~3-7x that.
* the workloads' lambda: a 1e-6 relative perturbation of y (the size of the
  GPU's forward error) moves the oracle's own dL/dy by 1.2e-4 and its scalar
  gradients by 1e-5 on the tiny workload, through such branch flips.  KTOL =
  1e-3 on dL/dy and KSTOL = 2e-4 on the scalars cover that with margin.

Separately the GPU gradient is checked against central finite differences
of the GPU's own forward on kink-free inputs (FDTOL = 5e-3: in FP64 the same
differences land within 3e-5 of the oracle's derivatives; FP32 rounding of
the loss adds up to ~1e-3 for the lambda step).
"""

import numpy as np
import pytest

import oracle
import synthdata

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5
GTOL = 2e-5
STOL = 1e-4
KTOL = 1e-3
KSTOL = 2e-4
KTOL_SUBSET = 5e-3
FDTOL = 5e-3
LAM_SMOOTH = 3e-4


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300))


def as64(x):
    return np.asarray(x, dtype=np.complex64).astype(np.complex128)


def gpu(x):
    return torch.from_numpy(np.asarray(x, dtype=np.complex64)).cuda()


def host(t):
    return t.detach().cpu().numpy().astype(np.complex128)


def make(name, **over):
    case = synthdata.make_case(name, **over)
    case.kspace = as64(case.kspace)
    case.sens = as64(case.sens)
    return case


def plan_for(case, iters, **opts):
    from paper_1203_4587_gb300 import Plan
    return Plan(case.mask.astype(np.uint8), gpu(case.sens), case.lam, case.mu, prior="tv", rho=case.rho,
                max_iters=iters, objective=0, tol=0.0, **opts)


def oracle_state(case, iters, cols=None):
    """(b, inverse, x_K) of the oracle on the given columns."""
    b = oracle.adjoint_op(case.kspace, case.sens, case.mask)
    inv = oracle.ColumnInverse(case.sens, case.mask, case.mu, cols)
    if cols is not None:
        b = b[:, :, cols]
    S = oracle.unrolled_tv_forward(b, inv, case.lam, case.mu, case.rho, iters)
    return b, inv, S[-1][0]


def kink_margin(case, b, inv, lam, iters):
    """min over steps and values of ||a| - tau| / tau in the oracle's forward."""
    S = oracle.unrolled_tv_forward(b, inv, lam, case.mu, case.rho, iters)
    tau = lam * case.rho / (2.0 * case.mu)
    out, below = np.inf, 0
    for k in range(iters):
        x0, m0, d10, _ = S[k]
        a = np.abs(oracle.tv_D(m0) + d10)
        out = min(out, float(np.min(np.abs(a - tau)) / tau))
        below += int(np.sum(a <= tau))
    return out, below


def small_case(case, iters, every, lam):
    from paper_1203_4587_gb300 import Grad, Plan
    case.lam = lam
    P = plan_for(case, iters)
    G = Grad([P], checkpoint_every=every)
    x = host(G.forward([gpu(case.kspace)])[0])
    b, inv, xK = oracle_state(case, iters)
    assert rel(x, xK) < TOL
    xb = 2.0 * (xK - case.x_true)
    gk, gl, gm = G.backward([gpu(xb)])
    L, gy, gl_ref, gm_ref, bb = oracle.unrolled_tv_loss_and_grad(case.kspace, case.sens, case.mask, case.x_true,
                                                                 case.lam, case.mu, case.rho, iters)
    return G, xb, (host(gk[0]), gl[0], gm[0]), (gy, gl_ref, gm_ref), (b, inv)


@pytest.mark.parametrize("iters,every", [(12, 5), (7, 1), (6, 6)], ids=["K12_every5", "K7_every1", "K6_every6"])
def test_gradient_matches_oracle_kink_free(iters, every):
    """64x64, 8 frames, 4 coils, R=4, lambda = 3e-4: every gradient on the whole field."""
    case = make("tiny")
    G, xb, (gk, gl, gm), (gy, gl_ref, gm_ref), (b, inv) = small_case(case, iters, every, LAM_SMOOTH)
    margin, below = kink_margin(case, b, inv, LAM_SMOOTH, iters)
    assert margin > 1e-3 and below > 0          # precondition of GTOL: no value near the kink, both branches used
    assert rel(gk, gy) < GTOL
    assert abs(gl - gl_ref) <= STOL * abs(gl_ref)
    assert abs(gm - gm_ref) <= STOL * abs(gm_ref)
    # unsampled rows of dL/dy are exactly zero
    assert np.all(gk[~np.broadcast_to(case.mask[:, None, :, None], gk.shape)] == 0)
    # a second backward with the same forward gives the same result
    gk2, gl2, gm2 = G.backward([gpu(xb)])
    assert rel(host(gk2[0]), gk) < 1e-6 and abs(gl2[0] - gl) <= 1e-6 * abs(gl)


@pytest.mark.parametrize("iters", [12, 50])
def test_gradient_matches_oracle_workload_lambda(iters):
    """The tiny workload's own lambda = 0.01 (values near the kink): KTOL, KSTOL."""
    case = make("tiny")
    G, xb, (gk, gl, gm), (gy, gl_ref, gm_ref), _ = small_case(case, iters, 5, case.lam)
    assert rel(gk, gy) < KTOL
    assert abs(gl - gl_ref) <= KSTOL * abs(gl_ref)
    assert abs(gm - gm_ref) <= KSTOL * abs(gm_ref)


def test_gradient_matches_finite_differences_of_gpu_forward():
    """Central differences of L(y, lambda, mu) = ||x_K - x_true||^2 through the
    GPU forward against the GPU backward (directional derivatives)."""
    from paper_1203_4587_gb300 import Grad
    case = make("tiny", Nx=48, Ny=64, Nt=6, Nc=3)
    case.lam = LAM_SMOOTH
    iters = 10
    xt = as64(case.x_true)

    def loss(kspace, lam, mu):
        c = make("tiny", Nx=48, Ny=64, Nt=6, Nc=3)
        c.lam, c.mu = lam, mu
        G = Grad([plan_for(c, iters)], checkpoint_every=5)
        x = host(G.forward([gpu(kspace)])[0])
        G.close()
        return float(np.sum(np.abs(x - xt) ** 2)), x

    L0, x0 = loss(case.kspace, case.lam, case.mu)
    G = Grad([plan_for(case, iters)], checkpoint_every=5)
    G.forward([gpu(case.kspace)])
    gk, gl, gm = G.backward([gpu(2.0 * (x0 - xt))])
    gk = host(gk[0])
    h = 3e-3
    # lambda and mu: relative steps
    for which, g in (("lam", gl[0]), ("mu", gm[0])):
        v = case.lam if which == "lam" else case.mu
        args_p = (case.lam * (1 + h), case.mu) if which == "lam" else (case.lam, case.mu * (1 + h))
        args_m = (case.lam * (1 - h), case.mu) if which == "lam" else (case.lam, case.mu * (1 - h))
        fd = (loss(case.kspace, *args_p)[0] - loss(case.kspace, *args_m)[0]) / (2 * h * v)
        assert abs(fd - g) <= FDTOL * abs(g), (which, fd, g)
    # k-space: along the GPU's own dL/dy (the largest directional derivative,
    # so FP32 rounding of L matters least), |delta| = |y|, step 1e-3
    d = gk / np.linalg.norm(gk) * np.linalg.norm(case.kspace)
    hy = 1e-3
    fd = (loss(case.kspace + hy * d, case.lam, case.mu)[0] - loss(case.kspace - hy * d, case.lam, case.mu)[0]) / (2 * hy)
    dd = float(np.real(np.vdot(gk, d)))
    assert abs(fd - dd) <= FDTOL * abs(dd), (fd, dd)


def test_autograd_function():
    """torch.autograd through unrolled_tv equals the explicit backward."""
    from paper_1203_4587_gb300 import Grad, unrolled_tv
    case = make("tiny", Nx=48, Ny=64, Nt=6, Nc=3)
    iters = 8
    P = plan_for(case, iters)
    G = Grad([P], checkpoint_every=3)
    k = gpu(case.kspace).requires_grad_(True)
    lam = torch.tensor([case.lam], dtype=torch.float64, requires_grad=True)
    mu = torch.tensor([case.mu], dtype=torch.float64, requires_grad=True)
    xt = gpu(case.x_true)
    (x,) = unrolled_tv(G, [k], lam, mu)
    loss = torch.sum(torch.abs(x - xt) ** 2)
    loss.backward()
    xb = 2.0 * (host(x) - as64(case.x_true))
    gk, gl, gm = G.backward([gpu(xb)])
    assert rel(host(k.grad), host(gk[0])) < 1e-5
    assert abs(lam.grad.item() - gl[0]) <= 1e-5 * abs(gl[0])
    assert abs(mu.grad.item() - gm[0]) <= 1e-5 * abs(gm[0])
    _, gy, gl_ref, gm_ref, _ = oracle.unrolled_tv_loss_and_grad(case.kspace, case.sens, case.mask, case.x_true,
                                                                case.lam, case.mu, case.rho, iters)
    assert rel(host(k.grad), gy) < KTOL
    assert abs(lam.grad.item() - gl_ref) <= KSTOL * abs(gl_ref)
    assert abs(mu.grad.item() - gm_ref) <= KSTOL * abs(gm_ref)
    with pytest.raises(ValueError):
        unrolled_tv(G, [k], lam * 2, mu)


@pytest.mark.parametrize("regime", ["kink_free", "workload_lambda"])
def test_gradient_batch_of_four_column_subset(regime):
    """192x192, 24 frames, 8 coils, R=8, 20 iterations, 4 slices in one
    gradient batch.  The loss weights only a seeded subset of columns of each
    slice (columns are independent), so the oracle's gradient on that subset
    is the whole gradient: dL/dlambda and dL/dmu compare directly, and dL/dy
    through H' dL/dy = H'H b_bar, which on a column equals G_{i,t} b_bar.

    kink_free: lambda = 1e-4 (the oracle checks the margin): GTOL, STOL.
    workload_lambda: lambda = 0.005.  A branch flip's effect is measured
    against the norm of only 5 of 192 columns here, so the bound on H' dL/dy
    is KTOL_SUBSET = 5e-3 (the full-field equivalent is KTOL); scalars KSTOL."""
    from paper_1203_4587_gb300 import Grad
    cases = [make("diff", seed=q) for q in range(4)]
    if regime == "kink_free":
        for c in cases:
            c.lam = 1e-4
    vtol, stol = (GTOL, STOL) if regime == "kink_free" else (KTOL_SUBSET, KSTOL)
    iters = cases[0].iters
    plans = [plan_for(c, iters) for c in cases]
    G = Grad(plans, checkpoint_every=5)
    xs = [host(x) for x in G.forward([gpu(c.kspace) for c in cases])]
    rng = np.random.default_rng(11)
    gimg, refs = [], []
    below = 0
    for c, x in zip(cases, xs):
        Nx = c.x_true.shape[2]
        cols = np.sort(rng.choice(Nx, size=5, replace=False))
        b, inv, xK = oracle_state(c, iters, cols)
        assert rel(x[:, :, cols], xK) < TOL
        if regime == "kink_free":
            margin, nb = kink_margin(c, b, inv, c.lam, iters)
            assert margin > 1e-3
            below += nb
        xt = c.x_true[:, :, cols]
        g = np.zeros_like(c.x_true, dtype=np.complex128)
        g[:, :, cols] = 2.0 * (xK - xt)
        gimg.append(gpu(g))
        L, bb, gl_ref, gm_ref = oracle.unrolled_tv_adjoint(b, inv, xt, c.lam, c.mu, c.rho, iters)
        refs.append((cols, inv, bb, gl_ref, gm_ref))
    if regime == "kink_free":
        assert below > 0
    gk, gl, gm = G.backward(gimg)
    for q, (c, (cols, inv, bb, gl_ref, gm_ref)) in enumerate(zip(cases, refs)):
        hty = oracle.adjoint_op(host(gk[q]), c.sens, c.mask)[:, :, cols]
        ref = np.einsum("tijk,tki->tji", inv.G, bb)
        assert rel(hty, ref) < vtol, q
        assert abs(gl[q] - gl_ref) <= stol * abs(gl_ref), q
        assert abs(gm[q] - gm_ref) <= stol * abs(gm_ref), q


def test_grad_rejects_bad_arguments():
    from paper_1203_4587_gb300 import Grad, Plan, ReconError
    case = make("tiny", Nx=16, Ny=32, Nt=3, Nc=2)
    Pd = Plan(case.mask.astype(np.uint8), gpu(case.sens), case.lam, case.mu, prior="dft", max_iters=3)
    with pytest.raises(ReconError):
        Grad([Pd])
    P3 = plan_for(case, 3)
    P4 = plan_for(case, 4)
    with pytest.raises(ReconError):
        Grad([P3, P4])
