"""The persistent temporal-TV solve (all K iterations in one cooperative launch)
against the FP64 oracle and against the one-launch-per-step path.

Algorithm 2 separates along the horizontal axis (Section IV-C, Section V), so
the persistent kernel lets every column wait only for its own image column's
temporal step.  Both paths run the same arithmetic per pixel and per column;
only the FP32 rounding order of the column sums differs, so they agree to
the solver tolerance, and each matches the oracle at relative L2 1e-5.
"""

import numpy as np
import pytest

import oracle
import synthdata

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def make(name="tiny", **over):
    c = synthdata.make_case(name, **over)
    c.kspace = c.kspace.astype(np.complex64).astype(np.complex128)
    c.sens = c.sens.astype(np.complex64).astype(np.complex128)
    return c


def gpu(x):
    return torch.from_numpy(np.asarray(x, dtype=np.complex64)).cuda()


def plan(c, **opts):
    from paper_1203_4587_gb300 import Plan
    opts.setdefault("max_iters", c.iters)
    return Plan(c.mask.astype(np.uint8), gpu(c.sens), c.lam, c.mu, prior="tv", rho=c.rho, **opts)


SHAPES = [
    dict(Nx=64, Ny=64, Nt=8, Nc=4, R=4),       # tiny workload
    dict(Nx=45, Ny=40, Nt=3, Nc=3, R=3),       # ragged Ny, few frames
    dict(Nx=20, Ny=97, Nt=2, Nc=2, R=4),       # prime Ny, two frames
    dict(Nx=9, Ny=32, Nt=1, Nc=2, R=2),        # one frame: no differences
    dict(Nx=12, Ny=48, Nt=40, Nc=3, R=4),      # the largest Nt of the persistent path, 5 frames a segment
    dict(Nx=200, Ny=32, Nt=7, Nc=2, R=4),      # more image columns than CTAs
]


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "x".join(str(s[k]) for k in ("Nx", "Ny", "Nt", "Nc")))
def test_persistent_solve_matches_oracle_and_per_step(shape):
    c = make("tiny", iters=25, **shape)
    P1 = plan(c, persistent=1)
    x1, i1 = P1.solve(gpu(c.kspace))
    P0 = plan(c, persistent=0)
    x0, i0 = P0.solve(gpu(c.kspace))
    prob = oracle.Problem(c.kspace, c.sens, c.mask, c.mu)
    xr, oinfo = prob.solve("tv", c.lam, c.mu, c.rho, c.iters)
    a1 = x1.cpu().numpy().astype(np.complex128)
    a0 = x0.cpu().numpy().astype(np.complex128)
    assert rel(a1, xr) < TOL
    assert rel(a0, xr) < TOL
    assert rel(a1, a0) < TOL
    Jr = np.array(oinfo["J"])
    J1 = np.array(P1.trace(c.iters + 1))
    Ny = c.x_true.shape[1]
    bound = 2 * (1 + c.mu) * np.sqrt(Ny) * 2.0 ** -24 * np.linalg.norm(xr) ** 2 + TOL * Jr
    assert np.all(np.abs(J1 - Jr) <= bound)
    # the ADMM residuals read the same state buffers on both paths
    assert abs(i1.primal_res - i0.primal_res) <= 1e-4 * max(i0.primal_res, 1e-30)
    assert abs(i1.dual_res - i0.dual_res) <= 1e-4 * max(i0.dual_res, 1e-30)
    P1.close()
    P0.close()


def test_profile_reports_one_persistent_launch():
    c = make("tiny", iters=12)
    P = plan(c, profile=1, persistent=1)
    P.solve(gpu(c.kspace))
    pr = P.profile()
    assert pr.persistent == 1 and pr.inverse_launches == 1 and pr.inverse_passes == 12
    assert pr.temporal_launches == 1        # T_1 only; T_2..T_13 run inside the launch
    P.close()
    Q = plan(c, profile=1, persistent=0)
    Q.solve(gpu(c.kspace))
    pq = Q.profile()
    assert pq.persistent == 0 and pq.inverse_launches == 12 and pq.inverse_passes == 12
    Q.close()


def test_paths_not_eligible_run_per_step():
    """With the persistent launch asked for, an early stop (tol > 0), 16-bit
    storage with the objective, or Nt > 40 keep one launch per step; the
    default is one launch per step."""
    c = make("tiny", Nx=16, Ny=32, Nt=4, Nc=2, iters=6)
    for opts in (dict(tol=1e-9), dict(storage="fp16"), dict(objective=2)):
        P = plan(c, profile=1, persistent=1, **opts)
        P.solve(gpu(c.kspace))
        assert P.profile().persistent == 0, opts
        P.close()
    P = plan(c, profile=1)
    P.solve(gpu(c.kspace))
    assert P.profile().persistent == 0
    P.close()
    c2 = make("tiny", Nx=8, Ny=32, Nt=41, Nc=2, iters=3)
    P = plan(c2, profile=1, persistent=1)
    P.solve(gpu(c2.kspace))
    assert P.profile().persistent == 0
    P.close()


BATCH = [
    dict(Nx=24, Ny=64, Nt=6, Nc=3, R=4, seed=11),
    dict(Nx=40, Ny=40, Nt=8, Nc=4, R=3, seed=12),
    dict(Nx=16, Ny=96, Nt=5, Nc=2, R=4, seed=13),
    dict(Nx=33, Ny=128, Nt=7, Nc=3, R=6, seed=14),
    dict(Nx=70, Ny=32, Nt=16, Nc=2, R=2, seed=15),
]


def test_persistent_batch_matches_oracle_twice():
    """Uneven slices in one persistent launch; the second call replays (or
    reruns) the same sequence."""
    from paper_1203_4587_gb300 import Batch
    iters = 15
    cases = [make("tiny", iters=iters, **sh) for sh in BATCH]
    plans = [plan(c, persistent=1) for c in cases]
    batch = Batch(plans)
    ks = [gpu(c.kspace) for c in cases]
    refs = []
    for c in cases:
        prob = oracle.Problem(c.kspace, c.sens, c.mask, c.mu)
        refs.append(prob.solve("tv", c.lam, c.mu, c.rho, iters))
    for call in range(2):
        outs = batch.solve(ks)
        infos = batch.info()
        for q, (c, (xr, oinfo)) in enumerate(zip(cases, refs)):
            xb = outs[q].cpu().numpy().astype(np.complex128)
            assert rel(xb, xr) < TOL, (call, q)
            assert infos[q].iters == iters
            Jr = oinfo["J"][-1]
            Ny = c.x_true.shape[1]
            assert abs(infos[q].J - Jr) <= 2 * (1 + c.mu) * np.sqrt(Ny) * 2.0 ** -24 * np.linalg.norm(xr) ** 2 + TOL * Jr
    batch.close()
    for p in plans:
        p.close()


def test_repeated_persistent_solves_are_identical():
    """The dataflow order between CTAs varies from run to run, but every
    column's and pixel's arithmetic does not: results are bit-identical."""
    c = make("tiny", Nx=96, Ny=64, Nt=12, Nc=3, iters=20)
    P = plan(c, persistent=1)
    k = gpu(c.kspace)
    a = P.solve(k)[0].cpu().numpy()
    b = P.solve(k)[0].cpu().numpy()
    assert np.array_equal(a, b)
    P.close()
