"""GPU parity of Algorithm 1 with the undecimated temporal Haar frame (a
redundant tight frame: the lemma of Section IV-A keeps its (1/mu)(I - Psi Psi')
term) against the FP64 oracle.  Same bar as the other priors: relative L2
image error <= 1e-5 and J(k) within 1e-5 relative (exact objective) or the
fused objective's bound.
"""

import numpy as np
import pytest

import oracle
import synthdata

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300))


def as64(x):
    return np.asarray(x, dtype=np.complex64).astype(np.complex128)


def gpu(x):
    return torch.from_numpy(np.asarray(x, dtype=np.complex64)).cuda()


def host(t):
    return t.detach().cpu().numpy().astype(np.complex128)


def make(name="tiny", **over):
    case = synthdata.make_case(name, **over)
    case.kspace = as64(case.kspace)
    case.sens = as64(case.sens)
    return case


def plan_for(case, levels, **opts):
    from paper_1203_4587_gb300 import Plan
    opts.setdefault("max_iters", case.iters)
    return Plan(case.mask.astype(np.uint8), gpu(case.sens), case.lam, case.mu, prior="haar", rho=case.rho,
                frame_levels=levels, **opts)


def oracle_solve(case, levels, iters, cols=None, objective=True):
    prob = oracle.Problem(case.kspace, case.sens, case.mask, case.mu, cols)
    return prob.solve("haar", case.lam, case.mu, case.rho, iters, levels=levels, objective=objective)


@pytest.mark.parametrize("objective", [1, 2], ids=["fused_objective", "exact_objective"])
@pytest.mark.parametrize("levels", [1, 2, 3])
def test_tiny_workload_parity(levels, objective):
    """64x64, 8 frames, 4 coils, R=4, lambda=0.01, mu=0.1, 50 iterations."""
    case = make("tiny")
    P = plan_for(case, levels, objective=objective)
    x, info = P.solve(gpu(case.kspace))
    xr, oinfo = oracle_solve(case, levels, case.iters)
    assert info.iters == case.iters
    assert rel(host(x), xr) < TOL
    J = np.array(P.trace(case.iters + 1))
    Jr = np.array(oinfo["J"])
    if objective == 2:
        assert np.max(np.abs(J - Jr) / Jr) < TOL
    else:
        Ny = case.x_true.shape[1]
        bound = 2 * (1 + case.mu) * np.sqrt(Ny) * 2.0 ** -24 * np.linalg.norm(xr) ** 2 + TOL * Jr
        assert np.all(np.abs(J - Jr) <= bound)


@pytest.mark.parametrize("shape", [dict(Nx=12, Ny=16, Nt=1, Nc=2, R=2),     # one frame: details are 0
                                   dict(Nx=10, Ny=32, Nt=2, Nc=3, R=2),
                                   dict(Nx=18, Ny=40, Nt=5, Nc=2, R=3),     # shifts 1, 2, 4 wrap mod 5
                                   dict(Nx=8, Ny=64, Nt=7, Nc=2, R=4),
                                   dict(Nx=6, Ny=32, Nt=24, Nc=2, R=4)],
                         ids=lambda s: "x".join(str(s[k]) for k in ("Nx", "Ny", "Nt", "Nc")))
def test_edge_shapes(shape):
    case = make("tiny", **shape)
    iters, levels = 12, 3
    P = plan_for(case, levels, max_iters=iters, objective=2)
    x, _ = P.solve(gpu(case.kspace))
    xr, oinfo = oracle_solve(case, levels, iters)
    assert rel(host(x), xr) < TOL
    J = np.array(P.trace(iters + 1))
    Jr = np.array(oinfo["J"])
    assert np.max(np.abs(J - Jr) / Jr) < TOL


def test_cardiac_workload_column_subset():
    """256x256, 32 frames, 12 coils, R=8, 100 iterations, 2 levels: a seeded
    subset of columns (columns are independent) against the oracle."""
    case = make("cardiac")
    P = plan_for(case, 2, objective=0)
    x, _ = P.solve(gpu(case.kspace), info=False)
    cols = np.sort(np.random.default_rng(8).choice(256, size=3, replace=False))
    xr, _ = oracle_solve(case, 2, case.iters, cols=cols, objective=False)
    assert rel(host(x)[:, :, cols], xr) < TOL


def test_batched_haar_matches_single_solves():
    from paper_1203_4587_gb300 import Batch
    shapes = [dict(Nx=24, Ny=64, Nt=6, Nc=3, seed=41), dict(Nx=40, Ny=40, Nt=8, Nc=4, seed=42),
              dict(Nx=16, Ny=96, Nt=5, Nc=2, seed=43)]
    cases = [make("tiny", **sh) for sh in shapes]
    iters, levels = 15, 2
    plans = [plan_for(c, levels, max_iters=iters) for c in cases]
    b = Batch(plans)
    xs = b.solve([gpu(c.kspace) for c in cases])
    for c, x in zip(cases, xs):
        xr, _ = oracle_solve(c, levels, iters, objective=False)
        assert rel(host(x), xr) < TOL


def test_invalid_levels_rejected():
    from paper_1203_4587_gb300 import ReconError
    case = make("tiny", Nx=16, Ny=32, Nt=4, Nc=2)
    for bad in (0, 7):
        with pytest.raises(ReconError):
            plan_for(case, bad, max_iters=2)
