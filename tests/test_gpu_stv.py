"""GPU parity of Algorithm 2 with the spatio-temporal analysis operator
R = (D_t, w D_x, w D_y) and the CG m-update against the FP64 oracle (the same
number of CG steps from the same start, Section IV-B).

Bar: relative L2 image error <= 1e-5 (FP32 path, FP64 oracle) and J(k)
within 1e-5 relative (exact objective) or the fused objective's bound.  The
CG inner products are FP64 sums of FP32 products, alpha and beta FP64.
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


def plan_for(case, ws, cg, **opts):
    from paper_1203_4587_gb300 import Plan
    opts.setdefault("max_iters", case.iters)
    return Plan(case.mask.astype(np.uint8), gpu(case.sens), case.lam, case.mu, prior="stv", rho=case.rho,
                spatial_weight=ws, cg_steps=cg, **opts)


def oracle_solve(case, ws, cg, iters, objective=True):
    prob = oracle.Problem(case.kspace, case.sens, case.mask, case.mu)
    return prob.solve("stv", case.lam, case.mu, case.rho, iters, ws=ws, cg=cg, objective=objective)


def check_J(P, case, iters, oinfo, objective, xr):
    J = np.array(P.trace(iters + 1))
    Jr = np.array(oinfo["J"])
    if objective == 2:
        assert np.max(np.abs(J - Jr) / Jr) < TOL
    else:   # the fused data term's bound (recon.h, opts.objective)
        Ny = case.sens.shape[1]
        bound = 2 * (1 + case.mu) * np.sqrt(Ny) * 2.0 ** -24 * np.linalg.norm(xr) ** 2 + TOL * Jr
        assert np.all(np.abs(J - Jr) <= bound)


@pytest.mark.parametrize("objective", [1, 2], ids=["fused_objective", "exact_objective"])
def test_tiny_workload_parity(objective):
    """64x64, 8 frames, 4 coils, R=4, lambda=0.01, mu=0.1, 50 iterations, w = 1, 5 CG steps."""
    case = make("tiny")
    P = plan_for(case, 1.0, 5, objective=objective)
    x, info = P.solve(gpu(case.kspace))
    xr, oinfo = oracle_solve(case, 1.0, 5, case.iters)
    assert info.iters == case.iters
    assert rel(host(x), xr) < TOL
    check_J(P, case, case.iters, oinfo, objective, xr)


@pytest.mark.parametrize("ws,cg", [(0.5, 3), (2.0, 8), (1.0, 1), (0.0, 4)])
def test_weights_and_cg_steps(ws, cg):
    case = make("tiny", Nx=40, Ny=48, Nt=6, Nc=3, seed=31)
    iters = 20
    P = plan_for(case, ws, cg, max_iters=iters, objective=2)
    x, _ = P.solve(gpu(case.kspace))
    xr, oinfo = oracle_solve(case, ws, cg, iters)
    assert rel(host(x), xr) < TOL
    check_J(P, case, iters, oinfo, 2, xr)


@pytest.mark.parametrize("shape", [dict(Nx=12, Ny=16, Nt=1, Nc=2, R=2),     # one frame: no temporal differences
                                   dict(Nx=1, Ny=32, Nt=4, Nc=2, R=2),      # one column: no horizontal differences
                                   dict(Nx=18, Ny=40, Nt=5, Nc=2, R=3),
                                   dict(Nx=20, Ny=97, Nt=3, Nc=2, R=4),     # odd Ny, ragged last block
                                   dict(Nx=33, Ny=31, Nt=7, Nc=3, R=4)],
                         ids=lambda s: "x".join(str(s[k]) for k in ("Nx", "Ny", "Nt", "Nc")))
def test_edge_shapes(shape):
    case = make("tiny", **shape)
    iters = 12
    P = plan_for(case, 0.8, 4, max_iters=iters, objective=2)
    x, _ = P.solve(gpu(case.kspace))
    xr, oinfo = oracle_solve(case, 0.8, 4, iters)
    assert rel(host(x), xr) < TOL
    check_J(P, case, iters, oinfo, 2, xr)


def test_many_blocks_per_slice():
    """128x128, 16 frames: 256 blocks per launch, so the CG sums cross many blocks."""
    case = make("tiny", Nx=128, Ny=128, Nt=16, Nc=4, R=4, seed=33)
    iters = 15
    P = plan_for(case, 1.0, 5, max_iters=iters, objective=1)
    x, _ = P.solve(gpu(case.kspace))
    xr, oinfo = oracle_solve(case, 1.0, 5, iters)
    assert rel(host(x), xr) < TOL
    check_J(P, case, iters, oinfo, 1, xr)


def test_repeated_solves_are_identical():
    """The CG sums add block partials in a fixed order: two solves agree bit for bit."""
    case = make("tiny", Nx=64, Ny=64, Nt=8, Nc=4, seed=34)
    P = plan_for(case, 1.0, 5, max_iters=10, objective=0)
    k = gpu(case.kspace)
    x0, _ = P.solve(k, info=False)
    x0 = x0.cpu().numpy()
    x1, _ = P.solve(k, info=False)
    np.testing.assert_array_equal(x1.cpu().numpy(), x0)


def test_batched_matches_oracle():
    from paper_1203_4587_gb300 import Batch
    shapes = [dict(Nx=24, Ny=64, Nt=6, Nc=3, seed=41), dict(Nx=40, Ny=40, Nt=8, Nc=4, seed=42),
              dict(Nx=16, Ny=96, Nt=5, Nc=2, seed=43)]
    weights = [1.0, 0.5, 1.5]
    cases = [make("tiny", **sh) for sh in shapes]
    iters, cg = 15, 4
    plans = [plan_for(c, w, cg, max_iters=iters) for c, w in zip(cases, weights)]
    b = Batch(plans)
    for _ in range(2):                       # direct run, then graph replay
        xs = b.solve([gpu(c.kspace) for c in cases])
        for c, w, x in zip(cases, weights, xs):
            xr, _ = oracle_solve(c, w, cg, iters, objective=False)
            assert rel(host(x), xr) < TOL


def test_batch_with_different_cg_steps_rejected():
    from paper_1203_4587_gb300 import Batch, ReconError
    case = make("tiny", Nx=16, Ny=32, Nt=4, Nc=2)
    plans = [plan_for(case, 1.0, 3, max_iters=4), plan_for(case, 1.0, 4, max_iters=4)]
    with pytest.raises(ReconError):
        Batch(plans)


def test_slab_plan_rejected():
    from paper_1203_4587_gb300 import Plan, ReconError
    case = make("tiny", Nx=16, Ny=32, Nt=4, Nc=2)
    with pytest.raises(ReconError):
        Plan(case.mask.astype(np.uint8), gpu(case.sens), case.lam, case.mu, prior="stv", slab=(0, 8), max_iters=2)


def test_autotuned_block_rows_keep_parity():
    """The autotuner picks the image columns per block of the spatio-temporal
    kernels (4, 8 or 16) by timing the whole step.  That moves the CG inner
    products' block partials, so the image may change in rounding only: it
    still matches the oracle, and repeated solves after tuning agree."""
    case = make("tiny", Nx=48, Ny=40, Nt=12, Nc=3, seed=35)
    P = plan_for(case, 1.0, 5, max_iters=15)
    t = P.autotune()
    assert t.temporal_tile_px in (4, 8, 16) and t.temporal_ms > 0
    k = gpu(case.kspace)
    x1, _ = P.solve(k)
    x2, _ = P.solve(k)
    np.testing.assert_array_equal(x1.cpu().numpy(), x2.cpu().numpy())
    xr, _ = oracle_solve(case, 1.0, 5, 15, objective=False)
    assert rel(host(x1), xr) < TOL
