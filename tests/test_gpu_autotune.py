"""GPU checks of the launch-shape autotuner (recon_autotune, recon_batch_autotune).

The tuned shapes change how work is split into blocks, never the arithmetic
of a pixel or a column: the temporal kernels compute each pixel's t-series
alone, the inverse kernel each column alone, the prologue each row / column
alone with the coil sum in a fixed order.  So images after tuning are
bit-identical to images before it, and J(k) differs only by the order of its
FP64 sums.
"""

import numpy as np
import pytest

import synthdata

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def gpu(x):
    return torch.from_numpy(np.asarray(x, dtype=np.complex64)).cuda()


def make(name, **over):
    return synthdata.make_case(name, **over)


@pytest.mark.parametrize("prior,storage,objective", [("tv", "fp32", 1), ("dft", "fp32", 1), ("tv", "fp16", 1),
                                                     ("tv", "fp32", 2)])
def test_autotune_leaves_results_unchanged(prior, storage, objective):
    from paper_1203_4587_gb300 import Plan
    case = make("tiny", Nx=48, Ny=64, Nt=10, Nc=5, seed=21)
    P = Plan(case.mask.astype(np.uint8), gpu(case.sens), case.lam, case.mu, prior=prior, rho=case.rho,
             max_iters=12, storage=storage, objective=objective)
    k = gpu(case.kspace)
    x0, i0 = P.solve(k)
    x0 = x0.cpu().numpy()
    t = P.autotune()
    assert t.temporal_tile_px in ((16,) if prior == "tv" else (16, 32, 64, 128))
    quantum = 8 if storage == "fp32" else 12          # the consumer warp count of the inverse kernel
    assert t.col_stages % quantum == 0 and t.col_stages >= quantum
    assert 1 <= t.rows_per_block <= 8 and 1 <= t.combine_coils <= 8
    exact = storage != "fp32" or objective == 2
    assert (t.objective_coils >= 1) == exact
    assert t.col_ms > 0 and t.temporal_ms > 0
    x1, i1 = P.solve(k)
    np.testing.assert_array_equal(x1.cpu().numpy(), x0)
    assert abs(i1.J - i0.J) <= 1e-12 * abs(i0.J)


def test_autotune_cache_by_shape():
    from paper_1203_4587_gb300 import Plan
    case = make("tiny", Nx=40, Ny=32, Nt=6, Nc=3, seed=22)
    plans = [Plan(case.mask.astype(np.uint8), gpu(case.sens), case.lam, case.mu, max_iters=5) for _ in range(2)]
    t0 = plans[0].autotune()
    t1 = plans[1].autotune()
    assert t1.from_cache == 1
    for f in ("temporal_tile_px", "col_stages", "rows_per_block", "combine_coils", "objective_coils"):
        assert getattr(t0, f) == getattr(t1, f)
    x0, _ = plans[0].solve(gpu(case.kspace))
    x1, _ = plans[1].solve(gpu(case.kspace))
    np.testing.assert_array_equal(x0.cpu().numpy(), x1.cpu().numpy())


def test_batch_autotune_leaves_results_unchanged():
    from paper_1203_4587_gb300 import Batch, Plan
    shapes = [dict(Nx=24, Ny=64, Nt=6, Nc=3, seed=31), dict(Nx=40, Ny=40, Nt=9, Nc=4, seed=32),
              dict(Nx=16, Ny=96, Nt=5, Nc=2, seed=33)]
    cases = [make("tiny", **sh) for sh in shapes]
    plans = [Plan(c.mask.astype(np.uint8), gpu(c.sens), c.lam, c.mu, max_iters=10) for c in cases]
    b = Batch(plans)
    ks = [gpu(c.kspace) for c in cases]
    x0 = [x.cpu().numpy() for x in b.solve(ks)]
    t = b.autotune()
    assert t.temporal_tile_px == 16 and t.col_stages % 8 == 0
    # each slice's prologue shapes, reported for the largest slice
    assert 1 <= t.rows_per_block <= 8 and 1 <= t.combine_coils <= 8 and t.rows_ms > 0 and t.combine_ms > 0
    x1 = [x.cpu().numpy() for x in b.solve(ks)]      # re-captured graph
    x2 = [x.cpu().numpy() for x in b.solve(ks)]      # replay
    for a, c, d in zip(x0, x1, x2):
        np.testing.assert_array_equal(a, c)
        np.testing.assert_array_equal(a, d)
