"""GPU parity of the batched form at its full size: 64 slices of uneven shape.

The batched workload: Nx, Ny in {128, 160, 192, 256}, Nt in {16, 24, 32, 40},
Nc in {8, 12, 16}, R in {4, 6, 8}, temporal TV, lambda = 0.005, mu = 0.1,
80 iterations, every slice its own seed.  All 64 slices are solved in one
batch, in the launch configuration the benchmark times (autotuned shapes, one
launch per step, then a replay of the captured CUDA graph).  Columns and
slices are independent (Section IV-C), so the FP64 oracle restricted to a few
image columns of a slice computes exactly those columns; it is run on:

* a set of slices that together cover every Ny and every Nt of the workload,
  two seeded image columns each;
* the image columns of the (slice, column) work items that the longest-
  processing-time assignment gives to the last CTA of the inverse kernel
  (the assignment is restated here only to choose columns: a slip in it
  would just move the check to other columns);
* the smallest slice on every column, with its J(k) trace.

Bar: relative L2 1e-5 per checked slice (FP32 path against FP64), on the
first direct run and on the graph replay; J(k) within 1e-5 relative plus the
fused objective's rounding bound.
"""

import concurrent.futures as cf
import heapq
import os

import numpy as np
import pytest

import oracle
import synthdata

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5
NSLICES = 64


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _case(sh):
    c = synthdata.make_case("batched", **sh)
    c.kspace = c.kspace.astype(np.complex64).astype(np.complex128)
    c.sens = c.sens.astype(np.complex64).astype(np.complex128)
    return c


def _last_cta_items(shapes, grid):
    """(slice, column) items of the last CTA under longest-processing-time-
    first: every column (i, t) of slice q costs its packed stream (bytes) and
    goes to the least-loaded CTA (ties to the lower index)."""
    def nb(ny):
        return (ny + 31) // 32
    cols = []
    for q, sh in enumerate(shapes):
        n = nb(sh["Ny"])
        elems = n * (n - 1) // 2 * 1024 + n * 640
        cost = elems * 8 + 4096
        cols += [(cost, q, c) for c in range(sh["Nx"] * sh["Nt"])]
    cols.sort(key=lambda x: -x[0])
    heap = [(0, b) for b in range(grid)]
    mine = []
    for cost, q, c in cols:
        load, b = heapq.heappop(heap)
        if b == grid - 1:
            mine.append((q, c))
        heapq.heappush(heap, (load + cost, b))
    return mine


@pytest.fixture(scope="module")
def batched_run():
    from paper_1203_4587_gb300 import Batch, Plan
    shapes = synthdata.batched_shapes(NSLICES, 64)
    with cf.ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 4)) as ex:
        cases = list(ex.map(_case, shapes))
    plans = [Plan(c.mask.astype(np.uint8), torch.from_numpy(c.sens.astype(np.complex64)).cuda(), c.lam, c.mu,
                  prior="tv", rho=c.rho, max_iters=c.iters) for c in cases]
    ks = [torch.from_numpy(c.kspace.astype(np.complex64)).cuda() for c in cases]
    batch = Batch(plans)
    batch.autotune()
    runs = []
    for call in range(2):                      # direct run, then graph replay
        outs = batch.solve(ks)
        infos = batch.info()
        torch.cuda.synchronize()
        runs.append(([o.cpu().numpy().astype(np.complex128) for o in outs],
                     [(i.iters, i.J) for i in infos],
                     [np.array(p.trace(c.iters + 1)) for p, c in zip(plans, cases)]))
    grid = torch.cuda.get_device_properties(0).multi_processor_count
    batch.close()
    for p in plans:
        p.close()
    del ks
    torch.cuda.empty_cache()
    return shapes, cases, runs, grid


def _checked_slices(shapes):
    """A few slices that together cover every Ny and every Nt value."""
    need_ny = {128, 160, 192, 256}
    need_nt = {16, 24, 32, 40}
    pick = []
    for q, sh in enumerate(shapes):
        if sh["Ny"] in need_ny or sh["Nt"] in need_nt:
            pick.append(q)
            need_ny.discard(sh["Ny"])
            need_nt.discard(sh["Nt"])
    assert not need_ny and not need_nt, (need_ny, need_nt)
    return pick


def _oracle_cols(c, cols):
    prob = oracle.Problem(c.kspace, c.sens, c.mask, c.mu, np.asarray(cols))
    xr, info = prob.solve("tv", c.lam, c.mu, c.rho, c.iters, objective=False)
    return xr


def test_batched_workload_slices_cover_every_size(batched_run):
    shapes, cases, runs, _ = batched_run
    for x, its, _ in runs:
        assert all(n == 80 and np.isfinite(J) for n, J in its)
    rng = np.random.default_rng(5)
    for q in _checked_slices(shapes):
        c = cases[q]
        cols = np.sort(rng.choice(c.x_true.shape[2], size=2, replace=False))
        xr = _oracle_cols(c, cols)
        for call, (xs, _, _) in enumerate(runs):
            e = rel(xs[q][:, :, cols], xr)
            assert e < TOL, (q, shapes[q], call, e)


def test_batched_workload_last_cta_columns(batched_run):
    shapes, cases, runs, grid = batched_run
    items = _last_cta_items(shapes, grid)
    assert items
    # two items of the last CTA from different slices: the columns i of col = t * Nx + i
    chosen = {}
    for q, col in items[::-1]:
        if q not in chosen:
            chosen[q] = col % shapes[q]["Nx"]
        if len(chosen) == 2:
            break
    for q, i in chosen.items():
        xr = _oracle_cols(cases[q], [i])
        for call, (xs, _, _) in enumerate(runs):
            e = rel(xs[q][:, :, [i]], xr)
            assert e < TOL, (q, i, call, e)


def test_batched_workload_smallest_slice_whole_with_objective(batched_run):
    shapes, cases, runs, _ = batched_run
    q = min(range(len(shapes)), key=lambda k: shapes[k]["Nx"] * shapes[k]["Ny"] ** 2 * shapes[k]["Nt"])
    c = cases[q]
    prob = oracle.Problem(c.kspace, c.sens, c.mask, c.mu)
    xr, oinfo = prob.solve("tv", c.lam, c.mu, c.rho, c.iters)
    Jr = np.array(oinfo["J"])
    Ny = c.x_true.shape[1]
    for call, (xs, its, traces) in enumerate(runs):
        assert rel(xs[q], xr) < TOL, (call, q)
        # fused objective: the identity's error on top of the 1e-5 relative bar
        bound = 2 * (1 + c.mu) * np.sqrt(Ny) * 2.0 ** -24 * np.linalg.norm(xr) ** 2 + TOL * Jr
        assert np.all(np.abs(traces[q] - Jr) <= bound), call
