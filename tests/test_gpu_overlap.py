"""Programmatic dependent launches between the temporal-TV and inverse kernels
(opts.overlap) and the whole-chunk temporal kernel, against the plain stream
order and the FP64 oracle.

With overlap on, each kernel of the one-launch-per-step TV solve may start
while the previous one finishes and waits in-device before it touches the
iteration's state; the arithmetic of every pixel and column is unchanged, so
the images must be bit-identical to overlap off (and J(k), an FP64 sum of
atomic adds in any order, equal to 1e-12).  The shapes
cover the whole-chunk temporal kernel (Nt a multiple of 8, Nx*Ny a multiple
of 16), the general one, the fused objective, the explicit one (16-bit
storage) and a batch (run directly, then as a captured graph).
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


def make(**over):
    c = synthdata.make_case("tiny", **over)
    c.kspace = c.kspace.astype(np.complex64).astype(np.complex128)
    c.sens = c.sens.astype(np.complex64).astype(np.complex128)
    return c


def gpu(x):
    return torch.from_numpy(np.asarray(x, dtype=np.complex64)).cuda()


def plan(c, prior="tv", **opts):
    from paper_1203_4587_gb300 import Plan
    opts.setdefault("max_iters", c.iters)
    return Plan(c.mask.astype(np.uint8), gpu(c.sens), c.lam, c.mu, prior=prior, rho=c.rho, **opts)


SHAPES = [
    dict(Nx=64, Ny=64, Nt=32, Nc=4, R=4),      # whole chunks, 4 frames a segment (the cardiac shape's Nt)
    dict(Nx=48, Ny=40, Nt=8, Nc=3, R=3),       # whole chunks, 1 frame a segment, ragged Ny
    dict(Nx=20, Ny=36, Nt=48, Nc=2, R=4),      # whole chunks, 6 frames a segment
    dict(Nx=45, Ny=40, Nt=3, Nc=3, R=3),       # general kernel: Nt not a multiple of 8
    dict(Nx=9, Ny=33, Nt=16, Nc=2, R=2),       # general kernel: Nx*Ny not a multiple of 16
]


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "x".join(str(s[k]) for k in ("Nx", "Ny", "Nt", "Nc")))
@pytest.mark.parametrize("storage", ["fp32", "fp16"])
def test_overlap_bit_identical_and_matches_oracle(shape, storage):
    c = make(iters=20, **shape)
    P1 = plan(c, overlap=1, storage=storage)
    P0 = plan(c, overlap=0, storage=storage)
    k = gpu(c.kspace)
    x1, i1 = P1.solve(k)
    x0, i0 = P0.solve(k)
    a1, a0 = x1.cpu().numpy(), x0.cpu().numpy()
    assert np.array_equal(a1, a0)
    # J(k) and the residuals are FP64 sums whose atomic adds land in any order
    n = c.iters + 1
    J1, J0 = np.array(P1.trace(n)), np.array(P0.trace(n))
    assert np.all(np.abs(J1 - J0) <= 1e-12 * np.abs(J0))
    assert abs(i1.primal_res - i0.primal_res) <= 1e-12 * i0.primal_res
    assert abs(i1.dual_res - i0.dual_res) <= 1e-12 * i0.dual_res
    if storage == "fp32":
        xr, oinfo = oracle.Problem(c.kspace, c.sens, c.mask, c.mu).solve("tv", c.lam, c.mu, c.rho, c.iters)
        assert rel(a1.astype(np.complex128), xr) < TOL
        Jr = np.array(oinfo["J"])
        Ny = shape["Ny"]
        bound = 2 * (1 + c.mu) * np.sqrt(Ny) * 2.0 ** -24 * np.linalg.norm(xr) ** 2 + TOL * Jr
        assert np.all(np.abs(np.array(P1.trace(n)) - Jr) <= bound)
    # a second solve on the same plan repeats the first exactly
    assert np.array_equal(P1.solve(k)[0].cpu().numpy(), a1)
    P1.close()
    P0.close()


@pytest.mark.parametrize("prior", ["dft", "haar", "stv"])
def test_overlap_other_priors_bit_identical(prior):
    """Algorithm 1 (temporal DFT, Haar frame): the same launches with and
    without the programmatic dependency give the same image, which matches the
    oracle.  The spatio-temporal prior ignores the option (plain stream order)
    and must give the same image either way too."""
    c = make(Nx=40, Ny=48, Nt=12, Nc=3, R=3, iters=15)
    P1 = plan(c, prior=prior, overlap=1, frame_levels=2, spatial_weight=1.0, cg_steps=5)
    P0 = plan(c, prior=prior, overlap=0, frame_levels=2, spatial_weight=1.0, cg_steps=5)
    k = gpu(c.kspace)
    a1 = P1.solve(k)[0].cpu().numpy()
    a0 = P0.solve(k)[0].cpu().numpy()
    assert np.array_equal(a1, a0)
    prob = oracle.Problem(c.kspace, c.sens, c.mask, c.mu)
    if prior == "dft":
        xr, _ = prob.solve("dft", c.lam, c.mu, c.rho, c.iters)
    elif prior == "haar":
        xr, _ = prob.solve("haar", c.lam, c.mu, c.rho, c.iters, levels=2)
    else:
        xr, _ = prob.solve("stv", c.lam, c.mu, c.rho, c.iters, ws=1.0, cg=5)
    assert rel(a1.astype(np.complex128), xr) < TOL
    P1.close()
    P0.close()


def test_overlap_batch_direct_and_graph_replay():
    """Batches run in plain stream order whatever the plans' option: the same
    images either way, on the direct run and on the graph replay."""
    from paper_1203_4587_gb300 import Batch
    shapes = [dict(Nx=32, Ny=64, Nt=16, Nc=3, R=4, seed=31), dict(Nx=40, Ny=48, Nt=16, Nc=2, R=3, seed=32),
              dict(Nx=16, Ny=32, Nt=16, Nc=2, R=2, seed=33)]
    cases = [make(iters=12, **sh) for sh in shapes]
    ks = [gpu(c.kspace) for c in cases]
    outs = {}
    for ov in (0, 1):
        plans = [plan(c, overlap=ov) for c in cases]
        b = Batch(plans)
        runs = []
        for _ in range(2):      # the first call runs the launches, the second replays the captured graph
            runs.append([x.cpu().numpy() for x in b.solve(ks)])
        for a, g in zip(*runs):
            assert np.array_equal(a, g)
        outs[ov] = runs[0]
        b.close()
        for p in plans:
            p.close()
    for a, z in zip(outs[1], outs[0]):
        assert np.array_equal(a, z)
    for c, a in zip(cases, outs[1]):
        xr, _ = oracle.Problem(c.kspace, c.sens, c.mask, c.mu).solve("tv", c.lam, c.mu, c.rho, c.iters)
        assert rel(a.astype(np.complex128), xr) < TOL


def test_profile_toggle_keeps_results():
    """recon_plan_set_profile: events on (overlap then unused) and off give the same image."""
    c = make(Nx=32, Ny=32, Nt=8, Nc=2, R=2, iters=6)
    P = plan(c)
    k = gpu(c.kspace)
    x_off = P.solve(k)[0].cpu().numpy()
    P.set_profile(True)
    x_on = P.solve(k)[0].cpu().numpy()
    pr = P.profile()
    assert pr.inverse_launches == 6 and pr.temporal_launches >= 6 and pr.inverse_ms > 0
    P.set_profile(False)
    assert np.array_equal(P.solve(k)[0].cpu().numpy(), x_off)
    assert np.array_equal(x_on, x_off)
    P.close()
