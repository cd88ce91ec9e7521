"""GPU parity at the plan's size limits and in degenerate cases, against the
FP64 oracle.

The plan accepts Nx <= 1024, Nt <= 128, Nc <= 64 with (Nc + 1) Ny <= 12800,
and Ny <= 768 with FP32 storage, 640 with 16-bit storage (recon_plan_create).  Each limit is
reached with the other dimensions small, so the oracle (dense per-column
inverses) stays fast.  Degenerate cases: a frame without a sampled row
(its Gram blocks are zero and the inverse is I / mu), and a fully sampled
frame next to an empty one.  Bar: relative L2 1e-5 for the image and 1e-5
relative for J(k) with the exact objective.
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


def solve_both(c, prior, iters):
    from paper_1203_4587_gb300 import Plan
    P = Plan(c.mask.astype(np.uint8), gpu(c.sens), c.lam, c.mu, prior=prior, rho=c.rho, max_iters=iters,
             objective=2)
    x, info = P.solve(gpu(c.kspace))
    J = np.array(P.trace(iters + 1))
    P.close()
    xr, oinfo = oracle.Problem(c.kspace, c.sens, c.mask, c.mu).solve(prior, c.lam, c.mu, c.rho, iters)
    return x.cpu().numpy().astype(np.complex128), J, xr, np.array(oinfo["J"]), info


LIMITS = [
    dict(Nx=2, Ny=768, Nt=2, Nc=2, R=4),       # the largest Ny with FP32 storage: 24 blocks of 32
    dict(Nx=1024, Ny=16, Nt=2, Nc=2, R=2),     # the largest Nx
    dict(Nx=4, Ny=16, Nt=128, Nc=2, R=2),      # the largest Nt: 16 frames a Thomas segment
    dict(Nx=4, Ny=128, Nt=2, Nc=64, R=4),      # the most coils at this Ny (65 x 128 x 16 B = 130 KB)
]


@pytest.mark.parametrize("shape", LIMITS, ids=lambda s: "x".join(str(s[k]) for k in ("Nx", "Ny", "Nt", "Nc")))
@pytest.mark.parametrize("prior", ["tv", "dft"])
def test_size_limits_match_oracle(shape, prior):
    c = make(iters=6, **shape)
    x, J, xr, Jr, _ = solve_both(c, prior, 6)
    assert rel(x, xr) < TOL
    assert np.max(np.abs(J - Jr) / Jr) < TOL


def test_beyond_the_limits_is_rejected():
    from paper_1203_4587_gb300 import Plan, ReconError
    for sh, storage in ((dict(Nx=2, Ny=769, Nt=1, Nc=1), "fp32"), (dict(Nx=2, Ny=641, Nt=1, Nc=1), "fp16"),
                        (dict(Nx=1025, Ny=16, Nt=1, Nc=1), "fp32"), (dict(Nx=2, Ny=16, Nt=129, Nc=1), "fp32"),
                        (dict(Nx=2, Ny=16, Nt=1, Nc=65), "fp32")):
        mask = np.ones((sh["Nt"], sh["Ny"]), dtype=np.uint8)
        sens = torch.ones((sh["Nc"], sh["Ny"], sh["Nx"]), dtype=torch.complex64, device="cuda")
        with pytest.raises(ReconError) as ei:
            Plan(mask, sens, 0.01, 0.1, max_iters=2, storage=storage)
        assert ei.value.status == 7, sh      # RECON_ERR_UNSUPPORTED
    # a mask that samples nothing: no data to reconstruct from
    sens = torch.ones((2, 16, 4), dtype=torch.complex64, device="cuda")
    with pytest.raises(ReconError):
        Plan(np.zeros((3, 16), dtype=np.uint8), sens, 0.01, 0.1, max_iters=2)


def test_largest_ny_with_16bit_storage():
    """Ny = 640, the 16-bit limit: the 16-bit solve stays within its stated
    error of the FP64 oracle (the FP16 inverses' rounding, as in the precision
    tests), and its J(k) within the bound derived from the 16-bit data."""
    from paper_1203_4587_gb300 import Plan
    c = make(Nx=2, Ny=640, Nt=2, Nc=2, R=4, iters=6)
    P = Plan(c.mask.astype(np.uint8), gpu(c.sens), c.lam, c.mu, prior="tv", rho=c.rho, max_iters=6, storage="fp16")
    x, info = P.solve(gpu(c.kspace))
    xr, _ = oracle.Problem(c.kspace, c.sens, c.mask, c.mu).solve("tv", c.lam, c.mu, c.rho, 6)
    assert rel(x.cpu().numpy().astype(np.complex128), xr) < 3e-2
    assert np.isfinite(info.J)
    P.close()


@pytest.mark.parametrize("prior", ["tv", "dft", "stv"])
def test_frame_without_samples(prior):
    """Frame 1 has no sampled row (zero Gram blocks, A = I / mu there) and frame
    2 is fully sampled; the others keep the variable-density pattern."""
    rng = np.random.default_rng(5)
    mask = synthdata.make_mask(32, 5, 4, rng)
    mask[1] = False
    mask[2] = True
    c = make(Nx=24, Ny=32, Nt=5, Nc=3, mask=mask, iters=8)
    assert not c.mask[1].any() and c.mask[2].all()
    x, J, xr, Jr, info = solve_both(c, prior, 8)
    assert rel(x, xr) < TOL
    assert np.max(np.abs(J - Jr) / Jr) < TOL
    assert np.isfinite(info.primal_res) and np.isfinite(info.dual_res)
