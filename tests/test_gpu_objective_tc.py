"""The explicit data term ||y - H x||^2 on the tensor cores (objective_tc.cu)
against the FP64 oracle.

With `objective=2` and an even Ny the plan forms J(k) with the tcgen05 kernel:
the sampled DFT rows of each frame times s_c . x, split into FP16 pairs
(three products).  The shapes reach the kernel's tiling edges: several
column tiles of 256 (i, c) with a ragged last one, an odd coil count (column
pairs that straddle two image columns), a single coil, several tiles of 64
sampled rows with a ragged last one, and Ny that is not a multiple of the
16-value K chunk.  Bar: relative L2 1e-5 for the image and 1e-5 relative
for every J(k), as for the FFT form of the explicit objective.
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


SHAPES = [
    dict(Nx=40, Ny=48, Nt=3, Nc=7, R=2),      # 280 columns: two tiles, the second ragged; Nc odd
    dict(Nx=100, Ny=64, Nt=2, Nc=1, R=2),     # one coil: 100 image columns in a tile
    dict(Nx=12, Ny=144, Nt=2, Nc=3, R=1),     # 144 sampled rows: tiles of 64, 64, 16; 9 K chunks
    dict(Nx=30, Ny=10, Nt=4, Nc=2, R=2),      # Ny below one K chunk
    dict(Nx=33, Ny=40, Nt=5, Nc=8, R=3),      # 264 columns; Ny = 2.5 K chunks
]


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "x".join(str(s[k]) for k in ("Nx", "Ny", "Nt", "Nc")))
@pytest.mark.parametrize("prior", ["tv", "dft"])
def test_tensor_core_objective_matches_oracle(shape, prior):
    from paper_1203_4587_gb300 import Plan
    iters = 6
    c = synthdata.make_case("tiny", iters=iters, **shape)
    c.kspace = c.kspace.astype(np.complex64).astype(np.complex128)
    c.sens = c.sens.astype(np.complex64).astype(np.complex128)
    sens = torch.from_numpy(c.sens.astype(np.complex64)).cuda()
    k = torch.from_numpy(c.kspace.astype(np.complex64)).cuda()
    P = Plan(c.mask.astype(np.uint8), sens, c.lam, c.mu, prior=prior, rho=c.rho, max_iters=iters, objective=2)
    x, _ = P.solve(k)
    J = np.array(P.trace(iters + 1))
    P.close()
    xr, oinfo = oracle.Problem(c.kspace, c.sens, c.mask, c.mu).solve(prior, c.lam, c.mu, c.rho, iters)
    Jr = np.array(oinfo["J"])
    assert rel(x.cpu().numpy().astype(np.complex128), xr) < TOL
    assert np.max(np.abs(J - Jr) / Jr) < TOL


def test_dispatch_tensor_cores_for_even_ny_only():
    """16-bit plans form J(k) on the tensor cores for even Ny: two launches an
    iteration (the scales' max |x| pass and k_objective_tc) where the FFT form
    for odd Ny takes one, everything else being equal; the autotuner reports
    the tensor-core form's one shape (objective_coils = 1)."""
    from paper_1203_4587_gb300 import Plan
    from paper_1203_4587_gb300.binding import kernel_launches

    def per_iteration(Ny):
        c = synthdata.make_case("tiny", Nx=24, Ny=Ny, Nt=4, Nc=8, R=3, iters=4)
        sens = torch.from_numpy(c.sens.astype(np.complex64)).cuda()
        k = torch.from_numpy(c.kspace.astype(np.complex64)).cuda()
        n = []
        for K in (2, 4):
            P = Plan(c.mask.astype(np.uint8), sens, c.lam, c.mu, prior="tv", rho=c.rho, max_iters=K, storage="fp16")
            P.solve(k)
            torch.cuda.synchronize()
            n0 = kernel_launches()
            P.solve(k)
            torch.cuda.synchronize()
            n.append(kernel_launches() - n0)
            if K == 4:
                t = P.autotune()
                assert t.objective_ms > 0
                coils = t.objective_coils
            P.close()
        return (n[1] - n[0]) / 2, coils

    even, coils_even = per_iteration(40)
    odd, _ = per_iteration(33)
    assert even == odd + 1
    assert coils_even == 1
