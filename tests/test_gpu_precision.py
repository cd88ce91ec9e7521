"""GPU checks of the reduced-precision storage form (FP16 / BF16).

* k-space quantisation (recon_quantize_kspace) is byte work: bit-exact
  against the oracle's encoding (oracle.precision, pinned on the CPU).
* An FP32 plan fed 16-bit k-space computes exactly the FP32 method on the
  dequantised data: within TOL = 1e-5 of the oracle run on those values.
* 16-bit plans (inverses and hybrid coil data in 16 bits, FP32 arithmetic,
  FP64 reductions) are reported against the FP64 oracle on the original data,
  per frame.  The solution amplifies input errors ~100x (an FP32 experiment
  on the tiny workload: FP32 rounding of A and H'y, ~6e-8, gives ~5e-6), so
  16-bit rounding (unit roundoff 2^-11 FP16, 2^-8 BF16) is expected near
  1e-2 / 1e-1: the bounds are 3e-2 (FP16) and 2e-1 (BF16) overall, and twice
  that for any single frame.
* J(k) in that form uses the 16-bit hybrid data: with delta the rounding of
  the data (|delta| <= 2u ||y||, k-space and hybrid data each rounded once),
  |J - J(x)| <= 2 sqrt(fid) |delta| + |delta|^2 + 1e-5 J(x), where J(x) is
  the oracle's objective of the GPU's own iterate.
"""

import json
import os

import numpy as np
import pytest

import oracle
import synthdata
from oracle import precision as OP

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5
BOUND = {"fp16": 3e-2, "bf16": 2e-1}
UNIT = {"fp16": 2.0 ** -11, "bf16": 2.0 ** -8}


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


def plan_for(case, storage, **opts):
    from paper_1203_4587_gb300 import Plan
    opts.setdefault("max_iters", case.iters)
    return Plan(case.mask.astype(np.uint8), gpu(case.sens), case.lam, case.mu, prior="tv", rho=case.rho,
                storage=storage, **opts)


def pair_bits(q):
    """(re_bits, im_bits) uint16 arrays of a QuantizedKspace's data."""
    u = q.data.cpu().numpy().view(np.uint16).reshape(q.data.shape + (2,))
    return u[..., 0], u[..., 1]


def per_frame(x, xr):
    return [rel(x[t], xr[t]) for t in range(x.shape[0])]


@pytest.mark.parametrize("storage", ["fp16", "bf16"])
def test_quantize_kspace_bit_exact(storage):
    from paper_1203_4587_gb300.binding import quantize_kspace
    case = make("tiny", Nx=40, Ny=48, Nt=5, Nc=3)
    k = case.kspace.copy()
    k[2] *= 1e-4            # frames of very different scale
    k[4] = 0.0              # an empty frame: scale 1
    q = quantize_kspace(gpu(k), storage)
    re, im = pair_bits(q)
    ore, oim, os_ = OP.quantize_frames(k, storage)
    np.testing.assert_array_equal(q.frame_scale.cpu().numpy().astype(np.float64), os_)
    np.testing.assert_array_equal(re, ore)
    np.testing.assert_array_equal(im, oim)


@pytest.mark.parametrize("storage", ["fp16", "bf16"])
def test_fp32_plan_with_16bit_kspace_is_exact_on_dequantised_data(storage):
    from paper_1203_4587_gb300.binding import quantize_kspace
    case = make("tiny")
    P = plan_for(case, "fp32")
    q = quantize_kspace(gpu(case.kspace), storage)
    x, info = P.solve_quantized(q)
    ore, oim, os_ = OP.quantize_frames(case.kspace, storage)
    kd = OP.dequantize_frames(ore, oim, os_, storage)
    prob = oracle.Problem(kd, case.sens, case.mask, case.mu)
    xr, oinfo = prob.solve("tv", case.lam, case.mu, case.rho, case.iters)
    assert rel(host(x), xr) < TOL
    assert abs(info.J - oinfo["J"][-1]) / oinfo["J"][-1] < TOL


@pytest.mark.parametrize("storage", ["fp16", "bf16"])
def test_16bit_plan_error_per_frame_against_fp64(storage):
    """Tiny workload, 16-bit k-space and 16-bit plan storage."""
    from paper_1203_4587_gb300.binding import quantize_kspace
    case = make("tiny")
    P = plan_for(case, storage)
    x, info = P.solve_quantized(quantize_kspace(gpu(case.kspace), storage))
    x = host(x)
    prob = oracle.Problem(case.kspace, case.sens, case.mask, case.mu)
    xr, _ = prob.solve("tv", case.lam, case.mu, case.rho, case.iters, objective=False)
    e = rel(x, xr)
    frames = per_frame(x, xr)
    print(f"\n{storage} tiny: overall {e:.3e}, per frame " + " ".join(f"{v:.2e}" for v in frames))
    assert e < BOUND[storage] and max(frames) < 2 * BOUND[storage]
    # J(K) of the 16-bit form against the oracle's J of the same iterate
    fid = float(prob.fid(x))
    J_of_x = oracle.objective_tv(x, case.lam, prob.fid)
    ynorm = float(np.linalg.norm(case.kspace * case.mask[:, None, :, None]))
    d = 2 * UNIT[storage] * ynorm
    assert abs(info.J - J_of_x) <= 2 * np.sqrt(fid) * d + d * d + 1e-5 * J_of_x


def test_precision_workload_per_frame_errors():
    """384x384, 48 frames, 16 coils, R=6, TV, 100 iterations: FP32, FP16 and
    BF16 storage on 16-bit k-space (FP32 k-space for the FP32 run), compared
    with the FP64 oracle on a seeded subset of 3 columns (columns are
    independent), per frame.  Writes the table to $PRECISION_REPORT if set."""
    from paper_1203_4587_gb300.binding import quantize_kspace
    case = make("precision")
    cols = np.sort(np.random.default_rng(5).choice(case.x_true.shape[2], size=3, replace=False))
    prob = oracle.Problem(case.kspace, case.sens, case.mask, case.mu, cols)
    xr, _ = prob.solve("tv", case.lam, case.mu, case.rho, case.iters, objective=False)
    report = {"workload": "precision 384x384x48x16 R=6 TV lambda=0.005 mu=0.1 100 iterations",
              "columns": cols.tolist()}
    kg = gpu(case.kspace)
    for storage in ("fp32", "fp16", "bf16"):
        P = plan_for(case, storage, objective=0)
        if storage == "fp32":
            x, _ = P.solve(kg, info=False)
        else:
            x, _ = P.solve_quantized(quantize_kspace(kg, storage), info=False)
        xs = host(x)[:, :, cols]
        P.close()
        frames = per_frame(xs, xr)
        report[storage] = {"overall": rel(xs, xr), "per_frame": frames}
        print(f"\n{storage}: overall {report[storage]['overall']:.3e}, max frame {max(frames):.3e}")
        if storage == "fp32":
            assert report[storage]["overall"] < TOL
        else:
            assert report[storage]["overall"] < BOUND[storage] and max(frames) < 2 * BOUND[storage]
    path = os.environ.get("PRECISION_REPORT")
    if path:
        with open(path, "w") as f:
            json.dump(report, f, indent=1)
