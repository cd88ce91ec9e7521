"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances: FP32 results must be within relative L2 1e-5 of the oracle (image
after K iterations, and every J(k)); single operator applications (H, H',
the packed inverses) within 1e-5 as well.  Inputs are the seeded synthetic
workloads of ``synthdata``; the oracle sees the same complex64-rounded data.
"""

import numpy as np
import pytest

import oracle
import synthdata

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5


def rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def c64(x):
    return np.asarray(x, dtype=np.complex64)


def as64(x):
    return np.asarray(x, dtype=np.complex64).astype(np.complex128)


def gpu(x):
    return torch.from_numpy(c64(x)).cuda()


def host(t):
    return t.detach().cpu().numpy().astype(np.complex128)


def make(name="tiny", **over):
    case = synthdata.make_case(name, **over)
    # both sides see the complex64-rounded inputs
    case.kspace = as64(case.kspace)
    case.sens = as64(case.sens)
    return case


def plan_for(case, prior="tv", **opts):
    from paper_1203_4587_gb300 import Plan
    opts.setdefault("max_iters", case.iters)
    return Plan(case.mask.astype(np.uint8), gpu(case.sens), case.lam, case.mu, prior=prior, rho=case.rho, **opts)


SHAPES = [
    dict(Nx=64, Ny=64, Nt=8, Nc=4, R=4),      # tiny workload
    dict(Nx=45, Ny=40, Nt=3, Nc=3, R=3),      # radix 3/5, Ny not a multiple of 32
    dict(Nx=20, Ny=97, Nt=2, Nc=2, R=4),      # prime length: direct DFT stage; odd block count
    dict(Nx=33, Ny=96, Nt=5, Nc=1, R=2),      # single coil, 3 blocks (odd), radix 3 in Ny
]


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "x".join(str(s[k]) for k in ("Nx", "Ny", "Nt", "Nc")))
def test_adjoint_and_forward_operators(shape):
    case = make("tiny", **shape)
    P = plan_for(case, max_iters=1)
    b = host(P.adjoint(gpu(case.kspace)))
    ref = oracle.adjoint_op(case.kspace, case.sens, case.mask)
    assert rel(b, ref) < TOL
    rng = np.random.default_rng(0)
    x = as64(rng.standard_normal(case.x_true.shape) + 1j * rng.standard_normal(case.x_true.shape))
    y = host(P.forward(gpu(x)))
    yref = oracle.forward_op(x, case.sens, case.mask)
    assert rel(y, yref) < TOL
    # unsampled rows are exactly zero
    assert np.all(y[~np.broadcast_to(case.mask[:, None, :, None], y.shape)] == 0)


def test_frame_without_samples_and_full_frame():
    case = make("tiny", Nx=16, Ny=32, Nt=3, Nc=2)
    mask = case.mask.copy()
    mask[1] = False
    mask[2] = True
    case.mask = mask
    case.kspace = case.kspace * mask[:, None, :, None]
    P = plan_for(case, max_iters=1)
    assert rel(host(P.adjoint(gpu(case.kspace))), oracle.adjoint_op(case.kspace, case.sens, mask)) < TOL
    A1 = host(P.export_inverse(3, 1))
    np.testing.assert_allclose(A1, np.eye(32) / case.mu, atol=1e-6 / case.mu)


@pytest.mark.parametrize("shape", SHAPES[:3], ids=["tiny", "45x40", "20x97"])
def test_packed_inverse_blocks(shape):
    case = make("tiny", **shape)
    P = plan_for(case, max_iters=1)
    Nt, Ny, Nx = case.x_true.shape
    rng = np.random.default_rng(1)
    for _ in range(4):
        i, t = int(rng.integers(Nx)), int(rng.integers(Nt))
        G = oracle.gram_blocks(case.sens, case.mask, [i])[t, 0]
        Aref = oracle.inverse_blocks(G, case.mu)
        A = host(P.export_inverse(i, t))
        assert rel(A, Aref) < 2e-7          # FP64 factorisation, one FP32 rounding
        res = A @ (case.mu * np.eye(Ny) + G) - np.eye(Ny)
        assert np.abs(res).max() < 1e-5


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "x".join(str(s[k]) for k in ("Nx", "Ny", "Nt", "Nc")))
def test_inverse_rounded_once(shape):
    """The factorisation (double-float, about 48 bits) is rounded once: every
    element is within half an FP32 ulp of the FP64 oracle's value plus
    2^-36 max|A|, and the larger elements equal its FP32 rounding."""
    case = make("tiny", **shape)
    P = plan_for(case, max_iters=1)
    Nt, Ny, Nx = case.x_true.shape
    mu32 = float(np.float32(case.mu))   # the plan holds mu as an FP32 value (recon_plan_create takes float)
    rng = np.random.default_rng(3)
    for _ in range(3):
        i, t = int(rng.integers(Nx)), int(rng.integers(Nt))
        Aref = oracle.inverse_blocks(oracle.gram_blocks(case.sens, case.mask, [i])[t, 0], mu32)
        A = P.export_inverse(i, t).cpu().numpy()
        top = np.abs(Aref).max()
        for part in (np.real, np.imag):
            a, r = part(A).astype(np.float64), part(Aref)
            ulp = np.spacing(np.abs(r).astype(np.float32)).astype(np.float64)
            assert np.all(np.abs(a - r) <= 0.5 * ulp + 2.0 ** -36 * top)
            big = np.abs(r) > 1e-2 * top
            assert np.mean(a[big] == r[big].astype(np.float32)) > 0.999


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "x".join(str(s[k]) for k in ("Nx", "Ny", "Nt", "Nc")))
def test_adjoint_rounded_once(shape):
    """H'y is formed in double-float arithmetic (about 48 bits) and rounded
    once: every element is within half an FP32 ulp of the FP64 oracle's value
    plus 2^-36 max|H'y|, and the larger elements equal its FP32 rounding."""
    case = make("tiny", **shape)
    P = plan_for(case, max_iters=1)
    b = P.adjoint(gpu(case.kspace)).cpu().numpy()
    ref = oracle.adjoint_op(case.kspace, case.sens, case.mask)
    top = np.abs(ref).max()
    for part in (np.real, np.imag):
        a, r = part(b).astype(np.float64), part(ref)
        ulp = np.spacing(np.abs(r).astype(np.float32)).astype(np.float64)
        assert np.all(np.abs(a - r) <= 0.5 * ulp + 2.0 ** -36 * top)
        big = np.abs(r) > 1e-2 * top
        assert np.mean(a[big] == r[big].astype(np.float32)) > 0.999


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "x".join(str(s[k]) for k in ("Nx", "Ny", "Nt", "Nc")))
def test_apply_inverse(shape):
    case = make("tiny", **shape)
    P = plan_for(case, max_iters=1)
    rng = np.random.default_rng(2)
    r = as64(rng.standard_normal(case.x_true.shape) + 1j * rng.standard_normal(case.x_true.shape))
    x = host(P.inverse(gpu(r)))
    inv = oracle.ColumnInverse(case.sens, case.mask, case.mu)
    assert rel(x, inv.apply(r)) < TOL


def _oracle_solve(case, prior, iters=None, cols=None, tol=0.0):
    prob = oracle.Problem(case.kspace, case.sens, case.mask, case.mu, cols)
    return prob.solve(prior, case.lam, case.mu, case.rho, case.iters if iters is None else iters, tol=tol)


@pytest.mark.parametrize("objective", [1, 2], ids=["fused_objective", "exact_objective"])
@pytest.mark.parametrize("prior", ["tv", "dft"])
def test_tiny_workload_parity(prior, objective):
    """64x64, 8 frames, 4 coils, R=4, lambda=0.01, mu=0.1, 50 iterations."""
    case = make("tiny")
    P = plan_for(case, prior=prior, objective=objective)
    x, info = P.solve(gpu(case.kspace))
    xr, oinfo = _oracle_solve(case, prior)
    assert info.iters == case.iters
    assert rel(host(x), xr) < TOL
    J = np.array(P.trace(case.iters + 1))
    Jr = np.array(oinfo["J"])
    assert np.max(np.abs(J - Jr) / Jr) < TOL
    assert abs(info.J - Jr[-1]) / Jr[-1] < TOL and abs(info.J0 - Jr[0]) / Jr[0] < TOL


@pytest.mark.parametrize("prior", ["tv", "dft"])
def test_coil_phase_along_y(prior):
    """Coil maps whose phase varies along y make every column's coil Gram
    sum_c conj(s_j) s_k complex and non-symmetric, so this case fixes the side
    of the conjugation in Eq. HconjH (a real Gram hides it): the packed
    inverses and the solve match the oracle, and the other side would not."""
    case = make("tiny", Nx=24, Ny=40, Nt=4, Nc=3, R=3, phase_y=1.5, iters=20)
    P = plan_for(case, prior=prior)
    mu32 = float(np.float32(case.mu))
    for i, t in ((5, 1), (17, 3)):
        Aref = oracle.inverse_blocks(oracle.gram_blocks(case.sens, case.mask, [i])[t, 0], mu32)
        other = oracle.inverse_blocks(oracle.gram_blocks(np.conj(case.sens), case.mask, [i])[t, 0], mu32)
        assert rel(other, Aref) > 1e-3          # the conjugation is visible in this case
        assert rel(host(P.export_inverse(i, t)), Aref) < 2e-7
    x, _ = P.solve(gpu(case.kspace))
    xr, _ = _oracle_solve(case, prior)
    assert rel(host(x), xr) < TOL


@pytest.mark.parametrize("storage", ["fp32", "fp16"])
def test_unsampled_entries_are_ignored(storage):
    """recon_solve reads only the sampled k-space rows: large values at the
    unsampled entries change neither the image (bit for bit) nor J, in FP32 and
    in 16-bit storage (whose per-frame scales come from the sampled rows)."""
    case = make("tiny", Nx=24, Ny=32, Nt=4, Nc=2, R=2, iters=6)
    P = plan_for(case, storage=storage)
    x0, i0 = P.solve(gpu(case.kspace))
    x0 = x0.cpu().numpy()
    junk = case.kspace.copy()
    off = ~np.broadcast_to(case.mask[:, None, :, None], junk.shape)
    rng = np.random.default_rng(9)
    junk[off] = 1e3 * (rng.standard_normal(off.sum()) + 1j * rng.standard_normal(off.sum()))
    x1, i1 = P.solve(gpu(junk))
    np.testing.assert_array_equal(x1.cpu().numpy(), x0)
    assert abs(i1.J - i0.J) <= 1e-12 * abs(i0.J)   # FP64 sums added across CTAs in any order


EDGE = [
    dict(Nx=12, Ny=16, Nt=1, Nc=2, R=2),      # one frame: no temporal differences
    dict(Nx=10, Ny=32, Nt=2, Nc=3, R=2),      # two frames
    dict(Nx=45, Ny=40, Nt=6, Nc=3, R=3),      # ragged Ny (padded block), radix 3/5
    dict(Nx=18, Ny=96, Nt=7, Nc=2, R=4),      # odd block count, odd Nt (radix 7)
    dict(Nx=8, Ny=64, Nt=22, Nc=2, R=8),      # Nt = 22 = 2*11 (generic radix stage)
    dict(Nx=6, Ny=32, Nt=24, Nc=2, R=4),      # TV tile of exactly 48 KB dynamic shared memory
]


@pytest.mark.parametrize("prior", ["tv", "dft"])
@pytest.mark.parametrize("shape", EDGE, ids=lambda s: "x".join(str(s[k]) for k in ("Nx", "Ny", "Nt", "Nc")))
def test_edge_shapes(shape, prior):
    case = make("tiny", **shape)
    iters = 12
    xr, oinfo = _oracle_solve(case, prior, iters)
    Jr = np.array(oinfo["J"])
    # exact objective: J(k) within 1e-5 relative
    P = plan_for(case, prior=prior, max_iters=iters, objective=2)
    x, info = P.solve(gpu(case.kspace))
    assert rel(host(x), xr) < TOL
    J = np.array(P.trace(iters + 1))
    assert np.max(np.abs(J - Jr) / Jr) < TOL
    # fused objective: same iterates; data term within its stated bound
    # (the identity's error is <x, e> with e the FP32 residual of (mu I + H'H) x = r:
    # |error| <= 2 (1 + mu) sqrt(Ny) eps ||x||^2, eps = 2^-24) on top of the 1e-5 relative bar
    P2 = plan_for(case, prior=prior, max_iters=iters, objective=1)
    x2, _ = P2.solve(gpu(case.kspace))
    assert rel(host(x2), xr) < TOL
    J2 = np.array(P2.trace(iters + 1))
    Ny = case.x_true.shape[1]
    bound = 2 * (1 + case.mu) * np.sqrt(Ny) * 2.0 ** -24 * np.linalg.norm(xr) ** 2 + TOL * Jr
    assert np.all(np.abs(J2 - Jr) <= bound)


def test_zero_iterations_returns_adjoint():
    case = make("tiny", Nx=16, Ny=32, Nt=3, Nc=2)
    P = plan_for(case, max_iters=0)
    x, info = P.solve(gpu(case.kspace))
    assert info.iters == 0
    assert rel(host(x), oracle.adjoint_op(case.kspace, case.sens, case.mask)) < TOL


def test_full_sampling_alg1_reaches_closed_form():
    case = make("tiny", Nx=16, Ny=32, Nt=8, Nc=3, mask=np.ones((8, 32), bool), lam=0.05, mu=0.2)
    P = plan_for(case, prior="dft", max_iters=60)
    x, _ = P.solve(gpu(case.kspace))
    b = oracle.adjoint_op(case.kspace, case.sens, case.mask)
    w_star = oracle.soft(oracle.psi_dft(b), case.lam / 2)
    assert rel(oracle.psi_dft(host(x)), w_star) < 1e-5


def test_lambda_zero_full_sampling_is_sense():
    case = make("tiny", Nx=16, Ny=32, Nt=4, Nc=3, mask=np.ones((4, 32), bool), lam=0.0, noise=0.0)
    P = plan_for(case, prior="tv", max_iters=40)
    x, _ = P.solve(gpu(case.kspace))
    assert rel(host(x), case.x_true) < 1e-5


def test_tolerance_stop_matches_oracle():
    case = make("tiny")
    _, full = _oracle_solve(case, "tv", 40)
    J = np.array(full["J"])
    d = (J[:-1] - J[1:]) / J[1:]
    # the first k with 0 <= Delta(k) < tol, with tol chosen well inside a gap
    tol = float(np.sqrt(d[9] * d[10])) if d[10] < d[9] else float(d[9] * 1.001)
    _, ostop = _oracle_solve(case, "tv", 40, tol=tol)
    P = plan_for(case, prior="tv", max_iters=40, tol=tol)
    x, info = P.solve(gpu(case.kspace))
    assert info.stopped == 1 and info.iters == ostop["iters"]
    xr, _ = _oracle_solve(case, "tv", ostop["iters"])
    assert rel(host(x), xr) < TOL


def test_mask_not_cartesian_is_rejected():
    from paper_1203_4587_gb300 import Plan, ReconError
    case = make("tiny", Nx=16, Ny=32, Nt=2, Nc=2)
    full = np.repeat(case.mask[:, :, None], 16, axis=2).astype(np.uint8)
    Plan(full, gpu(case.sens), 0.01, 0.1).close()           # constant along kx: accepted
    full[1, 3, 5] ^= 1
    with pytest.raises(ReconError) as e:
        Plan(full, gpu(case.sens), 0.01, 0.1)
    assert e.value.status == 2


@pytest.mark.parametrize("prior", ["tv", "dft"])
def test_cardiac_workload_column_subset(prior):
    """256x256, 32 frames, 12 coils, R=8, 100 iterations: sampled columns vs the oracle.

    Columns are independent (Section IV-C), so the oracle restricted to a
    seeded subset of columns computes those columns exactly.
    """
    case = make("cardiac")
    P = plan_for(case, prior=prior)
    x, info = P.solve(gpu(case.kspace))
    assert info.iters == case.iters and np.isfinite(info.J)
    cols = np.sort(np.random.default_rng(7).choice(256, size=4, replace=False))
    xr, _ = _oracle_solve(case, prior, cols=cols)
    xg = host(x)[:, :, cols]
    assert rel(xg, xr) < TOL


@pytest.mark.parametrize("storage,tol", [("fp16", 3e-2), ("bf16", 2e-1)])
def test_reduced_precision_storage_error_is_reported(storage, tol):
    """16-bit storage (inverses and hybrid coil data), FP32 arithmetic, FP32
    k-space: the error against FP64 is stated, not bit-level.

    The 50-iteration solution amplifies input errors about 100x, so the 16-bit
    rounding (unit roundoff u = 2^-11 fp16, 2^-8 bf16) shows up as ~1e-2 / 1e-1.
    J(k) is evaluated by explicit FFTs on the 16-bit hybrid data: with d = u ||y||
    (the data rounded once), |J - J(x)| <= 2 sqrt(fid) d + d^2 + 1e-5 J(x) against
    the oracle's J of the GPU's own iterate.
    """
    case = make("tiny")
    P = plan_for(case, prior="tv", storage=storage)
    x, info = P.solve(gpu(case.kspace))
    xr, _ = _oracle_solve(case, "tv")
    e = rel(host(x), xr)
    assert e < tol, e
    prob = oracle.Problem(case.kspace, case.sens, case.mask, case.mu)
    J_of_x = oracle.objective_tv(host(x), case.lam, prob.fid)
    fid = float(prob.fid(host(x)))
    d = {"fp16": 2.0 ** -11, "bf16": 2.0 ** -8}[storage] * float(
        np.linalg.norm(case.kspace * case.mask[:, None, :, None]))
    assert abs(info.J - J_of_x) <= 2 * np.sqrt(fid) * d + d * d + 1e-5 * J_of_x


BATCH = [
    dict(Nx=24, Ny=64, Nt=6, Nc=3, R=4, seed=11),
    dict(Nx=40, Ny=40, Nt=8, Nc=4, R=3, seed=12),     # ragged Ny (padded block)
    dict(Nx=16, Ny=96, Nt=5, Nc=2, R=4, seed=13),     # odd block count
    dict(Nx=33, Ny=128, Nt=7, Nc=3, R=6, seed=14),
]


@pytest.mark.parametrize("prior", ["tv", "dft"])
def test_batched_solve_matches_single_solves(prior):
    """Uneven slices in one batch: one launch per step, then a graph replay."""
    from paper_1203_4587_gb300 import Batch
    iters = 15
    cases = [make("tiny", **{k: v for k, v in sh.items()}) for sh in BATCH]
    plans = [plan_for(c, prior=prior, max_iters=iters) for c in cases]
    singles = []
    for c, p in zip(cases, plans):
        x, info = p.solve(gpu(c.kspace))
        singles.append((host(x), info.J))
    batch = Batch(plans)
    ks = [gpu(c.kspace) for c in cases]
    for call in range(2):          # direct run, then graph replay
        outs = batch.solve(ks)
        infos = batch.info()
        for q, (c, (xs, Js)) in enumerate(zip(cases, singles)):
            xb = host(outs[q])
            # same arithmetic, different unit-to-warp assignment (rounding order)
            assert rel(xb, xs) < TOL, (call, q)
            assert infos[q].iters == iters
            # fused objective: absolute error about 2 eps ||x||^2 either way
            assert abs(infos[q].J - Js) <= 4 * 2.0 ** -24 * np.linalg.norm(xs) ** 2 + 1e-6 * Js
            if call == 0:
                xr, _ = _oracle_solve(c, prior, iters)
                assert rel(xb, xr) < TOL, q
    batch.close()


def test_solve_host_pinned_and_pageable_match_device_solve():
    """recon_solve_host reads pinned k-space in place (only the sampled rows,
    through the device mapping) and copies pageable k-space first: both give
    the device solve's image bit for bit, and unsampled entries stay ignored."""
    case = make("tiny", Nx=40, Ny=48, Nt=6, Nc=3, R=4, iters=8)
    P = plan_for(case)
    x_dev, i_dev = P.solve(gpu(case.kspace))
    x_dev = x_dev.cpu().numpy()
    junk = c64(case.kspace).copy()
    off = ~np.broadcast_to(case.mask[:, None, :, None], junk.shape)
    junk[off] = 7e3 + 3e3j                       # never read
    for pinned in (True, False):
        kh = torch.from_numpy(junk.copy())
        if pinned:
            kh = kh.pin_memory()
        ih = torch.zeros((6, 48, 40), dtype=torch.complex64)
        if pinned:
            ih = ih.pin_memory()
        info = P.solve_host(kh, ih)
        np.testing.assert_array_equal(ih.numpy(), x_dev)
        assert abs(info.J - i_dev.J) <= 1e-12 * abs(i_dev.J)
    P.close()
