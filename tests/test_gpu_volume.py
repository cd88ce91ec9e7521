"""GPU parity of 3D volumes: slices in z order coupled by w_z D_z in the
spatio-temporal prior, one CG over the volume (recon_volume_create), against
the FP64 oracle's volume algorithm (oracle.admm_analysis_stv_volume).
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


def slices(nz, **shape):
    out = []
    for z in range(nz):
        c = synthdata.make_case("tiny", seed=70 + z, **shape)
        c.kspace = as64(c.kspace)
        c.sens = as64(c.sens)
        out.append(c)
    return out


def plans_for(cases, ws, cg, iters, **opts):
    from paper_1203_4587_gb300 import Plan
    return [Plan(c.mask.astype(np.uint8), gpu(c.sens), c.lam, c.mu, prior="stv", rho=c.rho, max_iters=iters,
                 spatial_weight=ws, cg_steps=cg, **opts) for c in cases]


def oracle_volume(cases, ws, wz, cg, iters):
    c0 = cases[0]
    probs = [oracle.Problem(c.kspace, c.sens, c.mask, c.mu) for c in cases]
    return oracle.admm_analysis_stv_volume([p.b for p in probs], [p.inv for p in probs], c0.lam, c0.mu, c0.rho, iters,
                                           ws=ws, wz=wz, cg=cg, fids=[p.fid for p in probs])


@pytest.mark.parametrize("wz", [1.0, 0.4, 0.0])
def test_volume_matches_oracle(wz):
    from paper_1203_4587_gb300 import Volume
    cases = slices(3, Nx=24, Ny=32, Nt=4, Nc=2, R=2)
    iters, ws, cg = 12, 0.8, 4
    P = plans_for(cases, ws, cg, iters, objective=2)
    V = Volume(P, wz)
    xs = V.solve([gpu(c.kspace) for c in cases])
    xg = np.stack([x.cpu().numpy().astype(np.complex128) for x in xs])
    xr, info = oracle_volume(cases, ws, wz, cg, iters)
    assert rel(xg, xr) < TOL
    J = np.sum([p.trace(iters + 1) for p in P], axis=0)   # the volume's J is the sum over slices
    Jr = np.array(info["J"])
    assert np.max(np.abs(J - Jr) / Jr) < TOL


def test_volume_of_one_slice_is_the_2d_solve():
    from paper_1203_4587_gb300 import Volume
    cases = slices(1, Nx=40, Ny=48, Nt=6, Nc=3, R=3)
    P = plans_for(cases, 1.0, 5, 10)
    k = gpu(cases[0].kspace)
    x2d, _ = P[0].solve(k)
    x2d = x2d.cpu().numpy()
    xv = Volume(P, 2.0).solve([k])[0].cpu().numpy()
    np.testing.assert_array_equal(xv, x2d)


def test_volume_graph_replay_and_uneven_rows():
    from paper_1203_4587_gb300 import Volume
    cases = slices(4, Nx=20, Ny=97, Nt=3, Nc=2, R=4)
    iters, ws, wz, cg = 8, 0.7, 1.3, 3
    V = Volume(plans_for(cases, ws, cg, iters, objective=0), wz)
    ks = [gpu(c.kspace) for c in cases]
    x1 = [x.cpu().numpy() for x in V.solve(ks)]      # direct run, then capture
    x2 = [x.cpu().numpy() for x in V.solve(ks)]      # graph replay
    for a, b in zip(x1, x2):
        np.testing.assert_array_equal(a, b)
    xr, _ = oracle_volume(cases, ws, wz, cg, iters)
    assert rel(np.stack(x1).astype(np.complex128), xr) < TOL


def test_volume_rejects_mixed_plans():
    from paper_1203_4587_gb300 import Plan, ReconError, Volume
    a = slices(2, Nx=16, Ny=32, Nt=4, Nc=2, R=2)
    b = slices(1, Nx=16, Ny=32, Nt=5, Nc=2, R=2)
    with pytest.raises(ReconError):                    # Nt differs
        Volume(plans_for(a, 1.0, 3, 4) + plans_for(b, 1.0, 3, 4), 1.0)
    with pytest.raises(ReconError):                    # a stop tolerance
        Volume(plans_for(a, 1.0, 3, 4, tol=1e-3), 1.0)
    tv = Plan(a[0].mask.astype(np.uint8), gpu(a[0].sens), a[0].lam, a[0].mu, prior="tv", max_iters=4)
    with pytest.raises(ReconError):                    # not the spatio-temporal prior
        Volume([tv], 1.0)
    with pytest.raises(ReconError):
        Volume(plans_for(a, 1.0, 3, 4), -1.0)
