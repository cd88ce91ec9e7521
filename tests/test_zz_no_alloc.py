"""The allocation-free entry point against the plan's inverses (GPU).

recon_gram_inverse_noalloc serves callers that cannot call cudaMalloc (for
example a real-time pipeline that reserves its device memory at start-up, or
code inside a framework whose allocator owns the device): it keeps its FP64
workspace in a fixed static device array.  This test calls it twice in a row
through the C ABI and compares both results with the per-column inverses that
recon_plan_create builds for the same columns (read back with
recon_export_inverse), at the tolerance the other inverse tests use.  It is
in a file of its own, collected last.
"""

import numpy as np
import pytest

import synthdata

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_noalloc_inverse_matches_plan_twice():
    from paper_1203_4587_gb300 import Plan, binding
    case = synthdata.make_case("tiny", Nx=12, Ny=64, Nt=3, Nc=4)
    sens = torch.from_numpy(case.sens.astype(np.complex64)).cuda()
    plan = Plan(case.mask.astype(np.uint8), sens, case.lam, case.mu, max_iters=1)
    cols = [(i, t) for t in range(3) for i in (0, 5, 11)]
    ref = torch.stack([plan.export_inverse(i, t) for i, t in cols])
    mask_rows = torch.from_numpy(np.stack([case.mask[t] for _, t in cols]).astype(np.uint8)).cuda()
    sens_cols = torch.stack([sens[:, :, i] for i, _ in cols]).contiguous()      # [nblk][Nc][Ny]
    out = torch.empty_like(ref)
    for call in range(2):
        out.fill_(float("nan"))
        binding.gram_inverse_noalloc(mask_rows, sens_cols, case.mu, out=out)
        torch.cuda.synchronize()
        a = out.cpu().numpy().astype(np.complex128)
        b = ref.cpu().numpy().astype(np.complex128)
        err = np.linalg.norm(a - b) / np.linalg.norm(b)
        assert err < 2e-7, (call, err)


def test_noalloc_more_blocks_than_workspaces():
    """Ny = 512: the 16 MiB array holds three 4 MiB workspaces, so five blocks
    run on three CTAs and two of them factorise a second block in the same
    workspace (the grid-stride path)."""
    from paper_1203_4587_gb300 import Plan, binding
    case = synthdata.make_case("tiny", Nx=5, Ny=512, Nt=1, Nc=3)
    sens = torch.from_numpy(case.sens.astype(np.complex64)).cuda()
    plan = Plan(case.mask.astype(np.uint8), sens, case.lam, case.mu, max_iters=1)
    ref = torch.stack([plan.export_inverse(i, 0) for i in range(5)])
    mask_rows = torch.from_numpy(np.repeat(case.mask[:1], 5, axis=0).astype(np.uint8)).cuda()
    sens_cols = torch.stack([sens[:, :, i] for i in range(5)]).contiguous()
    out = torch.full_like(ref, float("nan"))
    binding.gram_inverse_noalloc(mask_rows, sens_cols, case.mu, out=out)
    torch.cuda.synchronize()
    a = out.cpu().numpy().astype(np.complex128)
    b = ref.cpu().numpy().astype(np.complex128)
    for blk in range(5):
        err = np.linalg.norm(a[blk] - b[blk]) / np.linalg.norm(b[blk])
        assert err < 2e-7, (blk, err)
    plan.close()


def test_noalloc_reports_a_non_finite_coil_profile():
    """An infinite coil sample makes a non-finite pivot: the call returns
    RECON_ERR_NONFINITE (6), and a following call with finite input is fine."""
    from paper_1203_4587_gb300 import binding
    lib = binding.load()
    Ny, Nc = 32, 2
    m = torch.ones((2, Ny), dtype=torch.uint8, device="cuda")
    s = torch.full((2, Nc, Ny), 0.5 + 0.0j, dtype=torch.complex64, device="cuda")
    s[1, 0, 3] = complex(float("inf"), 0.0)
    o = torch.empty((2, Ny, Ny), dtype=torch.complex64, device="cuda")
    st = lib.recon_gram_inverse_noalloc(Ny, Nc, 2, binding._ptr(m), binding._ptr(s), 0.1, binding._ptr(o), None)
    assert st == 6, st
    s[1, 0, 3] = 0.5
    st = lib.recon_gram_inverse_noalloc(Ny, Nc, 2, binding._ptr(m), binding._ptr(s), 0.1, binding._ptr(o), None)
    assert st == 0, lib.recon_last_error()
    assert torch.isfinite(torch.view_as_real(o)).all()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    from paper_1203_4587_gb300 import binding
    lib = binding.load()
    m = torch.zeros((1, 1024), dtype=torch.uint8, device="cuda")
    s = torch.zeros((1, 1, 1024), dtype=torch.complex64, device="cuda")
    o = torch.zeros((1, 1), dtype=torch.complex64, device="cuda")
    st = lib.recon_gram_inverse_noalloc(1024, 1, 1, binding._ptr(m), binding._ptr(s), 0.1, binding._ptr(o), None)
    assert st == 7  # RECON_ERR_UNSUPPORTED
    assert b"static scratch" in lib.recon_last_error()
