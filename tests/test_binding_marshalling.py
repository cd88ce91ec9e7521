"""The Python binding's marshalling on the CPU, with a stand-in for the C
library (every call returns RECON_OK) and tensors kept on the host: every call
pattern the GPU tests and the benchmark use goes through the binding's own
argument checks and pointer arrays without error, and malformed arguments
raise before any C call.  The numerics are the GPU tests' business."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1203_4587_gb300 import binding as B  # noqa: E402

Nt, Nc, Ny, Nx = 4, 2, 32, 40


class _Fn:
    def __init__(self, name):
        self.name = name
        self.calls = 0

    def __call__(self, *args):
        self.calls += 1
        return b"" if self.name == "recon_last_error" else 0


class _Lib:
    def __init__(self):
        self.fns = {}

    def __getattr__(self, name):
        return self.fns.setdefault(name, _Fn(name))


@pytest.fixture
def lib(monkeypatch):
    fake = _Lib()
    monkeypatch.setattr(B, "load", lambda: fake)
    monkeypatch.setattr(B, "_lib", fake, raising=False)
    monkeypatch.setattr(B, "_stream", lambda stream=None: None)
    c64, need = B._c64, B._need
    monkeypatch.setattr(B, "_c64", lambda t, dev=None: c64(t, None))
    monkeypatch.setattr(B, "_need", lambda t, shape, name, where="cuda", dtype=None: need(t, shape, name, None, dtype))
    monkeypatch.setattr(torch.Tensor, "cuda", lambda self, *a, **k: self)
    for f in ("empty", "zeros"):
        real = getattr(torch, f)
        monkeypatch.setattr(torch, f, lambda *a, _r=real, **k: _r(*a, **{n: v for n, v in k.items() if n != "device"}))
    return fake


def _inputs():
    mask = (np.random.default_rng(0).random((Nt, Ny)) < 0.4).astype(np.uint8)
    sens = torch.zeros((Nc, Ny, Nx), dtype=torch.complex64)
    k = torch.zeros((Nt, Nc, Ny, Nx), dtype=torch.complex64)
    img = torch.zeros((Nt, Ny, Nx), dtype=torch.complex64)
    return mask, sens, k, img


def test_every_call_pattern_marshals(lib):
    mask, sens, k, img = _inputs()
    P = B.Plan(mask, sens, 0.01, 0.1, prior="tv", max_iters=3)
    assert P.kshape == (Nt, Nc, Ny, Nx) and P.ishape == (Nt, Ny, Nx)
    P.solve(k)
    P.solve(k, img, info=False)
    P.adjoint(k)
    P.forward(img)
    P.inverse(img)
    P.solve_host(k, img)
    full = B.Plan(np.repeat(mask[:, :, None], Nx, axis=2), sens, 0.01, 0.1, prior="dft", max_iters=3)
    assert full.opts.mask_full == 1
    B.Plan(mask, sens, 0.01, 0.1, max_iters=3, slab=(8, 16)).solve(k)
    b = B.Batch([P, full])
    b.solve([k, k])
    b.solve([k, k], [img, img.clone()])
    g = B.Grad([P])
    g.forward([k])
    g.backward([img])
    q = B.QuantizedKspace(torch.zeros((Nt, Nc, Ny, Nx), dtype=torch.int32), "fp16", torch.ones(Nt))
    P.solve_quantized(q)
    B.quantize_kspace(k, "bf16")
    rows = torch.zeros((6, Ny), dtype=torch.uint8)
    cols = torch.zeros((6, Nc, Ny), dtype=torch.complex64)
    B.gram_inverse_noalloc(rows, cols, 0.1, out=torch.zeros((6, Ny, Ny), dtype=torch.complex64))
    B.solve_slabs(mask, sens, 0.01, 0.1, k, 16, out=img, max_iters=3)
    lam = torch.tensor([0.01], dtype=torch.float64)
    mu = torch.tensor([0.1], dtype=torch.float64)
    B.unrolled_tv(g, [k.clone().requires_grad_(True)], lam, mu)
    for name in ("recon_plan_create", "recon_solve", "recon_solve_host", "recon_batch_solve", "recon_grad_forward",
                 "recon_grad_backward", "recon_solve_kspace", "recon_quantize_kspace", "recon_gram_inverse_noalloc",
                 "recon_solve_slabs", "recon_plan_create_slab"):
        assert lib.fns[name].calls >= 1, name


def test_malformed_arguments_raise_before_the_call(lib):
    mask, sens, k, img = _inputs()
    P = B.Plan(mask, sens, 0.01, 0.1, max_iters=3)
    b = B.Batch([P, P])
    g = B.Grad([P])
    solves = lib.recon_solve.calls
    bad = [
        lambda: P.solve(k[:, :, :, :-1]),                          # one column short
        lambda: P.solve(k, img[:, :, :-1]),                        # output too small
        lambda: P.solve_host(k.to(torch.complex128), img),        # twice the bytes per entry
        lambda: P.inverse(img.transpose(1, 2)),                    # wrong layout
        lambda: b.solve([k]),                                      # fewer entries than plans
        lambda: g.backward([img, img]),                            # more entries than plans
        lambda: B.Plan(mask[:, :-1], sens, 0.01, 0.1),             # mask rows do not match the image
        lambda: P.solve_quantized(B.QuantizedKspace(torch.zeros((Nt, Nc, Ny, Nx), dtype=torch.int16), "fp16",
                                                     torch.ones(Nt))),
        lambda: B.gram_inverse_noalloc(torch.zeros((5, Ny), dtype=torch.uint8),
                                       torch.zeros((6, Nc, Ny), dtype=torch.complex64), 0.1),
    ]
    for f in bad:
        with pytest.raises((ValueError, TypeError)):
            f()
    assert lib.recon_solve.calls == solves
