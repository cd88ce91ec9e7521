"""Thin Python binding of the C ABI in ``include/recon.h`` (ctypes).

Argument marshalling only: torch tensors supply device memory and the current
CUDA stream; every step of the reconstruction runs in the library's kernels.
There is no fallback: if the library is missing or cannot load, ``load()``
raises.

Layouts (complex64 tensors, row-major):
  mask   uint8 [Nt, Ny]        sens  [Nc, Ny, Nx]
  kspace [Nt, Nc, Ny, Nx]      image [Nt, Ny, Nx]
"""

from __future__ import annotations

import ctypes as C
import math
import os

import numpy as np

import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "lib", "librecon.so")

PRIOR = {"tv": 0, "dft": 1, "haar": 2, "stv": 3}
STORAGE = {"fp32": 0, "fp16": 1, "bf16": 2}
STATUS = {0: "RECON_OK", 1: "RECON_ERR_INVALID_ARG", 2: "RECON_ERR_MASK_NOT_CARTESIAN", 3: "RECON_ERR_OOM",
          4: "RECON_ERR_CUDA", 5: "RECON_ERR_TIMEOUT", 6: "RECON_ERR_NONFINITE", 7: "RECON_ERR_UNSUPPORTED"}

# every entry point declared in include/recon.h
EXPORTS = ["recon_default_opts", "recon_plan_create", "recon_solve", "recon_solve_host", "recon_get_trace",
           "recon_destroy", "recon_apply_adjoint", "recon_apply_forward", "recon_apply_inverse",
           "recon_export_inverse", "recon_inverse_bytes", "recon_status_string", "recon_last_error",
           "recon_get_profile", "recon_kernel_launches", "recon_gram_inverse_noalloc",
           "recon_batch_create", "recon_batch_solve", "recon_batch_info", "recon_batch_destroy",
           "recon_grad_create", "recon_grad_forward", "recon_grad_backward", "recon_grad_destroy",
           "recon_solve_kspace", "recon_quantize_kspace", "recon_autotune", "recon_batch_autotune",
           "recon_plan_create_slab", "recon_solve_slabs", "recon_plan_set_mu", "recon_selftest_wait_timeout",
           "recon_volume_create", "recon_plan_set_profile"]


class Opts(C.Structure):
    _fields_ = [("rho", C.c_float), ("max_iters", C.c_int), ("tol", C.c_double), ("storage", C.c_int),
                ("objective", C.c_int), ("mask_full", C.c_int), ("col_stages", C.c_int), ("profile", C.c_int),
                ("frame_levels", C.c_int), ("spatial_weight", C.c_float), ("cg_steps", C.c_int),
                ("persistent", C.c_int), ("overlap", C.c_int)]


class Info(C.Structure):
    _fields_ = [("iters", C.c_int), ("J", C.c_double), ("J0", C.c_double), ("delta", C.c_double),
                ("stopped", C.c_int), ("primal_res", C.c_double), ("dual_res", C.c_double)]


class KSpace(C.Structure):
    _fields_ = [("data", C.c_void_p), ("storage", C.c_int), ("frame_scale", C.c_void_p)]


class Tuning(C.Structure):
    _fields_ = [("temporal_tile_px", C.c_int), ("col_stages", C.c_int), ("rows_per_block", C.c_int),
                ("combine_coils", C.c_int), ("objective_coils", C.c_int), ("temporal_ms", C.c_float),
                ("col_ms", C.c_float), ("rows_ms", C.c_float), ("combine_ms", C.c_float),
                ("objective_ms", C.c_float), ("from_cache", C.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Profile(C.Structure):
    _fields_ = [("inverse_ms", C.c_double), ("inverse_launches", C.c_int), ("temporal_ms", C.c_double),
                ("temporal_launches", C.c_int), ("solve_ms", C.c_double), ("inverse_passes", C.c_int),
                ("persistent", C.c_int)]


class ReconError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


_lib = None


def load(path: str = LIB_PATH):
    """Loads the library and declares the signatures (raises if absent)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ReconError(-1, f"CUDA library not built: {path} (run paper_1203_4587_gb300.build)")
    lib = C.CDLL(path)
    vp, fp, i, f, d = C.c_void_p, C.c_void_p, C.c_int, C.c_float, C.c_double
    lib.recon_default_opts.argtypes = [C.POINTER(Opts)]
    lib.recon_default_opts.restype = None
    lib.recon_plan_create.argtypes = [C.POINTER(vp), i, i, i, i, vp, fp, f, f, i, C.POINTER(Opts), vp]
    lib.recon_plan_create.restype = i
    lib.recon_solve.argtypes = [vp, fp, fp, C.POINTER(Info), vp]
    lib.recon_solve.restype = i
    lib.recon_solve_host.argtypes = [vp, fp, fp, C.POINTER(Info), vp]
    lib.recon_solve_host.restype = i
    lib.recon_get_trace.argtypes = [vp, C.POINTER(C.c_double), i]
    lib.recon_get_trace.restype = i
    lib.recon_destroy.argtypes = [vp]
    lib.recon_destroy.restype = i
    for name in ("recon_apply_adjoint", "recon_apply_forward", "recon_apply_inverse"):
        getattr(lib, name).argtypes = [vp, fp, fp, vp]
        getattr(lib, name).restype = i
    lib.recon_export_inverse.argtypes = [vp, i, i, fp, vp]
    lib.recon_export_inverse.restype = i
    lib.recon_inverse_bytes.argtypes = [vp]
    lib.recon_inverse_bytes.restype = C.c_size_t
    lib.recon_status_string.argtypes = [i]
    lib.recon_status_string.restype = C.c_char_p
    lib.recon_last_error.argtypes = []
    lib.recon_last_error.restype = C.c_char_p
    lib.recon_get_profile.argtypes = [vp, C.POINTER(Profile)]
    lib.recon_get_profile.restype = i
    lib.recon_kernel_launches.argtypes = []
    lib.recon_kernel_launches.restype = C.c_ulonglong
    lib.recon_gram_inverse_noalloc.argtypes = [i, i, i, vp, fp, f, fp, vp]
    lib.recon_gram_inverse_noalloc.restype = i
    lib.recon_batch_create.argtypes = [C.POINTER(vp), C.POINTER(vp), i]
    lib.recon_batch_create.restype = i
    lib.recon_batch_solve.argtypes = [vp, C.POINTER(vp), C.POINTER(vp), vp]
    lib.recon_batch_solve.restype = i
    lib.recon_batch_info.argtypes = [vp, C.POINTER(Info), vp]
    lib.recon_batch_info.restype = i
    lib.recon_batch_destroy.argtypes = [vp]
    lib.recon_batch_destroy.restype = i
    lib.recon_grad_create.argtypes = [C.POINTER(vp), C.POINTER(vp), i, i]
    lib.recon_grad_create.restype = i
    lib.recon_grad_forward.argtypes = [vp, C.POINTER(vp), C.POINTER(vp), vp]
    lib.recon_grad_forward.restype = i
    lib.recon_grad_backward.argtypes = [vp, C.POINTER(vp), C.POINTER(vp), C.POINTER(C.c_double),
                                        C.POINTER(C.c_double), vp]
    lib.recon_grad_backward.restype = i
    lib.recon_grad_destroy.argtypes = [vp]
    lib.recon_grad_destroy.restype = i
    lib.recon_solve_kspace.argtypes = [vp, C.POINTER(KSpace), fp, C.POINTER(Info), vp]
    lib.recon_solve_kspace.restype = i
    lib.recon_quantize_kspace.argtypes = [i, i, i, i, fp, i, vp, fp, vp]
    lib.recon_quantize_kspace.restype = i
    lib.recon_plan_create_slab.argtypes = [C.POINTER(vp), i, i, i, i, vp, fp, f, f, i, C.POINTER(Opts), i, i, vp]
    lib.recon_plan_create_slab.restype = i
    lib.recon_solve_slabs.argtypes = [i, i, i, i, vp, fp, f, f, i, C.POINTER(Opts), i, fp, fp, C.POINTER(d),
                                      C.POINTER(Info), vp]
    lib.recon_solve_slabs.restype = i
    lib.recon_volume_create.argtypes = [C.POINTER(vp), C.POINTER(vp), i, f]
    lib.recon_volume_create.restype = i
    lib.recon_selftest_wait_timeout.argtypes = [i, C.POINTER(d), vp]
    lib.recon_selftest_wait_timeout.restype = i
    lib.recon_plan_set_mu.argtypes = [vp, f, vp]
    lib.recon_plan_set_mu.restype = i
    lib.recon_autotune.argtypes = [vp, C.POINTER(Tuning), vp]
    lib.recon_autotune.restype = i
    lib.recon_batch_autotune.argtypes = [vp, C.POINTER(Tuning), vp]
    lib.recon_batch_autotune.restype = i
    lib.recon_plan_set_profile.argtypes = [vp, i]
    lib.recon_plan_set_profile.restype = i
    _lib = lib
    return lib


def _check(st):
    if st != 0:
        raise ReconError(st, _lib.recon_last_error().decode())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _ptr(t: torch.Tensor):
    return C.c_void_p(t.data_ptr())


def _c64(t: torch.Tensor, dev=None) -> torch.Tensor:
    t = torch.as_tensor(t)
    if not torch.is_complex(t):
        raise TypeError("complex tensor expected")
    t = t.to(torch.complex64)
    if dev is not None:
        t = t.to(dev)
    return t.contiguous()


def _need(t, shape, name, where="cuda", dtype=None):
    """Returns ``t`` if it is a contiguous tensor of ``dtype`` (default
    complex64) and ``shape`` on device type ``where`` (None: any); raises
    otherwise.  The library receives raw pointers and cannot check the sizes
    of the buffers behind them."""
    dtype = torch.complex64 if dtype is None else dtype
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name}: a torch tensor is expected")
    if t.dtype != dtype:
        raise TypeError(f"{name}: {dtype} expected, got {t.dtype}")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name}: shape {tuple(t.shape)}, expected {tuple(shape)}")
    if not t.is_contiguous():
        raise ValueError(f"{name}: a contiguous tensor is expected")
    if where is not None and t.device.type != where:
        raise ValueError(f"{name}: a {where} tensor is expected, got {t.device.type}")
    return t


def _need_count(items, n, name):
    """One entry per plan: the library reads exactly n pointers."""
    items = list(items)
    if len(items) != n:
        raise ValueError(f"{name}: {len(items)} entries for {n} plans")
    return items


def _mask_shape_ok(mshape, Nt_ok, Ny, Nx):
    """A row mask [Nt][Ny] or a full mask [Nt][Ny][Nx] for images of Ny x Nx."""
    return Nt_ok and ((len(mshape) == 2 and mshape[1] == Ny) or
                      (len(mshape) == 3 and mshape[1] == Ny and mshape[2] == Nx))


def default_opts(**over) -> Opts:
    o = Opts()
    load().recon_default_opts(C.byref(o))
    names = {f for f, _ in Opts._fields_}
    for k, v in over.items():
        if k not in names:
            raise TypeError(f"unknown option {k!r}")
        if k == "storage" and isinstance(v, str):
            v = STORAGE[v]
        setattr(o, k, v)
    return o


class Plan:
    """Owns one ``recon_plan``: geometry, sensitivities, mask and the packed inverses."""

    def __init__(self, mask, sens, lam, mu, prior="tv", stream=None, slab=None, **opts):
        """slab=(i0, width): a plan over columns i0 .. i0+width-1 (recon_plan_create_slab)."""
        lib = load()
        sens = _c64(sens, "cuda")
        if sens.dim() != 3:
            raise ValueError(f"sens: [Nc, Ny, Nx] expected, got shape {tuple(sens.shape)}")
        Nc, Ny, Nx = sens.shape
        mask = torch.as_tensor(mask).to(torch.uint8).contiguous()
        if not _mask_shape_ok(tuple(mask.shape), mask.dim() >= 2 and mask.shape[0] >= 1, Ny, Nx):
            raise ValueError(f"mask: [Nt, {Ny}] or [Nt, {Ny}, {Nx}] expected, got shape {tuple(mask.shape)}")
        o = default_opts(**opts)
        if mask.dim() == 3:
            o.mask_full = 1
        Nt = mask.shape[0]
        self.shape = dict(Nx=int(Nx), Ny=int(Ny), Nt=int(Nt), Nc=int(Nc))
        self.prior, self.lam, self.mu, self.opts = prior, float(lam), float(mu), o
        self._h = C.c_void_p()
        mdev = mask.cuda() if mask.device.type != "cuda" else mask
        if slab is None:
            st = lib.recon_plan_create(C.byref(self._h), int(Nx), int(Ny), int(Nt), int(Nc), _ptr(mdev), _ptr(sens),
                                       float(lam), float(mu), PRIOR[prior], C.byref(o), _stream(stream))
        else:
            st = lib.recon_plan_create_slab(C.byref(self._h), int(Nx), int(Ny), int(Nt), int(Nc), _ptr(mdev),
                                            _ptr(sens), float(lam), float(mu), PRIOR[prior], C.byref(o),
                                            int(slab[0]), int(slab[1]), _stream(stream))
        _check(st)
        self._keep = (mdev, sens)
        self.slab = slab

    def set_mu(self, mu, stream=None):
        """Recomputes the inverses for a new mu (recon_plan_set_mu)."""
        _check(load().recon_plan_set_mu(self._h, float(mu), _stream(stream)))
        self.mu = float(mu)

    def close(self):
        if self._h:
            load().recon_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _img(self):
        s = self.shape
        alloc = torch.zeros if getattr(self, "slab", None) is not None else torch.empty   # a slab writes its columns only
        return alloc((s["Nt"], s["Ny"], s["Nx"]), dtype=torch.complex64, device="cuda")

    def _ksp(self):
        return torch.empty(self.kshape, dtype=torch.complex64, device="cuda")

    @property
    def kshape(self):
        """k-space layout [Nt, Nc, Ny, Nx]."""
        s = self.shape
        return (s["Nt"], s["Nc"], s["Ny"], s["Nx"])

    @property
    def ishape(self):
        """image layout [Nt, Ny, Nx]."""
        s = self.shape
        return (s["Nt"], s["Ny"], s["Nx"])

    def solve(self, kspace, out=None, info=True, stream=None):
        """Runs the reconstruction; returns (image, Info or None)."""
        k = _need(_c64(kspace, "cuda"), self.kshape, "kspace")
        out = self._img() if out is None else _need(out, self.ishape, "out")
        inf = Info() if info else None
        st = load().recon_solve(self._h, _ptr(k), _ptr(out), C.byref(inf) if info else None, _stream(stream))
        _check(st)
        return out, inf

    def autotune(self, stream=None) -> Tuning:
        """Picks the kernels' launch shapes by timing them (recon_autotune)."""
        t = Tuning()
        _check(load().recon_autotune(self._h, C.byref(t), _stream(stream)))
        return t

    def solve_quantized(self, q, out=None, info=True, stream=None):
        """Runs the reconstruction from 16-bit k-space ``q`` (a QuantizedKspace)."""
        _need(q.data, self.kshape, "q.data", dtype=torch.int32)
        _need(q.frame_scale, (self.kshape[0],), "q.frame_scale", dtype=torch.float32)
        if q.storage not in ("fp16", "bf16"):
            raise ValueError(f"q.storage: fp16 or bf16 expected, got {q.storage!r}")
        out = self._img() if out is None else _need(out, self.ishape, "out")
        inf = Info() if info else None
        y = KSpace(q.data.data_ptr(), STORAGE[q.storage], q.frame_scale.data_ptr())
        st = load().recon_solve_kspace(self._h, C.byref(y), _ptr(out), C.byref(inf) if info else None,
                                       _stream(stream))
        _check(st)
        return out, inf

    def solve_host(self, kspace_host, image_host, stream=None):
        """Host buffers in and out (copies inside the call); returns Info."""
        _need(kspace_host, self.kshape, "kspace_host", "cpu")
        _need(image_host, self.ishape, "image_host", "cpu")
        inf = Info()
        st = load().recon_solve_host(self._h, _ptr(kspace_host), _ptr(image_host), C.byref(inf), _stream(stream))
        _check(st)
        return inf

    def trace(self, n=None):
        n = self.opts.max_iters + 1 if n is None else n
        buf = (C.c_double * n)()
        _check(load().recon_get_trace(self._h, buf, n))
        return [buf[k] for k in range(n)]

    def adjoint(self, kspace, stream=None):
        k = _need(_c64(kspace, "cuda"), self.kshape, "kspace")
        out = self._img()
        _check(load().recon_apply_adjoint(self._h, _ptr(k), _ptr(out), _stream(stream)))
        return out

    def forward(self, image, stream=None):
        x = _need(_c64(image, "cuda"), self.ishape, "image")
        out = self._ksp()
        _check(load().recon_apply_forward(self._h, _ptr(x), _ptr(out), _stream(stream)))
        return out

    def inverse(self, image, stream=None):
        x = _need(_c64(image, "cuda"), self.ishape, "image")
        out = self._img()
        _check(load().recon_apply_inverse(self._h, _ptr(x), _ptr(out), _stream(stream)))
        return out

    def export_inverse(self, i, t, stream=None):
        Ny = self.shape["Ny"]
        out = torch.empty((Ny, Ny), dtype=torch.complex64, device="cuda")
        _check(load().recon_export_inverse(self._h, int(i), int(t), _ptr(out), _stream(stream)))
        return out

    def set_profile(self, on: bool):
        """Per-kernel event timing of later solves on or off (recon_plan_set_profile)."""
        _check(load().recon_plan_set_profile(self._h, 1 if on else 0))

    def profile(self) -> Profile:
        pr = Profile()
        _check(load().recon_get_profile(self._h, C.byref(pr)))
        return pr

    @property
    def inverse_bytes(self) -> int:
        return int(load().recon_inverse_bytes(self._h))


class Batch:
    """Several plans solved together (recon_batch_*): one launch per step, graph replay."""

    def __init__(self, plans):
        self.plans = list(plans)
        arr = (C.c_void_p * len(self.plans))(*[p._h.value for p in self.plans])
        self._h = C.c_void_p()
        _check(load().recon_batch_create(C.byref(self._h), arr, len(self.plans)))

    def solve(self, kspaces, outs=None, stream=None):
        """kspaces: list of device complex64 tensors; returns the list of images."""
        n = len(self.plans)
        ks = [_need(_c64(k, "cuda"), p.kshape, f"kspaces[{q}]")
              for q, (k, p) in enumerate(zip(_need_count(kspaces, n, "kspaces"), self.plans))]
        if outs is None:
            outs = [p._img() for p in self.plans]
        else:
            outs = [_need(o, p.ishape, f"outs[{q}]")
                    for q, (o, p) in enumerate(zip(_need_count(outs, n, "outs"), self.plans))]
        self._keep = (ks, outs)
        ka = (C.c_void_p * len(ks))(*[k.data_ptr() for k in ks])
        oa = (C.c_void_p * len(outs))(*[o.data_ptr() for o in outs])
        _check(load().recon_batch_solve(self._h, ka, oa, _stream(stream)))
        return outs

    def autotune(self, stream=None) -> Tuning:
        """Temporal tile width and ring depth for this batch (recon_batch_autotune)."""
        t = Tuning()
        _check(load().recon_batch_autotune(self._h, C.byref(t), _stream(stream)))
        return t

    def info(self, stream=None):
        arr = (Info * len(self.plans))()
        _check(load().recon_batch_info(self._h, arr, _stream(stream)))
        return list(arr)

    def close(self):
        if self._h:
            load().recon_batch_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Volume(Batch):
    """Slices of a 3D volume in z order, coupled by w_z D_z in the spatio-temporal
    prior (recon_volume_create); solved like a batch."""

    def __init__(self, plans, wz):
        self.plans = list(plans)
        arr = (C.c_void_p * len(self.plans))(*[p._h.value for p in self.plans])
        self._h = C.c_void_p()
        _check(load().recon_volume_create(C.byref(self._h), arr, len(self.plans), float(wz)))


class Grad:
    """Differentiable unrolled Algorithm 2 over plans (recon_grad_*).

    ``forward`` runs the plans' max_iters steps keeping checkpoints;
    ``backward`` takes dL/dx_K per slice and returns dL/dy per slice and
    dL/dlambda, dL/dmu (NumPy float64 arrays, one entry per slice).  The plans
    must not be solved with between the two calls.
    """

    def __init__(self, plans, checkpoint_every=5):
        self.plans = list(plans)
        arr = (C.c_void_p * len(self.plans))(*[p._h.value for p in self.plans])
        self._h = C.c_void_p()
        _check(load().recon_grad_create(C.byref(self._h), arr, len(self.plans), int(checkpoint_every)))

    def forward(self, kspaces, stream=None):
        n = len(self.plans)
        ks = [_need(_c64(k, "cuda"), p.kshape, f"kspaces[{q}]")
              for q, (k, p) in enumerate(zip(_need_count(kspaces, n, "kspaces"), self.plans))]
        outs = [p._img() for p in self.plans]
        ka = (C.c_void_p * len(ks))(*[k.data_ptr() for k in ks])
        oa = (C.c_void_p * len(outs))(*[o.data_ptr() for o in outs])
        _check(load().recon_grad_forward(self._h, ka, oa, _stream(stream)))
        return outs

    def backward(self, grad_images, stream=None):
        n = len(self.plans)
        gs = [_need(_c64(g, "cuda"), p.ishape, f"grad_images[{q}]")
              for q, (g, p) in enumerate(zip(_need_count(grad_images, n, "grad_images"), self.plans))]
        outs = [p._ksp() for p in self.plans]
        ga = (C.c_void_p * n)(*[g.data_ptr() for g in gs])
        oa = (C.c_void_p * n)(*[o.data_ptr() for o in outs])
        gl = (C.c_double * n)()
        gm = (C.c_double * n)()
        _check(load().recon_grad_backward(self._h, ga, oa, gl, gm, _stream(stream)))
        return outs, np.array(gl[:], dtype=np.float64), np.array(gm[:], dtype=np.float64)

    def close(self):
        if self._h:
            load().recon_grad_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class _UnrolledTV(torch.autograd.Function):
    @staticmethod
    def forward(ctx, grad, lam, mu, *kspaces):
        ctx.grad = grad
        return tuple(grad.forward(kspaces))

    @staticmethod
    def backward(ctx, *grad_images):
        g = [torch.zeros_like(p._img()) if gi is None else gi for p, gi in zip(ctx.grad.plans, grad_images)]
        gk, gl, gm = ctx.grad.backward(g)
        return (None, torch.from_numpy(gl), torch.from_numpy(gm), *gk)


def unrolled_tv(grad, kspaces, lam, mu):
    """Images x_K of every slice as a differentiable function of the k-space
    data and of lambda, mu (float64 tensors with one entry per slice).

    lam and mu must equal the plans' values (the plans hold the inverses for
    their mu); their gradients are dL/dlambda and dL/dmu at those values.
    """
    lam = torch.as_tensor(lam, dtype=torch.float64)
    mu = torch.as_tensor(mu, dtype=torch.float64)
    lv, mv = lam.detach().reshape(-1).tolist(), mu.detach().reshape(-1).tolist()
    for q, p in enumerate(grad.plans):
        if abs(lv[q] - p.lam) > 1e-6 * abs(p.lam) or abs(mv[q] - p.mu) > 1e-6 * abs(p.mu):
            raise ValueError(f"slice {q}: lambda/mu differ from the plan's")
    return list(_UnrolledTV.apply(grad, lam, mu, *kspaces))


class QuantizedKspace:
    """16-bit k-space with per-frame power-of-two scales (recon_quantize_kspace).

    ``data`` int32 [Nt, Nc, Ny, Nx] holding (re, im) 16-bit pairs, ``frame_scale``
    float32 [Nt]; entry = pair * frame_scale[t].
    """

    def __init__(self, data, storage, frame_scale):
        self.data, self.storage, self.frame_scale = data, storage, frame_scale

    def to_complex(self):
        """Dequantised complex64 copy (for inspection and tests)."""
        dt = torch.float16 if self.storage == "fp16" else torch.bfloat16
        pairs = self.data.view(dt).view(*self.data.shape, 2).float()
        return torch.complex(pairs[..., 0], pairs[..., 1]) * self.frame_scale.view(-1, 1, 1, 1)


def quantize_kspace(kspace, storage="fp16", stream=None):
    """complex64 [Nt, Nc, Ny, Nx] on the GPU -> QuantizedKspace (fp16 or bf16)."""
    k = _c64(kspace, "cuda")
    if k.dim() != 4:
        raise ValueError(f"kspace: [Nt, Nc, Ny, Nx] expected, got shape {tuple(k.shape)}")
    if storage not in ("fp16", "bf16"):
        raise ValueError(f"storage: fp16 or bf16 expected, got {storage!r}")
    Nt, Nc, Ny, Nx = k.shape
    data = torch.empty((Nt, Nc, Ny, Nx), dtype=torch.int32, device="cuda")
    scale = torch.empty((Nt,), dtype=torch.float32, device="cuda")
    _check(load().recon_quantize_kspace(int(Nx), int(Ny), int(Nt), int(Nc), _ptr(k), STORAGE[storage], _ptr(data),
                                        _ptr(scale), _stream(stream)))
    return QuantizedKspace(data, storage, scale)


def gram_inverse_noalloc(mask_rows, sens_cols, mu, out=None, stream=None):
    """Allocation-free per-column inverses (recon_gram_inverse_noalloc).

    mask_rows uint8 [nblk, Ny] and sens_cols complex64 [nblk, Nc, Ny] on the
    GPU; returns complex64 [nblk, Ny, Ny] (``out`` if given).
    """
    m = torch.as_tensor(mask_rows).to(torch.uint8).contiguous()
    s = _c64(sens_cols, "cuda")
    if s.dim() != 3:
        raise ValueError(f"sens_cols: [nblk, Nc, Ny] expected, got shape {tuple(s.shape)}")
    nblk, Nc, Ny = s.shape
    _need(m, (nblk, Ny), "mask_rows", dtype=torch.uint8)
    if out is None:
        out = torch.empty((nblk, Ny, Ny), dtype=torch.complex64, device="cuda")
    else:
        _need(out, (nblk, Ny, Ny), "out")
    _check(load().recon_gram_inverse_noalloc(int(Ny), int(Nc), int(nblk), _ptr(m), _ptr(s), float(mu), _ptr(out),
                                             _stream(stream)))
    return out


def solve_slabs(mask, sens, lam, mu, kspace, width, prior="tv", out=None, stream=None, **opts):
    """The whole problem solved slab after slab of `width` columns
    (recon_solve_slabs); returns (image, Info, J trace as a list)."""
    lib = load()
    s = _c64(sens, "cuda")
    k = _c64(kspace, "cuda")
    if s.dim() != 3:
        raise ValueError(f"sens: [Nc, Ny, Nx] expected, got shape {tuple(s.shape)}")
    Nc, Ny, Nx = s.shape
    m = torch.as_tensor(mask).to(torch.uint8).contiguous()
    if not _mask_shape_ok(tuple(m.shape), m.dim() >= 2 and m.shape[0] >= 1, Ny, Nx):
        raise ValueError(f"mask: [Nt, {Ny}] or [Nt, {Ny}, {Nx}] expected, got shape {tuple(m.shape)}")
    o = default_opts(**opts)
    if m.dim() == 3:
        o.mask_full = 1
    Nt = m.shape[0]
    _need(k, (Nt, Nc, Ny, Nx), "kspace")
    mdev = m.cuda() if m.device.type != "cuda" else m
    if out is None:
        out = torch.empty((Nt, Ny, Nx), dtype=torch.complex64, device="cuda")
    else:
        _need(out, (Nt, Ny, Nx), "out")
    tr = (C.c_double * (o.max_iters + 1))()
    inf = Info()
    _check(lib.recon_solve_slabs(int(Nx), int(Ny), int(Nt), int(Nc), _ptr(mdev), _ptr(s), float(lam), float(mu),
                                 PRIOR[prior], C.byref(o), int(width), _ptr(k), _ptr(out), tr, C.byref(inf),
                                 _stream(stream)))
    return out, inf, list(tr)


def selftest_wait_timeout(limit_us, stream=None):
    """Runs recon_selftest_wait_timeout: returns (status, host-measured ms)."""
    ms = C.c_double(0.0)
    st = load().recon_selftest_wait_timeout(int(limit_us), C.byref(ms), _stream(stream))
    return st, ms.value


def kernel_launches() -> int:
    """Kernels this library has launched in this process."""
    return int(load().recon_kernel_launches())


def algorithmic_bytes_per_iter(Nx, Ny, Nt, Nc, total_rows, esize=8):
    """Bytes one ADMM iteration must move at minimum: packed inverses
    Ny(Ny+1)/2 per column, plus sensitivities, hybrid data and H'y."""
    return (esize * Nx * Nt * Ny * (Ny + 1) // 2 + 8 * Nx * Ny * Nc + 8 * Nx * total_rows * Nc + 8 * Nx * Ny * Nt)


def rsqrt(n):
    return 1.0 / math.sqrt(n)
