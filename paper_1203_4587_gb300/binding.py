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

import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "lib", "librecon.so")

PRIOR = {"tv": 0, "dft": 1}
STORAGE = {"fp32": 0, "fp16": 1, "bf16": 2}
STATUS = {0: "RECON_OK", 1: "RECON_ERR_INVALID_ARG", 2: "RECON_ERR_MASK_NOT_CARTESIAN", 3: "RECON_ERR_OOM",
          4: "RECON_ERR_CUDA", 5: "RECON_ERR_TIMEOUT", 6: "RECON_ERR_NONFINITE", 7: "RECON_ERR_UNSUPPORTED"}

# every entry point declared in include/recon.h
EXPORTS = ["recon_default_opts", "recon_plan_create", "recon_solve", "recon_solve_host", "recon_get_trace",
           "recon_destroy", "recon_apply_adjoint", "recon_apply_forward", "recon_apply_inverse",
           "recon_export_inverse", "recon_inverse_bytes", "recon_status_string", "recon_last_error",
           "recon_get_profile", "recon_kernel_launches", "recon_gram_inverse_noalloc",
           "recon_batch_create", "recon_batch_solve", "recon_batch_info", "recon_batch_destroy"]


class Opts(C.Structure):
    _fields_ = [("rho", C.c_float), ("max_iters", C.c_int), ("tol", C.c_double), ("storage", C.c_int),
                ("objective", C.c_int), ("mask_full", C.c_int), ("col_stages", C.c_int), ("profile", C.c_int)]


class Info(C.Structure):
    _fields_ = [("iters", C.c_int), ("J", C.c_double), ("J0", C.c_double), ("delta", C.c_double),
                ("stopped", C.c_int)]


class Profile(C.Structure):
    _fields_ = [("inverse_ms", C.c_double), ("inverse_launches", C.c_int), ("temporal_ms", C.c_double),
                ("temporal_launches", C.c_int), ("solve_ms", C.c_double)]


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


def default_opts(**over) -> Opts:
    o = Opts()
    load().recon_default_opts(C.byref(o))
    for k, v in over.items():
        if k == "storage" and isinstance(v, str):
            v = STORAGE[v]
        setattr(o, k, v)
    return o


class Plan:
    """Owns one ``recon_plan``: geometry, sensitivities, mask and the packed inverses."""

    def __init__(self, mask, sens, lam, mu, prior="tv", stream=None, **opts):
        lib = load()
        sens = _c64(sens, "cuda")
        Nc, Ny, Nx = sens.shape
        mask = torch.as_tensor(mask).to(torch.uint8).contiguous()
        o = default_opts(**opts)
        if mask.dim() == 3:
            o.mask_full = 1
        Nt = mask.shape[0]
        self.shape = dict(Nx=int(Nx), Ny=int(Ny), Nt=int(Nt), Nc=int(Nc))
        self.prior, self.lam, self.mu, self.opts = prior, float(lam), float(mu), o
        self._h = C.c_void_p()
        mdev = mask.cuda() if mask.device.type != "cuda" else mask
        st = lib.recon_plan_create(C.byref(self._h), int(Nx), int(Ny), int(Nt), int(Nc), _ptr(mdev), _ptr(sens),
                                   float(lam), float(mu), PRIOR[prior], C.byref(o), _stream(stream))
        _check(st)
        self._keep = (mdev, sens)

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
        return torch.empty((s["Nt"], s["Ny"], s["Nx"]), dtype=torch.complex64, device="cuda")

    def _ksp(self):
        s = self.shape
        return torch.empty((s["Nt"], s["Nc"], s["Ny"], s["Nx"]), dtype=torch.complex64, device="cuda")

    def solve(self, kspace, out=None, info=True, stream=None):
        """Runs the reconstruction; returns (image, Info or None)."""
        k = _c64(kspace, "cuda")
        out = self._img() if out is None else out
        inf = Info() if info else None
        st = load().recon_solve(self._h, _ptr(k), _ptr(out), C.byref(inf) if info else None, _stream(stream))
        _check(st)
        return out, inf

    def solve_host(self, kspace_host, image_host, stream=None):
        """Host buffers in and out (copies inside the call); returns Info."""
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
        k = _c64(kspace, "cuda")
        out = self._img()
        _check(load().recon_apply_adjoint(self._h, _ptr(k), _ptr(out), _stream(stream)))
        return out

    def forward(self, image, stream=None):
        x = _c64(image, "cuda")
        out = self._ksp()
        _check(load().recon_apply_forward(self._h, _ptr(x), _ptr(out), _stream(stream)))
        return out

    def inverse(self, image, stream=None):
        x = _c64(image, "cuda")
        out = self._img()
        _check(load().recon_apply_inverse(self._h, _ptr(x), _ptr(out), _stream(stream)))
        return out

    def export_inverse(self, i, t, stream=None):
        Ny = self.shape["Ny"]
        out = torch.empty((Ny, Ny), dtype=torch.complex64, device="cuda")
        _check(load().recon_export_inverse(self._h, int(i), int(t), _ptr(out), _stream(stream)))
        return out

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
        ks = [_c64(k, "cuda") for k in kspaces]
        outs = [p._img() for p in self.plans] if outs is None else outs
        self._keep = (ks, outs)
        ka = (C.c_void_p * len(ks))(*[k.data_ptr() for k in ks])
        oa = (C.c_void_p * len(outs))(*[o.data_ptr() for o in outs])
        _check(load().recon_batch_solve(self._h, ka, oa, _stream(stream)))
        return outs

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


def gram_inverse_noalloc(mask_rows, sens_cols, mu, out=None, stream=None):
    """Allocation-free per-column inverses (recon_gram_inverse_noalloc).

    mask_rows uint8 [nblk, Ny] and sens_cols complex64 [nblk, Nc, Ny] on the
    GPU; returns complex64 [nblk, Ny, Ny] (``out`` if given).
    """
    m = torch.as_tensor(mask_rows).to(torch.uint8).contiguous()
    s = _c64(sens_cols, "cuda")
    nblk, Nc, Ny = s.shape
    if out is None:
        out = torch.empty((nblk, Ny, Ny), dtype=torch.complex64, device="cuda")
    _check(load().recon_gram_inverse_noalloc(int(Ny), int(Nc), int(nblk), _ptr(m), _ptr(s), float(mu), _ptr(out),
                                             _stream(stream)))
    return out


def kernel_launches() -> int:
    """Kernels this library has launched in this process."""
    return int(load().recon_kernel_launches())


def algorithmic_bytes_per_iter(Nx, Ny, Nt, Nc, total_rows, esize=8):
    """Bytes one ADMM iteration must move at minimum: packed inverses
    Ny(Ny+1)/2 per column, plus sensitivities, hybrid data and H'y."""
    return (esize * Nx * Nt * Ny * (Ny + 1) // 2 + 8 * Nx * Ny * Nc + 8 * Nx * total_rows * Nc + 8 * Nx * Ny * Nt)


def rsqrt(n):
    return 1.0 / math.sqrt(n)
