"""16-bit storage with per-frame power-of-two scales (test infrastructure only).

The paper computes in a single precision.  The reduced-precision form stores
the data a solve keeps (k-space, hybrid coil data, packed inverses) as 16-bit
(re, im) pairs; it is an encoding with plain rules, restated here:

  m_t     = largest |Re| or |Im| over frame t
  scale_t = 2^e with m_t / 2^e in [2^14, 2^15)   (1 when m_t = 0)
  q       = k / scale_t rounded to the nearest FP16 (IEEE binary16) or BF16
            (the upper 16 bits of binary32) value, ties to even
  value   = q * scale_t

k arrives in complex64, and dividing by a power of two is exact, so q is the
single rounding of a binary32 value.

Parity status: pinned in ``tests/test_oracle_precision.py`` (brute-force
nearest representable value over all 65536 codes of each format, exact powers
of two, the range rule of the scales).
"""

from __future__ import annotations

import numpy as np

__all__ = ["frame_scales", "round_bits", "bits_to_float", "quantize_frames", "dequantize_frames"]


def frame_scales(k):
    """scale_t for every frame of k[t, ...] (complex), as float64 powers of two."""
    k = np.asarray(k)
    Nt = k.shape[0]
    out = np.ones(Nt)
    for t in range(Nt):
        m = float(max(np.max(np.abs(k[t].real), initial=0.0), np.max(np.abs(k[t].imag), initial=0.0)))
        if m > 0.0:
            _, e = np.frexp(m)          # m = f 2^e, f in [0.5, 1)
            out[t] = 2.0 ** (int(e) - 15)
    return out


def round_bits(x, storage):
    """Bit patterns (uint16) of binary32 values x rounded to FP16 or BF16."""
    x = np.asarray(x, dtype=np.float32)
    if storage == "fp16":
        return x.astype(np.float16).view(np.uint16)
    if storage == "bf16":
        b = x.view(np.uint32).astype(np.uint64)
        lsb = (b >> 16) & 1
        return ((b + 0x7FFF + lsb) >> 16).astype(np.uint16)
    raise ValueError(storage)


def bits_to_float(bits, storage):
    """Values (float64) of FP16 / BF16 bit patterns."""
    bits = np.asarray(bits, dtype=np.uint16)
    if storage == "fp16":
        return bits.view(np.float16).astype(np.float64)
    if storage == "bf16":
        return (bits.astype(np.uint32) << 16).view(np.float32).astype(np.float64)
    raise ValueError(storage)


def quantize_frames(k, storage):
    """(re_bits, im_bits, scales) of complex64 k[t, ...]."""
    k = np.asarray(k, dtype=np.complex64)
    s = frame_scales(k)
    shape = (-1,) + (1,) * (k.ndim - 1)
    q = k / s.reshape(shape).astype(np.float32)
    return round_bits(q.real, storage), round_bits(q.imag, storage), s


def dequantize_frames(re_bits, im_bits, scales, storage):
    """complex128 values q * scale_t."""
    shape = (-1,) + (1,) * (np.ndim(re_bits) - 1)
    s = np.asarray(scales, dtype=np.float64).reshape(shape)
    return (bits_to_float(re_bits, storage) + 1j * bits_to_float(im_bits, storage)) * s
