"""Pins of the oracle's 16-bit encoding (oracle.precision), CPU only.

Each rule is checked against something other than its own code: the nearest
representable value found by brute force over all 65536 codes of the format
(ties to the even code), exact powers of two with the stated range, and the
format's relative error bound.
"""

import numpy as np
import pytest

from oracle import precision as P


def _all_values(storage):
    codes = np.arange(65536, dtype=np.uint32).astype(np.uint16)
    if storage == "fp16":
        v = codes.view(np.float16).astype(np.float64)
    else:
        with np.errstate(invalid="ignore"):
            v = (codes.astype(np.uint32) << 16).view(np.float32).astype(np.float64)
    ok = np.isfinite(v)
    return codes[ok], v[ok]


@pytest.mark.parametrize("storage", ["fp16", "bf16"])
def test_rounding_is_nearest_even_by_brute_force(storage):
    codes, vals = _all_values(storage)
    order = np.argsort(vals, kind="stable")
    codes, vals = codes[order], vals[order]
    rng = np.random.default_rng(0)
    x = (rng.standard_normal(400) * np.exp(rng.uniform(-12, 9, 400))).astype(np.float32)
    # exact ties: midpoints between neighbouring representable values
    lo = 20000 if storage == "fp16" else 2000
    mids = ((vals[lo:lo + 40] + vals[lo + 1:lo + 41]) / 2).astype(np.float32)
    x = np.concatenate([x, mids[(mids.astype(np.float64) == (vals[lo:lo + 40] + vals[lo + 1:lo + 41]) / 2)]])
    got = P.round_bits(x, storage)
    for xi, g in zip(x.astype(np.float64), got):
        d = np.abs(vals - xi)
        best = np.flatnonzero(d == d.min())
        cand = [int(codes[b]) for b in best]
        cand_vals = {float(vals[b]) for b in best}
        if len(cand_vals) > 1:   # a tie: the even significand wins
            cand = [c for c in cand if c % 2 == 0]
        assert int(g) in cand, (xi, g, cand)


def test_frame_scales_are_powers_of_two_in_range():
    rng = np.random.default_rng(1)
    k = (rng.standard_normal((5, 3, 8)) + 1j * rng.standard_normal((5, 3, 8))) * np.array(
        [1e-6, 1.0, 37.0, 1e5, 0.0])[:, None, None]
    s = P.frame_scales(k)
    for t in range(5):
        m = max(np.abs(k[t].real).max(), np.abs(k[t].imag).max())
        if m == 0:
            assert s[t] == 1.0
            continue
        e = np.log2(s[t])
        assert e == np.round(e)
        assert 2 ** 14 <= m / s[t] < 2 ** 15


@pytest.mark.parametrize("storage,bound", [("fp16", 2.0 ** -11), ("bf16", 2.0 ** -8)])
def test_round_trip_error_bound(storage, bound):
    rng = np.random.default_rng(2)
    k = ((rng.standard_normal((4, 2, 16, 16)) + 1j * rng.standard_normal((4, 2, 16, 16)))
         * np.array([1e-3, 1.0, 50.0, 3e4])[:, None, None, None]).astype(np.complex64)
    re, im, s = P.quantize_frames(k, storage)
    back = P.dequantize_frames(re, im, s, storage)
    kd = k.astype(np.complex128)
    for t in range(4):
        # components above the format's normal range relative to the frame scale
        big_r = np.abs(kd[t].real) >= 2.0 ** -14 * s[t]
        big_i = np.abs(kd[t].imag) >= 2.0 ** -14 * s[t]
        err_r = np.abs(back[t].real - kd[t].real)[big_r] / np.abs(kd[t].real)[big_r]
        err_i = np.abs(back[t].imag - kd[t].imag)[big_i] / np.abs(kd[t].imag)[big_i]
        assert err_r.max() <= bound and err_i.max() <= bound
