"""The oracle's pins catch plausible slips: each case plants one mistake in the
oracle's source (a dropped term, a wrong sign, conjugation or index, a
transposed operand, a wrong rounding rule) and checks that at least one of
the independent pins named beside it fails.

A mutant is the oracle module's source with one snippet replaced (the snippet
must occur exactly once, so a case cannot go stale silently), executed as a
fresh module whose functions and classes then stand in for the originals
everywhere in the ``oracle`` package for the duration of the case.  A control
case installs an unchanged copy and requires every pin to pass, so a failure
under a mutant comes from the planted mistake and not from the mechanism.

Mistakes are planted in the oracle only, on the CPU.
"""

import os
import sys
import types

import pytest

import oracle
import test_oracle_frame as FR
import test_oracle_grad as GR
import test_oracle_pins as PI
import test_oracle_precision as PR
import test_oracle_stv as ST

ORACLE_DIR = os.path.dirname(oracle.__file__)
PACKAGE_MODULES = ("oracle", "oracle.admm", "oracle.stv", "oracle.grad", "oracle.precision")


def install(monkeypatch, module, old, new):
    """Swaps in a copy of ``oracle.<module>`` with ``old`` replaced by ``new``."""
    path = os.path.join(ORACLE_DIR, module + ".py")
    with open(path) as fh:
        src = fh.read()
    assert src.count(old) == 1, f"snippet not found exactly once in {module}.py: {old!r}"
    real = sys.modules["oracle." + module]
    mutant = types.ModuleType(real.__name__)
    mutant.__package__ = "oracle"
    mutant.__file__ = path
    exec(compile(src.replace(old, new), path, "exec"), mutant.__dict__)
    for name, obj in list(vars(real).items()):
        if name.startswith("__") or not callable(obj) or name not in mutant.__dict__:
            continue
        for mname in PACKAGE_MODULES:
            m = sys.modules[mname]
            if getattr(m, name, None) is obj:
                monkeypatch.setattr(m, name, mutant.__dict__[name])


def fails(pin, *args):
    try:
        pin(*args)
    except Exception:   # AssertionError from the pin, or an error the mistake provokes
        return True
    return False


def P(fn, *args):
    return (fn, args)


# (id, module, snippet, replacement, pins that must include a failure)
MUTATIONS = [
    # Section III: the soft threshold
    ("soft-half-threshold", "admm", "out[keep] = (mag[keep] - tau) * a[keep] / mag[keep]",
     "out[keep] = (mag[keep] - 0.5 * tau) * a[keep] / mag[keep]",
     [P(PI.test_soft_threshold_special_values), P(PI.test_soft_threshold_is_the_prox_by_grid_search)]),
    ("soft-l1-modulus", "admm", "mag = np.abs(a)\n", "mag = np.abs(a.real) + np.abs(a.imag)\n",
     [P(PI.test_soft_threshold_special_values), P(PI.test_soft_threshold_is_the_prox_by_grid_search)]),
    # Section II-A: the operators
    ("forward-vertical-sign", "admm", 'k = np.fft.fft(coil, axis=-2, norm="ortho")',
     'k = np.fft.ifft(coil, axis=-2, norm="ortho")',
     [P(PI.test_adjoint_identity), P(PI.test_unitary_parseval_and_impulse),
      P(PI.test_forward_matches_acquisition_simulator_noise_free)]),
    ("forward-mask-dropped", "admm", "return k * mask[:, None, :, None]", "return k",
     [P(PI.test_adjoint_identity), P(PI.test_forward_matches_acquisition_simulator_noise_free),
      P(PI.test_gram_blocks_equal_dense_HtH, 0.0)]),
    ("adjoint-without-conj", "admm", "return np.sum(np.conj(sens)[None] * img, axis=1)",
     "return np.sum(sens[None] * img, axis=1)",
     [P(PI.test_adjoint_identity)]),
    ("hybrid-data-forward-fft", "admm", 'return np.fft.ifft(y * mask[:, None, :, None], axis=-1, norm="ortho")',
     'return np.fft.fft(y * mask[:, None, :, None], axis=-1, norm="ortho")',
     [P(PI.test_hybrid_residual_equals_full_residual)]),
    ("residual-columns-mask-dropped", "admm", "r = (yhat[:, :, :, cols] - z) * mask[:, None, :, None]",
     "r = yhat[:, :, :, cols] - z",
     [P(PI.test_hybrid_residual_equals_full_residual)]),
    # Section IV-C: Gram blocks and the inverse
    ("gram-printed-conjugation", "admm", 'K = np.einsum("cji,cki->ijk", np.conj(S), S)',
     'K = np.einsum("cji,cki->ijk", S, np.conj(S))',
     [P(PI.test_gram_blocks_equal_dense_HtH, 1.5)]),
    ("gram-unsampled-rows", "admm", "Ft = F[mask[t], :]", "Ft = F[~mask[t], :]",
     [P(PI.test_gram_blocks_equal_dense_HtH, 0.0), P(PI.test_gram_full_sampling_is_identity_and_circulant)]),
    ("inverse-mu-squared", "admm", "1.0 / (e + mu)", "1.0 / (e + mu * mu)",
     [P(PI.test_inverse_blocks_identity), P(PI.test_inverse_single_coil_is_pointwise_kspace_inverse)]),
    ("inverse-applied-transposed", "admm", 'np.einsum("tijk,tki->tji", self.A, r)',
     'np.einsum("tikj,tki->tji", self.A, r)',
     [P(PI.test_inverse_single_coil_is_pointwise_kspace_inverse), P(PI.test_kkt_tv_on_tiny_problem)]),
    # Eq. TV and the m-update
    ("tv-difference-reversed", "admm", "return x[1:] - x[:-1]", "return x[:-1] - x[1:]",
     [P(PI.test_tv_difference_and_adjoint)]),
    ("tv-adjoint-sign", "admm", "out[:-1] -= u\n    out[1:] += u", "out[:-1] += u\n    out[1:] -= u",
     [P(PI.test_tv_difference_and_adjoint)]),
    ("tv-matrix-wrong-index", "admm", "D[t, t + 1] = 1.0", "D[t, (t + 2) % Nt] = 1.0",
     [P(PI.test_tv_m_matrix_matches_dct_eigen_closed_form), P(PI.test_alg2_two_frames_closed_form)]),
    # Algorithm 2
    ("alg2-threshold-mu2", "admm", "v = soft(tv_D(m) + d1, lam / (2.0 * mu1))",
     "v = soft(tv_D(m) + d1, lam / (2.0 * mu2))",
     [P(PI.test_kkt_tv_on_tiny_problem), P(PI.test_alg2_two_frames_closed_form)]),
    ("alg2-rhs-without-rho", "admm", "rhs = tv_Dadj(v - d1, Nt) + (mu2 / mu1) * (x + d2)",
     "rhs = tv_Dadj(v - d1, Nt) + (x + d2)",
     [P(PI.test_kkt_tv_on_tiny_problem), P(PI.test_alg2_two_frames_closed_form)]),
    ("alg2-d2-sign", "admm", "        d2 = d2 - (m - x)\n        k_done = k\n        if fid is not None:\n"
     "            J.append(objective_tv(x, lam, fid))",
     "        d2 = d2 + (m - x)\n        k_done = k\n        if fid is not None:\n"
     "            J.append(objective_tv(x, lam, fid))",
     [P(PI.test_kkt_tv_on_tiny_problem), P(PI.test_alg2_two_frames_closed_form)]),
    # Algorithm 1
    ("alg1-d-sign", "admm", "d = d - (w - v)", "d = d + (w - v)",
     [P(PI.test_kkt_dft_on_tiny_problem), P(PI.test_alg1_full_sampling_reaches_soft_threshold_closed_form)]),
    ("alg1-lemma-term-dropped", "admm",
     "w = (u - psi(psi_adj(u))) / mu + psi(inv.apply(b + mu * psi_adj(v + d)))",
     "w = psi(inv.apply(b + mu * psi_adj(v + d)))",
     [P(FR.test_kkt_alg1_with_redundant_haar_frame)]),
    ("psi-dft-not-unitary", "admm", 'return np.fft.fft(x, axis=0, norm="ortho")', "return np.fft.fft(x, axis=0)",
     [P(PI.test_kkt_dft_on_tiny_problem), P(PI.test_alg1_full_sampling_reaches_soft_threshold_closed_form)]),
    ("psi-dft-adjoint-not-unitary", "admm", 'return np.fft.ifft(w, axis=0, norm="ortho")',
     "return np.fft.ifft(w, axis=0)",
     [P(PI.test_kkt_dft_on_tiny_problem), P(PI.test_objectives_closed_forms)]),
    ("dft-matrix-sign", "admm", "return np.exp(-2j * np.pi * np.outer(q, q) / n) / np.sqrt(n)",
     "return np.exp(2j * np.pi * np.outer(q, q) / n) / np.sqrt(n)",
     [P(PI.test_gram_blocks_equal_dense_HtH, 0.0)]),
    ("column-subset-wrong-columns", "admm", "self.b = self.b_full[:, :, self.cols]",
     "self.b = self.b_full[:, :, :len(self.cols)]",
     [P(PI.test_column_subset_is_exact)]),
    ("haar-detail-scale", "admm", "out.append((a - nxt) / 2.0)", "out.append((a - nxt) / np.sqrt(2.0))",
     [P(FR.test_tight_and_redundant, 8, 3), P(FR.test_channel_frequency_response_closed_form, 8, 2)]),
    # Objective, Eq. r_ratio, residuals
    ("objective-without-lambda", "admm", "return lam * float(np.abs(tv_D(x)).sum()) + fid(x)",
     "return float(np.abs(tv_D(x)).sum()) + fid(x)",
     [P(PI.test_objectives_closed_forms)]),
    ("dft-objective-halved-fidelity", "admm", "return lam * float(np.abs(w).sum()) + fid(psi_dft_adj(w))",
     "return lam * float(np.abs(w).sum()) + 0.5 * fid(psi_dft_adj(w))",
     [P(PI.test_objectives_closed_forms)]),
    ("data-residual-not-squared", "admm", "return float(np.vdot(r, r).real)\n\n\ndef data_residual_columns",
     "return float(np.sqrt(np.vdot(r, r).real))\n\n\ndef data_residual_columns",
     [P(PI.test_objectives_closed_forms)]),
    ("delta-over-previous", "admm", "return (J_prev - J) / J\n", "return (J_prev - J) / J_prev\n",
     [P(PI.test_objective_and_delta_definitions)]),
    ("tv-residual-split-dropped", "admm",
     "rp = np.vdot(v - tv_D(m), v - tv_D(m)).real + np.vdot(m - x, m - x).real",
     "rp = np.vdot(v - tv_D(m), v - tv_D(m)).real",
     [P(PI.test_tv_residuals_vanish_at_convergence_and_follow_the_duals)]),
    ("synthesis-dual-wrong-difference", "admm", "dw = w - w_prev", "dw = w - v",
     [P(PI.test_synthesis_residuals_vanish_at_convergence_and_follow_the_dual, "dft")]),
    # Spatio-temporal prior and CG (Section IV-B)
    ("stv-adjoint-boundary-sign", "stv", "out[tuple(lo)] -= u", "out[tuple(lo)] += u",
     [P(ST.test_R_adjoint, (4, 5, 6), 0.37), P(ST.test_M_equals_kronecker_assembly, (3, 4, 5), 0.5)]),
    ("stv-adjoint-weight-dropped", "stv", "+ ws * _diff_adj(uy, 1, Ny)", "+ _diff_adj(uy, 1, Ny)",
     [P(ST.test_R_adjoint, (4, 5, 6), 0.37)]),
    ("cg-beta-inverted", "stv", "p = r + (gamma_new / gamma) * p", "p = r + (gamma / gamma_new) * p",
     [P(ST.test_cg_exact_after_n_steps), P(ST.test_cg_converges_to_dct_closed_form, 1.0)]),
    ("cg-alpha-wrong-product", "stv", "alpha = gamma / _dot(p, q).real", "alpha = gamma / _dot(q, q).real",
     [P(ST.test_cg_exact_after_n_steps), P(ST.test_cg_converges_to_dct_closed_form, 1.0)]),
    ("stv-rhs-without-rho", "stv", "rhs = stv_Radj(tuple(a - d for a, d in zip(v, d1)), ws, shape) + r2 * (x + d2)",
     "rhs = stv_Radj(tuple(a - d for a, d in zip(v, d1)), ws, shape) + (x + d2)",
     [P(ST.test_zero_spatial_weight_is_temporal_tv)]),
    ("stv-residual-split-dropped", "stv",
     "rp = sum(np.vdot(a - b, a - b).real for a, b in zip(v, R(m))) + np.vdot(m - x, m - x).real",
     "rp = sum(np.vdot(a - b, a - b).real for a, b in zip(v, R(m)))",
     [P(ST.test_stv_residuals_follow_the_duals_and_vanish)]),
    ("stv-dual-wrong-weight", "stv", "rd = mu1 ** 2 * sum(", "rd = mu2 ** 2 * sum(",
     [P(ST.test_zero_spatial_weight_is_temporal_tv)]),
    ("stv-objective-unweighted", "stv", "return lam * float(sum(np.abs(c).sum() for c in stv_R(x, ws))) + fid(x)",
     "return lam * float(sum(np.abs(c).sum() for c in stv_R(x, 1.0))) + fid(x)",
     [P(ST.test_objective_is_lambda_l1_plus_fidelity)]),
    ("volume-z-weight-dropped", "stv", "wz * (x[1:] - x[:-1]))", "(x[1:] - x[:-1]))",
     [P(ST.test_volume_R_adjoint, (3, 2, 4, 5))]),
    ("haar-adjoint-shift-direction", "admm", "a = (a + np.roll(a, sh, axis=0)) / 2.0 + (d - np.roll(d, sh, axis=0)) / 2.0",
     "a = (a + np.roll(a, -sh, axis=0)) / 2.0 + (d - np.roll(d, -sh, axis=0)) / 2.0",
     [P(FR.test_tight_and_redundant, 8, 3)]),
    ("stv-R-weight-dropped", "stv", "ws * (x[:, :, 1:] - x[:, :, :-1])", "(x[:, :, 1:] - x[:, :, :-1])",
     [P(ST.test_R_adjoint, (4, 5, 6), 0.37)]),
    ("volume-d1-sign", "stv", "d1 = tuple(d - (a - c) for d, a, c in zip(d1, v, Rm))\n        d2 = d2 - (m - x)\n"
     "        if fids is not None:",
     "d1 = tuple(d + (a - c) for d, a, c in zip(d1, v, Rm))\n        d2 = d2 - (m - x)\n"
     "        if fids is not None:",
     [P(ST.test_volume_of_one_slice_is_the_2d_algorithm)]),
    # Differentiable form (unrolled Algorithm 2 and its reverse pass)
    ("unrolled-threshold-doubled", "grad", "v = soft(tv_D(m) + d1, tau1)", "v = soft(tv_D(m) + d1, 2.0 * tau1)",
     [P(GR.test_forward_is_algorithm_2, 4)]),
    ("unrolled-d2-sign", "grad", "d2 = d2 - m_new + x_new", "d2 = d2 + m_new - x_new",
     [P(GR.test_forward_is_algorithm_2, 4)]),
    ("soft-adjoint-tangent-sign", "grad", "(vbar[on] - n[on] * proj[on])", "(vbar[on] + n[on] * proj[on])",
     [P(GR.test_soft_threshold_adjoint_matches_fd)]),
    ("mu-gradient-stale-iterate", "grad", "mu_bar += float(np.vdot(rb, m1 - d20).real)",
     "mu_bar += float(np.vdot(rb, m0 - d20).real)",
     [P(GR.test_unrolled_gradient_matches_central_differences, 1)]),
    # 16-bit storage encoding
    ("bf16-round-half-up", "precision", "((b + 0x7FFF + lsb) >> 16)", "((b + 0x8000) >> 16)",
     [P(PR.test_rounding_is_nearest_even_by_brute_force, "bf16")]),
    ("dequantize-scale-dropped", "precision",
     "return (bits_to_float(re_bits, storage) + 1j * bits_to_float(im_bits, storage)) * s",
     "return bits_to_float(re_bits, storage) + 1j * bits_to_float(im_bits, storage)",
     [P(PR.test_round_trip_error_bound, "fp16", 2.0 ** -11)]),
    ("frame-scale-exponent", "precision", "out[t] = 2.0 ** (int(e) - 15)", "out[t] = 2.0 ** (int(e) - 14)",
     [P(PR.test_frame_scales_are_powers_of_two_in_range)]),
]


@pytest.mark.parametrize("case", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_pins_catch_planted_mistake(case, monkeypatch):
    _, module, old, new, pins = case
    install(monkeypatch, module, old, new)
    caught = [pin.__name__ for pin, args in pins if fails(pin, *args)]
    assert caught, "no pin caught the planted mistake"


@pytest.mark.parametrize("module", ["admm", "stv", "grad", "precision"])
def test_unchanged_copy_passes_every_pin(module, monkeypatch):
    install(monkeypatch, module, "import numpy as np\n", "import numpy as np\n")
    pins = {pin: args for _, mod, _, _, ps in MUTATIONS if mod == module for pin, args in ps}
    failed = [pin.__name__ for pin, args in pins.items() if fails(pin, *args)]
    assert not failed, failed
