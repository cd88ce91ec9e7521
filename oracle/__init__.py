"""FP64 CPU oracle of the augmented-Lagrangian (ADMM) dynamic-SENSE method.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The CUDA library
never calls it, and it shares no code with the CUDA path.

Plain NumPy complex128 restatement of Bilen, Wang & Selesnick, "High Speed
Compressed Sensing Reconstruction in Dynamic Parallel MRI Using Augmented
Lagrangian and Parallel Processing":

* operators H, H' of the Cartesian multi-coil model (Section II-A, Eqs.
  mri_csmcoill, H_1, S, F)
* complex soft threshold (Section III, definition of S(a, tau))
* per-column Gram blocks and the exact inverse (mu I + H'H)^{-1}
  (Section IV-C, Eqs. HconjH, separate_x, eigen_mu)
* Algorithm 1 (synthesis prior, temporal DFT, or the undecimated temporal Haar
  frame, a redundant tight frame) and Algorithm 2 (analysis prior, temporal
  TV; or spatio-temporal differences with a conjugate-gradient m-update,
  ``stv.py``), step by step in the paper's order
* objective J and the convergence ratio Delta(k) (Section V, Eq. r_ratio)
* the reverse-mode gradient of unrolled Algorithm 2 (``grad.py``)
* the 16-bit storage encoding with per-frame power-of-two scales
  (``precision.py``)

Every function here is pinned by a ``-m "not gpu"`` test in
``tests/test_oracle_pins.py``, ``tests/test_oracle_grad.py``,
``tests/test_oracle_frame.py``, ``tests/test_oracle_precision.py`` and
``tests/test_oracle_stv.py`` against closed
forms, brute force, finite differences or invariants.  The pins are checked
in turn by ``tests/test_oracle_mutations.py``, which plants plausible slips
in this package's source one at a time and requires a pin to fail for each.
"""

from .admm import *  # noqa: F401,F403
from .admm import __all__ as _admm_all
from .grad import unrolled_tv_adjoint, unrolled_tv_forward, unrolled_tv_loss_and_grad  # noqa: F401
from . import precision  # noqa: F401
from .stv import (admm_analysis_stv, admm_analysis_stv_volume, cg_steps, objective_stv,  # noqa: F401
                  objective_stv_vol, stacked_residuals, stv_M, stv_M_vol, stv_R, stv_R_vol, stv_Radj,
                  stv_Radj_vol)

__all__ = list(_admm_all) + ["unrolled_tv_forward", "unrolled_tv_adjoint", "unrolled_tv_loss_and_grad",
                             "admm_analysis_stv", "cg_steps", "objective_stv", "stv_M", "stv_R", "stv_Radj",
                             "admm_analysis_stv_volume", "objective_stv_vol", "stv_M_vol", "stv_R_vol", "stv_Radj_vol",
                             "stacked_residuals"]
