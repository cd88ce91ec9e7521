"""GB300-native dynamic-SENSE ADMM reconstruction (sm_103a CUDA behind a C ABI).

Bilen, Wang & Selesnick's augmented-Lagrangian method for Cartesian ky-t
undersampled multi-coil dynamic MRI: Algorithm 1 (synthesis prior: temporal
DFT, or an undecimated temporal Haar frame) and Algorithm 2 (analysis prior:
temporal TV, or spatio-temporal differences with a CG m-update, also over 3D
volumes) with the exact per-column data-consistency inverse of Section IV-C.  The C ABI is in
``include/recon.h``; ``binding`` is its ctypes wrapper, with ``unrolled_tv``
the differentiable (autograd) form of K steps of Algorithm 2.
"""

from .binding import Batch, Grad, Plan, ReconError, Volume, default_opts, load, unrolled_tv  # noqa: F401

__all__ = ["Batch", "Grad", "Plan", "ReconError", "Volume", "load", "default_opts", "unrolled_tv"]
