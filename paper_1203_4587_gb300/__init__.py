"""GB300-native dynamic-SENSE ADMM reconstruction (sm_103a CUDA behind a C ABI).

Bilen, Wang & Selesnick's augmented-Lagrangian method for Cartesian ky-t
undersampled multi-coil dynamic MRI: Algorithm 1 (synthesis prior, temporal
DFT) and Algorithm 2 (analysis prior, temporal TV) with the exact per-column
data-consistency inverse of Section IV-C.  The C ABI is in
``include/recon.h``; ``binding`` is its ctypes wrapper.
"""

from .binding import Batch, Plan, ReconError, load, default_opts  # noqa: F401

__all__ = ["Batch", "Plan", "ReconError", "load", "default_opts"]
