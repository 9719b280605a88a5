"""GB300-native low-rank noisy-circuit evolution (LRET, arXiv:2009.06657).

rho = V V^dag with V a 2^n x c complex slab on the GPU; gates, Kraus expansion,
Gram, eigensolve, projection and readouts run in the CUDA library liblret
(C ABI in include/lret.h). This package is its Python binding.
"""
from ._ffi import LIB_PATH, LRError, exported_symbols  # noqa: F401
from .sim import LRBatch, LRExpectation, LRSim, kraus_preset, launch_count, pauli_masks, run_ops  # noqa: F401
