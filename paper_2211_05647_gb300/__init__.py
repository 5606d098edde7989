"""GB300-native coupled Yee-FDTD + kinetic electron solver (arXiv 2211.05647).

The computation lives in the CUDA library built from ``csrc/`` (C ABI:
``include/fdtd_plasma.h``); this package is its ctypes binding.
"""
from .fdtd_plasma import (Solver, Batch, MlpTrainer, mlp_forward, mlp_forward_tc, MLP_NPARAMS, FdtdError, load_library, LIB_PATH, SIGNATURES, QUANTITY, selftest_wait_timeout, selftest_timed_wait)  # noqa: F401

__all__ = ["Solver", "Batch", "MlpTrainer", "mlp_forward", "mlp_forward_tc", "MLP_NPARAMS", "FdtdError", "load_library", "LIB_PATH", "SIGNATURES", "QUANTITY", "selftest_wait_timeout", "selftest_timed_wait"]
