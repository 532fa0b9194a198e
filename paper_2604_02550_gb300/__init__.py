"""GB300-native ACSE hot path: residual, propagation step, energy and adjoint of the
anti-Hermitian contracted Schroedinger equation with the Valdemoro 3-RDM reconstruction.

The computation lives in libacse.so (CUDA, sm_103a) behind the C ABI of include/acse.h;
`_lib` is its ctypes binding and `api` a small torch-facing convenience layer.
"""
from ._lib import (ACSE_BF16X3, ACSE_FP64, ACSE_TF32, AcseError, acse_create, acse_destroy, acse_energy,
                   acse_residual, acse_residual_backward, acse_step, lib, strerror, version)

__all__ = ["ACSE_FP64", "ACSE_BF16X3", "ACSE_TF32", "AcseError", "acse_create", "acse_destroy",
           "acse_energy", "acse_residual", "acse_step", "acse_residual_backward", "lib", "strerror",
           "version"]
