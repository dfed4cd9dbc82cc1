"""GB300 (sm_103a) implementation of the heat-diffusion hot path of
"Distributed Parallelization of xPU Stencil Computations in Julia"
(arXiv 2211.15716): implicit global grid, halo update, 7-point diffusion step,
hidden communication, reduced-precision, batched and adjoint forms.

The compute runs in libigg.so (hand-written CUDA, see csrc/); `igg` is its
ctypes binding. The library is loaded on first use, never replaced by a CPU
path.
"""
from .igg import (BF16, F32, F64, Batch, RED_MAX, RED_SUM, RED_SUM_DIV, RED_SUM_SQDIFF, Grid,
                  IggError, bounds_status, dtype_code, lib, library_path, reduce)

__all__ = ["Grid", "Batch", "IggError", "reduce", "lib", "library_path", "dtype_code", "bounds_status",
           "F64", "F32", "BF16", "RED_MAX", "RED_SUM", "RED_SUM_DIV", "RED_SUM_SQDIFF"]
