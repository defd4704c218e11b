"""GB300-native implicit Discrete Elastic Rods step (DisMech, arXiv 2311.18126).

The compute path is the CUDA library ``libdismech.so`` (C ABI in
``include/dismech.h``); ``dismech.System`` is its Python binding.
"""
from .dismech import (System, DismechError, load_library, ensure_built,  # noqa: F401
                      fp64_peak_gflops, solve_band, solve_band_noalloc,
                      gemm_bf16, MLP)
