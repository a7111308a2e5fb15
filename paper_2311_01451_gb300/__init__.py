"""GB300 (sm_103a) implementation of randomized strong recursive skeletonization (RSRS).

The computation lives in ``librsrs.so`` (CUDA kernels behind the C ABI of
``include/rsrs.h``); this package only builds it and marshals arguments.
"""
from .rsrs import (RSRS_OP_CALLBACK, RSRS_OP_INVR3D, RSRS_OP_LOG2D, RSRS_PREC_FP64, RSRS_PREC_MIXED,
                   RSRS_SAMPLE_TILE_128x3, RSRS_SAMPLE_TILE_192x2, RSRS_SAMPLE_TILE_192x5_K16, RSRS_SAMPLE_TILE_256x2,
                   RSRS_SAMPLE_TILE_256x4_K16, RSRS_SAMPLE_TILE_2x192x4_K16, RSRS_SAMPLE_TILE_2x256x3_K16,
                   RSRS_SAMPLE_TILE_DEFAULT, RSRS_RESIDUAL_AUTO, RSRS_RESIDUAL_FP64, RSRS_RESIDUAL_FLOAT_FLOAT,
                   RSRS_RESIDUAL_OZAKI,
                   Factor, RSRSError, Stencil7, Tree, Tune, autotune, build_batched, kind_of, lib, wait_selftest, grid_wait_selftest, convert_selftest)

__all__ = ["Tree", "Factor", "Stencil7", "Tune", "autotune", "build_batched", "RSRSError", "lib", "kind_of", "wait_selftest", "grid_wait_selftest", "convert_selftest",
           "RSRS_OP_LOG2D", "RSRS_OP_INVR3D", "RSRS_OP_CALLBACK", "RSRS_PREC_FP64", "RSRS_PREC_MIXED",
           "RSRS_SAMPLE_TILE_DEFAULT", "RSRS_SAMPLE_TILE_256x2", "RSRS_SAMPLE_TILE_128x3", "RSRS_SAMPLE_TILE_192x2",
           "RSRS_SAMPLE_TILE_256x4_K16", "RSRS_SAMPLE_TILE_192x5_K16", "RSRS_SAMPLE_TILE_2x256x3_K16",
           "RSRS_SAMPLE_TILE_2x192x4_K16", "RSRS_RESIDUAL_AUTO", "RSRS_RESIDUAL_FP64", "RSRS_RESIDUAL_FLOAT_FLOAT",
           "RSRS_RESIDUAL_OZAKI"]
