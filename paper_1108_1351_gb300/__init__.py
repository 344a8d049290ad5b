"""GB300-native two-stage k-means (Salman et al., arXiv 1108.1351).

The hot path -- sampling, the fused distance / nearest-center / exact-sum
kernels, the FP64 near-tie recheck and the center update -- runs in the CUDA
library ``libkmeans2.so`` (C ABI in ``include/kmeans2.h``).  This package only
binds it (``binding``) and provides seeded synthetic inputs (``synth``).
"""
from .binding import (FitResult, KMeans2Error, LIB_PATH, Profile, Served, Server, Shard,
                      batched_tile_shape, declared_symbols, fit, fit_batched, fit_data_parallel, fit_sharded,
                      fit_streamed, footprint, load, release_memory, sample, step, step_noalloc,
                      strerror, subset_size, version)

__all__ = ["FitResult", "KMeans2Error", "LIB_PATH", "Profile", "Served", "Server", "Shard",
           "batched_tile_shape", "declared_symbols", "fit", "fit_batched", "fit_data_parallel", "fit_sharded",
           "fit_streamed", "footprint", "load", "release_memory", "sample", "step",
           "step_noalloc", "strerror", "subset_size", "version"]
