"""GB300-native interpolation MDS and divide-and-conquer MDS.

The compute path is libgbmds.so (hand-written sm_103a CUDA kernels behind the
C ABI in include/gbmds.h); ``paper_2007_11919_gb300.mds`` is its Python
binding.  Build with ``python -m paper_2007_11919_gb300.build``.
"""
from .mds import (MdsError, Model, mds_classical, mds_classical_dist, mds_divide_conquer,
                  mds_embed_new, mds_interpolate, mds_interpolate_affine, mds_interpolate_host,
                  mds_fast, mds_landmarks_maxmin, mds_pivot, mds_set_tune_cache, mds_tune_cache_lookup,
                  mds_tune_cache_store, mds_version)

__all__ = ["MdsError", "Model", "mds_classical", "mds_classical_dist", "mds_divide_conquer",
           "mds_embed_new", "mds_interpolate", "mds_interpolate_affine", "mds_interpolate_host",
           "mds_fast", "mds_landmarks_maxmin", "mds_pivot", "mds_set_tune_cache", "mds_tune_cache_lookup",
           "mds_tune_cache_store", "mds_version"]
