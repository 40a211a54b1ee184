"""GB300-native Compton ring localisation (arXiv 2411.04785, far-field hot
path): rings from events, ring x direction likelihood sweep with argmax and
seeds, Gauss-Newton refinement - CUDA kernels for sm_103a behind the C ABI of
``libcompton.so`` (``include/compton.h``), bound here with ctypes."""
from .api import (CCError, Localizer, Params, default_params, empty_rings,  # noqa: F401
                  grid_fibonacci, grid_gather, grid_healpix_ring, grid_healpix_nest, grid_order, lib,
                  localize, localize_static, localize_workspace_bytes, refine, refine_workspace_bytes,
                  rings_from_events, trace_enable, trace_read,
                  RingFilter, ring_features, ring_residuals,
                  cluster_maxstep, cluster_spectrum, cluster_workspace_bytes,
                  ring_apex, voxel_count, voxel_universe, backproject, backproject_workspace_bytes)
