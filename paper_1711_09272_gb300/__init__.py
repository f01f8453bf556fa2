"""GB300-native Roe-AM finite-volume solver (2D Euler) behind a C ABI.

The compute path is libroeam.so (CUDA, sm_103a): see include/roeam.h for the ABI
and `roeam` for its Python binding. PyTorch, when used, only provides device
memory, pinned host buffers and streams.
"""
from .roeam import (Batch, RoeamError, load_library, make_desc, roeam_cell_count, roeam_check,  # noqa: F401
                    roeam_conserved_totals, roeam_create_grid, roeam_destroy_grid, roeam_flux_residual,
                    roeam_get_state, roeam_launch_count, roeam_residual_norm, roeam_rk_step, roeam_set_state,
                    roeam_version, roeam_tile_config_count, roeam_tile_config_info, roeam_set_tile_config,
                    roeam_autotune, roeam_flux_residual_noalloc, EXPORTS, LIB_PATH, ROEAM_NORM_L2, ROEAM_NORM_LINF)
