"""GB300-native Roe-AM finite-volume solver (2D and 3D Euler) behind a C ABI.

The compute path is libroeam.so (CUDA, sm_103a): see include/roeam.h (2D) and
include/roeam3.h (3D with passive scalars) for the ABI and `roeam` for its Python binding.
PyTorch, when used, only provides device memory, pinned host buffers and streams.
"""
from .roeam import (Batch, RoeamError, load_library, make_desc, roeam_cell_count, roeam_check,  # noqa: F401
                    roeam_conserved_totals, roeam_create_grid, roeam_destroy_grid, roeam_flux_residual,
                    roeam_get_state, roeam_launch_count, roeam_residual_norm, roeam_rk_step, roeam_set_state,
                    roeam_version, roeam_tile_config_count, roeam_tile_config_info, roeam_set_tile_config,
                    roeam_autotune, roeam_flux_residual_noalloc, EXPORTS, LIB_PATH, ROEAM_NORM_L2, ROEAM_NORM_LINF,
                    Batch3, make_desc3, roeam3_create_grid, roeam3_destroy_grid, roeam3_set_state, roeam3_get_state,
                    roeam3_flux_residual, roeam3_rk_step, roeam3_conserved_totals, roeam3_check, roeam3_launch_count,
                    roeam_rk_stage, roeam_max_rate, roeam_edge_rows, roeam_set_halo, roeam_math_check,
                    roeam_step_host, roeam_set_state_device, roeam_get_state_device, roeam_rk_stage_part,
                    roeam_set_halo_solid, roeam_set_halo_vertices, ROEAM_PART_ALL, ROEAM_PART_INTERIOR,
                    ROEAM_PART_EDGES, roeam_step_host_f32, roeam_set_state_f32, roeam_get_state_f32)
