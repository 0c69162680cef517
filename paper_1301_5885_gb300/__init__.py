"""GB300 direct-sum boundary-integral linear Poisson-Boltzmann solver.

The numerical work lives in libgabipb.so (hand-written CUDA for sm_103a); this
package is its ctypes binding and the build step.  See include/pb.h for the C ABI.
"""
from ._ffi import (PB_ERR_ADMIT, PB_ERR_ARG, PB_ERR_BADMESH, PB_ERR_CUDA, PB_ERR_NAN,  # noqa: F401
                   PB_ERR_NOCONV, PB_ERR_OOM, PB_ERR_TIMEOUT, PB_FLOAT2, PB_FP32PAIR, PB_FP64, PB_OK, SIGNATURES,
                   Context, PBError, Server, SolveInfo, lib, library_path, pb_batch_clear_tuning, pb_batch_force_shape, pb_batch_set_streams, pb_batch_set_tuning,
                   pb_batch_shapes, pb_batch_solve, pb_create, pb_destroy, pb_energy,
                   pb_energy_of, pb_get_info, pb_kernel_launches, pb_last_error, pb_matvec, pb_matvec_f32_static, pb_matvec_rows,
                   pb_matvec_autotune, pb_matvec_configure, pb_matvec_configure_fp64, pb_matvec_get_config, pb_profile_enable,
                   pb_profile_read, pb_release_cached_memory, pb_scratch_plan, pb_set_bands, pb_set_charges,
                   pb_set_scratch_limit, pb_shard_rows, pb_sym_band_plan,
                   pb_shard_unpack_host, pb_solve_sharded,
                   pb_solve, pb_source, pb_status_string)
from . import build as build_module  # noqa: F401
