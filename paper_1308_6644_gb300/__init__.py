"""GB300-native non-uniform sampled scalar diffraction (NU-ASM / NU-FRE).

The computation lives in the CUDA library ``libnuasm.so`` (C ABI in
``include/nuasm.h``); this package holds its Python binding and the seeded
synthetic workload generators.
"""
from .nuasm import (  # noqa: F401
    NuasmError, Params, Plan, make_params, nuasm_plan, nuasm_plan_lattice, nuasm1_execute, nuasm2_execute,
    nuasm3_execute, nufresnel3_execute, nuasm_rs_direct,
    nufresnel_execute, nuasm_destroy, nuasm_strerror, nuasm_plan_info, nuasm_band,
    nuasm_kernel_shape, nuasm_autotune_tile, nuasm_autotune, nuasm_debug_bounded_wait, nuasm_debug_bounds, nuasm_debug_plan_wait,
    nuasm_debug_fail_alloc, nuasm_debug_live_resources, nuasm_profile_enable, nuasm2_solve_noalloc, nuasm_profile_read, lib, LIB_PATH, STAGES,
    KIND_ASM, KIND_FRESNEL, PREC_F32_F64PHASE, PREC_F64, KERNEL_ES, KERNEL_GAUSSIAN,
    Batch, nuasm_batch_create, nuasm_batch_execute, nuasm_batch_info, nuasm_batch_destroy,
    Server, nuasm_server_create, nuasm_server_submit, nuasm_server_wait, nuasm_server_stats, nuasm_server_destroy,
)
