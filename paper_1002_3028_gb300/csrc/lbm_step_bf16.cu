// Step, field and state kernels for bf16 population storage.
#define LBM_TAG bf16
#define LBM_S __nv_bfloat16
#define LBM_C float
#define LBM_MAX_NV 2  // widest strip: 32 LBM_MAX_NV columns
#include "lbm_step_inst.cuh"
