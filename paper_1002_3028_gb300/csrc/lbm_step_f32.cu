// Step, field and state kernels for f32 population storage.
#define LBM_TAG f32
#define LBM_S float
#define LBM_C float
#define LBM_MAX_NV 2  // widest strip: 32 LBM_MAX_NV columns
#include "lbm_step_inst.cuh"
