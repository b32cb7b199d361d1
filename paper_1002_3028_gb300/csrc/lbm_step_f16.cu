// Step, field and state kernels for f16 population storage.
#define LBM_TAG f16
#define LBM_S __half
#define LBM_C float
#define LBM_MAX_NV 2  // widest strip: 32 LBM_MAX_NV columns
#include "lbm_step_inst.cuh"
