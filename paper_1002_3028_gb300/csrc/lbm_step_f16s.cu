// Step, field and state kernels for FP16 moment-split population storage
// (two-buffer layout only).
#define LBM_TAG f16s
#define LBM_S half_s
#define LBM_C float
#define LBM_SPLIT 1
#define LBM_MAX_NV 2  // widest strip: 32 LBM_MAX_NV columns
#include "lbm_step_inst.cuh"
