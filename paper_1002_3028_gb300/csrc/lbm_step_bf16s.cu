// Step, field and state kernels for BF16 moment-split population storage
// (two-buffer layout only).
#define LBM_TAG bf16s
#define LBM_S bf16_s
#define LBM_C float
#define LBM_SPLIT 1
#define LBM_MAX_NV 2  // widest strip: 32 LBM_MAX_NV columns
#include "lbm_step_inst.cuh"
