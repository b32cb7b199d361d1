// Step, field and state kernels for BF16 moment-split population storage
// (two-buffer layout only).
#define LBM_TAG bf16s
#define LBM_S bf16_s
#define LBM_C float
#define LBM_SPLIT 1
#include "lbm_step_inst.cuh"
