// Step, field and state kernels for FP16 moment-split population storage
// (two-buffer layout only).
#define LBM_TAG f16s
#define LBM_S half_s
#define LBM_C float
#define LBM_SPLIT 1
#include "lbm_step_inst.cuh"
