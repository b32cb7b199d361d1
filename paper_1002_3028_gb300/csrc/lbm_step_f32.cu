// Step, field and state kernels for f32 population storage.
#define LBM_TAG f32
#define LBM_S float
#define LBM_C float
#include "lbm_step_inst.cuh"
