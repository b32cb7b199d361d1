// Step, field and state kernels for f16 population storage.
#define LBM_TAG f16
#define LBM_S __half
#define LBM_C float
#include "lbm_step_inst.cuh"
