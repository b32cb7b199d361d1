// Step, field and state kernels for f64 population storage.
#define LBM_TAG f64
#define LBM_S double
#define LBM_C double
#define LBM_MAX_NV 1  // widest strip: 32 LBM_MAX_NV columns
#include "lbm_step_inst.cuh"
