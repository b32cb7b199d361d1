// Step, field and state kernels for f64 population storage.
#define LBM_TAG f64
#define LBM_S double
#define LBM_C double
#include "lbm_step_inst.cuh"
