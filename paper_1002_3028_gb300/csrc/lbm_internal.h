// Declarations shared by the C-ABI translation unit and the per-storage-type
// kernel translation units of liblbm.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "lbm.h"
#include "lbm_aa_batch.cuh"

namespace lbm {

// Launchers, one set per storage type (defined in lbm_step_<type>.cu);
// the aa_ ones are for lattices in the AA layout (lbm_aa.cuh).  Each
// returns the cudaError_t of the launch.
#define LBM_DECLARE_LAUNCHERS(TAG, C)                                                                  \
    cudaError_t launch_run_##TAG(const StepParams<C> &p, const RunCtl &ctl, int warps_per_cta, int ctas,  \
                                 int nv, cudaStream_t s);                                              \
    cudaError_t occupancy_run_##TAG(int warps_per_cta, int nv, int *ctas_per_sm);                      \
    cudaError_t launch_batch_##TAG(const TileRef *tiles, int ntiles, StepParams<C> *lattices, int nlat,     \
                                   const RunCtl &ctl, int warps_per_cta, int ctas, int far, int nv,   \
                                   cudaStream_t s);                                                    \
    cudaError_t occupancy_batch_##TAG(int warps_per_cta, int nv, int *ctas_per_sm);                    \
    cudaError_t launch_fields_##TAG(const StepParams<C> &p, void *out, int out_f64, cudaStream_t s);   \
    cudaError_t launch_fill_##TAG(const StepParams<C> &p, cudaStream_t s);                             \
    cudaError_t launch_diag_##TAG(const StepParams<C> &p, int have_prev, double *partials, int nblocks,     \
                                  double *out, cudaStream_t s);                                        \
    cudaError_t launch_state_in_##TAG(void *buf, const double *f, const double *g, int nx, int nr,     \
                                      int pitch, int64_t plane, double rho0, double T0, cudaStream_t s); \
    cudaError_t launch_state_out_##TAG(const void *buf, double *f, double *g, int nx, int nr, int pitch, \
                                       int64_t plane, double rho0, double T0, cudaStream_t s);            \
    cudaError_t launch_aa_run_##TAG(const StepParams<C> &p, const RunCtl &ctl, int warps_per_cta, int ctas, \
                                    cudaStream_t s);                                                    \
    cudaError_t occupancy_aa_run_##TAG(int warps_per_cta, int *ctas_per_sm);                           \
    cudaError_t launch_aa_batch_##TAG(const TileRef *tiles, int ntiles, StepParams<C> *lattices, int nlat,  \
                                      const RunCtl &ctl, int warps_per_cta, int ctas, cudaStream_t s); \
    cudaError_t occupancy_aa_batch_##TAG(int warps_per_cta, int *ctas_per_sm);                         \
    cudaError_t launch_aa_fill_##TAG(const StepParams<C> &p, cudaStream_t s);                          \
    cudaError_t launch_aa_state_in_##TAG(void *buf, const double *f, const double *g, int nx, int nr,  \
                                         int pitch, int64_t plane, double rho0, double T0, cudaStream_t s); \
    cudaError_t launch_aa_state_out_##TAG(const void *buf, int phase, double *f, double *g, int nx, int nr, \
                                          int pitch, int64_t plane, double rho0, double T0, cudaStream_t s);

// the two-buffer launchers only (moment-split storage has no AA layout)
#define LBM_DECLARE_AB_LAUNCHERS(TAG, C)                                                               \
    cudaError_t launch_run_##TAG(const StepParams<C> &p, const RunCtl &ctl, int warps_per_cta, int ctas,  \
                                 int nv, cudaStream_t s);                                              \
    cudaError_t occupancy_run_##TAG(int warps_per_cta, int nv, int *ctas_per_sm);                      \
    cudaError_t launch_batch_##TAG(const TileRef *tiles, int ntiles, StepParams<C> *lattices, int nlat,     \
                                   const RunCtl &ctl, int warps_per_cta, int ctas, int far, int nv,   \
                                   cudaStream_t s);                                                    \
    cudaError_t occupancy_batch_##TAG(int warps_per_cta, int nv, int *ctas_per_sm);                    \
    cudaError_t launch_fields_##TAG(const StepParams<C> &p, void *out, int out_f64, cudaStream_t s);   \
    cudaError_t launch_fill_##TAG(const StepParams<C> &p, cudaStream_t s);                             \
    cudaError_t launch_diag_##TAG(const StepParams<C> &p, int have_prev, double *partials, int nblocks,     \
                                  double *out, cudaStream_t s);                                        \
    cudaError_t launch_state_in_##TAG(void *buf, const double *f, const double *g, int nx, int nr,     \
                                      int pitch, int64_t plane, double rho0, double T0, cudaStream_t s); \
    cudaError_t launch_state_out_##TAG(const void *buf, double *f, double *g, int nx, int nr, int pitch, \
                                       int64_t plane, double rho0, double T0, cudaStream_t s);

constexpr int DIAG_MAX_BLOCKS = 1024;  // partial-sum blocks of the diagnostics reduction

LBM_DECLARE_LAUNCHERS(f64, double)
LBM_DECLARE_LAUNCHERS(f32, float)
LBM_DECLARE_LAUNCHERS(f16, float)
LBM_DECLARE_LAUNCHERS(bf16, float)
LBM_DECLARE_AB_LAUNCHERS(f16s, float)
LBM_DECLARE_AB_LAUNCHERS(bf16s, float)

#undef LBM_DECLARE_LAUNCHERS
#undef LBM_DECLARE_AB_LAUNCHERS

// Read-only view of a lattice handle for entry points defined outside
// lbm_api.cu (parameters of both arithmetic types, current device, whether
// the other buffer holds the previous step).
struct LatticeView {
    int storage, device, prev_valid, nx, nr;
    StepParams<double> pd;
    StepParams<float> pf;
};
int lattice_view(const lbm_lattice *h, LatticeView *out);
// orders stream s after the lattice's set-up / records the call's work on s
// as the lattice's last use (returns rc, or an error of the record)
int lattice_enter(const lbm_lattice *h, cudaStream_t s);
int lattice_leave(lbm_lattice *h, cudaStream_t s, int rc);
int api_fail(int code, const char *msg);                       // sets lbm_last_error
int diag_finish(const double *v, int have_prev, lbm_diag *out); // fills lbm_diag from folded slots

}  // namespace lbm
