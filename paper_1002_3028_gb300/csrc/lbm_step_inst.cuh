// Instantiates the kernels and launchers of one storage type.  Included by
// lbm_step_<type>.cu with LBM_TAG, LBM_S (storage) and LBM_C (arithmetic).
#include "lbm_internal.h"

#define LBM_CAT2(a, b) a##b
#define LBM_CAT(a, b) LBM_CAT2(a, b)

namespace lbm {

// strip widths of the two-buffer step and batch kernels: 32 nv columns, nv nodes a lane
// (FP32 arithmetic: 1 or 2; FP64: 1)
template <int NV>
static cudaError_t run_nv(const StepParams<LBM_C> &p, const RunCtl &ctl, int warps_per_cta, int ctas, cudaStream_t s)
{
    const int smem = run_smem<LBM_S, LBM_C, NV>(warps_per_cta);
    if (far_wrap(p.bc_in, p.nx, p.nstrips, 32 * NV))
        step_run_kernel<LBM_S, LBM_C, true, NV><<<ctas, 32 * warps_per_cta, smem, s>>>(p, ctl);
    else
        step_run_kernel<LBM_S, LBM_C, false, NV><<<ctas, 32 * warps_per_cta, smem, s>>>(p, ctl);
    return cudaGetLastError();
}

cudaError_t LBM_CAT(launch_run_, LBM_TAG)(const StepParams<LBM_C> &p, const RunCtl &ctl, int warps_per_cta, int ctas,
                                          int nv, cudaStream_t s)
{
    if (p.ntiles <= 0 || ctl.nsteps <= 0)
        return cudaSuccess;
#if LBM_MAX_NV > 1
    if (nv == 2)
        return run_nv<2>(p, ctl, warps_per_cta, ctas, s);
#endif
    return nv == 1 ? run_nv<1>(p, ctl, warps_per_cta, ctas, s) : cudaErrorInvalidValue;
}

// allows the dynamic shared memory of the widest CTA and reports how many CTAs of
// the given width fit on one SM (the fewer of the two instantiations)
template <int NV>
static cudaError_t occupancy_run_nv(int warps_per_cta, int *ctas_per_sm)
{
    int n[2] = {0, 0};
    for (int far = 0; far < 2; ++far) {
        const void *fn = far ? reinterpret_cast<const void *>(step_run_kernel<LBM_S, LBM_C, true, NV>)
                             : reinterpret_cast<const void *>(step_run_kernel<LBM_S, LBM_C, false, NV>);
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             run_smem<LBM_S, LBM_C, NV>(8));
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n[far], fn, 32 * warps_per_cta,
                                                              run_smem<LBM_S, LBM_C, NV>(warps_per_cta));
        if (e != cudaSuccess)
            return e;
    }
    *ctas_per_sm = n[0] < n[1] ? n[0] : n[1];
    return cudaSuccess;
}

cudaError_t LBM_CAT(occupancy_run_, LBM_TAG)(int warps_per_cta, int nv, int *ctas_per_sm)
{
#if LBM_MAX_NV > 1
    if (nv == 2)
        return occupancy_run_nv<2>(warps_per_cta, ctas_per_sm);
#endif
    return nv == 1 ? occupancy_run_nv<1>(warps_per_cta, ctas_per_sm) : cudaErrorInvalidValue;
}

// nsteps steps of every member lattice in one persistent launch, then the
// device-side advance of the parameter table
template <int NV>
static cudaError_t batch_nv(const TileRef *tiles, int ntiles, StepParams<LBM_C> *lattices, const RunCtl &ctl,
                            int warps_per_cta, int ctas, int far, cudaStream_t s)
{
    const int smem = warps_per_cta * batch_smem_per_warp<LBM_S, LBM_C, NV>();
    if (far)
        batch_run_kernel<LBM_S, LBM_C, true, NV><<<ctas, 32 * warps_per_cta, smem, s>>>(tiles, ntiles, lattices, ctl);
    else
        batch_run_kernel<LBM_S, LBM_C, false, NV><<<ctas, 32 * warps_per_cta, smem, s>>>(tiles, ntiles, lattices, ctl);
    return cudaGetLastError();
}

cudaError_t LBM_CAT(launch_batch_, LBM_TAG)(const TileRef *tiles, int ntiles, StepParams<LBM_C> *lattices, int nlat,
                                            const RunCtl &ctl, int warps_per_cta, int ctas, int far, int nv,
                                            cudaStream_t s)
{
    if (ntiles <= 0 || nlat <= 0 || ctl.nsteps <= 0)
        return cudaSuccess;
    cudaError_t e = cudaErrorInvalidValue;
#if LBM_MAX_NV > 1
    if (nv == 2)
        e = batch_nv<2>(tiles, ntiles, lattices, ctl, warps_per_cta, ctas, far, s);
#endif
    if (nv == 1)
        e = batch_nv<1>(tiles, ntiles, lattices, ctl, warps_per_cta, ctas, far, s);
    if (e != cudaSuccess)
        return e;
    advance_kernel<LBM_C><<<(nlat + 127) / 128, 128, 0, s>>>(lattices, nlat, ctl.nsteps);
    return cudaGetLastError();
}

template <int NV>
static cudaError_t occupancy_batch_nv(int warps_per_cta, int *ctas_per_sm)
{
    int n[2] = {0, 0};
    for (int far = 0; far < 2; ++far) {
        const void *fn = far ? reinterpret_cast<const void *>(batch_run_kernel<LBM_S, LBM_C, true, NV>)
                             : reinterpret_cast<const void *>(batch_run_kernel<LBM_S, LBM_C, false, NV>);
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             8 * batch_smem_per_warp<LBM_S, LBM_C, NV>());
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n[far], fn, 32 * warps_per_cta,
                                                              warps_per_cta * batch_smem_per_warp<LBM_S, LBM_C, NV>());
        if (e != cudaSuccess)
            return e;
    }
    *ctas_per_sm = n[0] < n[1] ? n[0] : n[1];
    return cudaSuccess;
}

cudaError_t LBM_CAT(occupancy_batch_, LBM_TAG)(int warps_per_cta, int nv, int *ctas_per_sm)
{
#if LBM_MAX_NV > 1
    if (nv == 2)
        return occupancy_batch_nv<2>(warps_per_cta, ctas_per_sm);
#endif
    return nv == 1 ? occupancy_batch_nv<1>(warps_per_cta, ctas_per_sm) : cudaErrorInvalidValue;
}

cudaError_t LBM_CAT(launch_fields_, LBM_TAG)(const StepParams<LBM_C> &p, void *out, int out_f64, cudaStream_t s)
{
    const int64_t N = (int64_t)p.nx * p.nr;
    const int threads = 256;
    const int64_t blocks = (N + threads - 1) / threads;
    if (out_f64)
        fields_kernel<LBM_S, LBM_C, double><<<(unsigned)blocks, threads, 0, s>>>(p, static_cast<double *>(out));
    else
        fields_kernel<LBM_S, LBM_C, float><<<(unsigned)blocks, threads, 0, s>>>(p, static_cast<float *>(out));
    return cudaGetLastError();
}

cudaError_t LBM_CAT(launch_fill_, LBM_TAG)(const StepParams<LBM_C> &p, cudaStream_t s)
{
    const int64_t N = (int64_t)p.nx * p.nr;
    const int threads = 256;
    fill_ghosts_kernel<LBM_S, LBM_C><<<(unsigned)((N + threads - 1) / threads), threads, 0, s>>>(p);
    return cudaGetLastError();
}

// FP64 diagnostics: nblocks partial sums into `partials`, folded into out[DIAG_SLOTS]
cudaError_t LBM_CAT(launch_diag_, LBM_TAG)(const StepParams<LBM_C> &p, int have_prev, double *partials, int nblocks,
                                           double *out, cudaStream_t s)
{
    diag_kernel<LBM_S, LBM_C><<<nblocks, DIAG_THREADS, 0, s>>>(p, have_prev, partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return e;
    diag_final_kernel<<<1, DIAG_THREADS, 0, s>>>(partials, nblocks, out);
    return cudaGetLastError();
}

cudaError_t LBM_CAT(launch_state_in_, LBM_TAG)(void *buf, const double *f, const double *g, int nx, int nr, int pitch,
                                               int64_t plane, double rho0, double T0, cudaStream_t s)
{
    const int threads = 256;
#ifdef LBM_SPLIT  // one node per thread: the node's moments first
    const int64_t n = (int64_t)nx * nr;
    split_state_in_kernel<LBM_S><<<(unsigned)((n + threads - 1) / threads), threads, 0, s>>>(
        static_cast<LBM_S *>(buf), f, g, nx, nr, pitch, plane, rho0, T0);
#else
    const int64_t n = 13 * (int64_t)nx * nr;
    state_in_kernel<LBM_S><<<(unsigned)((n + threads - 1) / threads), threads, 0, s>>>(
        static_cast<LBM_S *>(buf), f, g, nx, nr, pitch, plane, rho0, T0);
#endif
    return cudaGetLastError();
}

cudaError_t LBM_CAT(launch_state_out_, LBM_TAG)(const void *buf, double *f, double *g, int nx, int nr, int pitch,
                                                int64_t plane, double rho0, double T0, cudaStream_t s)
{
    const int threads = 256;
#ifdef LBM_SPLIT
    const int64_t n = (int64_t)nx * nr;
    split_state_out_kernel<LBM_S><<<(unsigned)((n + threads - 1) / threads), threads, 0, s>>>(
        static_cast<const LBM_S *>(buf), f, g, nx, nr, pitch, plane, rho0, T0);
#else
    const int64_t n = 13 * (int64_t)nx * nr;
    state_out_kernel<LBM_S><<<(unsigned)((n + threads - 1) / threads), threads, 0, s>>>(
        static_cast<const LBM_S *>(buf), f, g, nx, nr, pitch, plane, rho0, T0);
#endif
    return cudaGetLastError();
}

#ifndef LBM_SPLIT  // moment-split storage has no AA layout
// ---- AA layout ------------------------------------------------------------------------
cudaError_t LBM_CAT(launch_aa_run_, LBM_TAG)(const StepParams<LBM_C> &p, const RunCtl &ctl, int warps_per_cta, int ctas,
                                             cudaStream_t s)
{
    if (p.ntiles <= 0 || ctl.nsteps <= 0)
        return cudaSuccess;
    const int smem = run_smem<LBM_S, LBM_C>(warps_per_cta);
    aa_run_kernel<LBM_S, LBM_C><<<ctas, 32 * warps_per_cta, smem, s>>>(p, ctl);
    return cudaGetLastError();
}

cudaError_t LBM_CAT(occupancy_aa_run_, LBM_TAG)(int warps_per_cta, int *ctas_per_sm)
{
    cudaError_t e = cudaFuncSetAttribute(aa_run_kernel<LBM_S, LBM_C>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         run_smem<LBM_S, LBM_C>(8));
    if (e != cudaSuccess)
        return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, aa_run_kernel<LBM_S, LBM_C>, 32 * warps_per_cta,
                                                         run_smem<LBM_S, LBM_C>(warps_per_cta));
}

cudaError_t LBM_CAT(launch_aa_batch_, LBM_TAG)(const TileRef *tiles, int ntiles, StepParams<LBM_C> *lattices,
                                               int nlat, const RunCtl &ctl, int warps_per_cta, int ctas,
                                               cudaStream_t s)
{
    if (ntiles <= 0 || nlat <= 0 || ctl.nsteps <= 0)
        return cudaSuccess;
    const int smem = warps_per_cta * batch_smem_per_warp<LBM_S, LBM_C>();
    aa_batch_run_kernel<LBM_S, LBM_C><<<ctas, 32 * warps_per_cta, smem, s>>>(tiles, ntiles, lattices, ctl);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return e;
    aa_advance_kernel<LBM_C><<<(nlat + 127) / 128, 128, 0, s>>>(lattices, nlat, ctl.nsteps);
    return cudaGetLastError();
}

cudaError_t LBM_CAT(occupancy_aa_batch_, LBM_TAG)(int warps_per_cta, int *ctas_per_sm)
{
    cudaError_t e = cudaFuncSetAttribute(aa_batch_run_kernel<LBM_S, LBM_C>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         8 * batch_smem_per_warp<LBM_S, LBM_C>());
    if (e != cudaSuccess)
        return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, aa_batch_run_kernel<LBM_S, LBM_C>,
                                                         32 * warps_per_cta,
                                                         warps_per_cta * batch_smem_per_warp<LBM_S, LBM_C>());
}

cudaError_t LBM_CAT(launch_aa_fill_, LBM_TAG)(const StepParams<LBM_C> &p, cudaStream_t s)
{
    const int64_t N = (int64_t)p.nx * p.nr;
    const int threads = 256;
    aa_fill_ghosts_kernel<LBM_S, LBM_C><<<(unsigned)((N + threads - 1) / threads), threads, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t LBM_CAT(launch_aa_state_in_, LBM_TAG)(void *buf, const double *f, const double *g, int nx, int nr,
                                                  int pitch, int64_t plane, double rho0, double T0, cudaStream_t s)
{
    const int64_t n = 13 * (int64_t)nx * nr;
    const int threads = 256;
    aa_state_in_kernel<LBM_S><<<(unsigned)((n + threads - 1) / threads), threads, 0, s>>>(
        static_cast<LBM_S *>(buf), f, g, nx, nr, pitch, plane, rho0, T0);
    return cudaGetLastError();
}

cudaError_t LBM_CAT(launch_aa_state_out_, LBM_TAG)(const void *buf, int phase, double *f, double *g, int nx, int nr,
                                                   int pitch, int64_t plane, double rho0, double T0, cudaStream_t s)
{
    const int64_t n = 13 * (int64_t)nx * nr;
    const int threads = 256;
    aa_state_out_kernel<LBM_S><<<(unsigned)((n + threads - 1) / threads), threads, 0, s>>>(
        static_cast<const LBM_S *>(buf), phase, f, g, nx, nr, pitch, plane, rho0, T0);
    return cudaGetLastError();
}

#endif  // LBM_SPLIT

}  // namespace lbm
