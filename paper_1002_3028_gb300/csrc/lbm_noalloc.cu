// lbm_diagnostics_noalloc: the FP64 diagnostics of a lattice computed with a
// fixed scratch array that lives in this library's device image, so that
// the call allocates no device memory and touches none beyond the lattice
// and a fixed array.  Declared in include/lbm.h.
#include <cuda_runtime.h>

#include <mutex>

#include "lbm.h"
#include "lbm_internal.h"

namespace lbm {
namespace {

constexpr int kMaxRows = 16384;                          // largest nr this entry point accepts
constexpr int kSlots = (kMaxRows + 1) * DIAG_SLOTS;      // one partial per row, then the folded result
constexpr int kMaxDevices = 64;

// Scratch of every call on a device: the per-row partial sums and the
// folded result.  It is held by every GPU that loads the library until the
// process exits.  Each call overwrites every slot it reads, so nothing has
// to start at zero; calls that overlap on the GPU share it and race.
static __device__ __align__(256) double g_scratch[kSlots];

std::mutex g_mutex;
double *g_scratch_ptr[kMaxDevices] = {};

// Device address of g_scratch on the current device.  It is looked up again
// on every call whose stream is not capturing (a cheap query that allocates
// nothing, so an address cached before a cudaDeviceReset is never reused);
// a call made while its stream captures a graph takes the address of the
// last lookup on the device, so the first call on a device must come before
// any stream capture.
int scratch_on(int device, cudaStream_t s, double **ptr)
{
    if (device < 0 || device >= kMaxDevices)
        return api_fail(LBM_ERR_INVALID_ARG, "device index out of range for the fixed scratch table");
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) {
        cudaGetLastError();
        return api_fail(LBM_ERR_CUDA, "querying the stream's capture status failed");
    }
    std::lock_guard<std::mutex> lock(g_mutex);
    if (cap == cudaStreamCaptureStatusNone || !g_scratch_ptr[device]) {
        if (cap != cudaStreamCaptureStatusNone)
            return api_fail(LBM_ERR_INVALID_ARG,
                            "the first lbm_diagnostics_noalloc call on a device must come before any stream capture");
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return api_fail(LBM_ERR_CUDA, "cudaGetSymbolAddress of the fixed diagnostics scratch failed");
        }
        g_scratch_ptr[device] = static_cast<double *>(p);
    }
    *ptr = g_scratch_ptr[device];
    return LBM_OK;
}

// One CTA per lattice row: the row's nodes (populations streamed from the
// current state, and from the previous one in the other buffer) reduced in FP64 into the
// row's DIAG_SLOTS partial slots; same per-node quantities as the
// lattice-scratch diagnostics.
template <class S, class C>
__global__ void __launch_bounds__(DIAG_THREADS) diag_rows_kernel(const __grid_constant__ StepParams<C> p,
                                                                 int have_prev, double *partials)
{
    double v[DIAG_SLOTS] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    const int j = blockIdx.x;
    for (int i = threadIdx.x; i < p.nx; i += blockDim.x)
        diag_node<S, C>(p, have_prev, i, j, v);
    diag_block_reduce(v);
    if (threadIdx.x == 0)
        for (int k = 0; k < DIAG_SLOTS; ++k)
            partials[(int64_t)j * DIAG_SLOTS + k] = v[k];
}

template <class S, class C>
cudaError_t launch_rows(const StepParams<C> &p, int have_prev, double *scratch, cudaStream_t s)
{
    diag_rows_kernel<S, C><<<p.nr, DIAG_THREADS, 0, s>>>(p, have_prev, scratch);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return e;
    diag_final_kernel<<<1, DIAG_THREADS, 0, s>>>(scratch, p.nr, scratch + (size_t)kMaxRows * DIAG_SLOTS);
    return cudaGetLastError();
}

}  // namespace
}  // namespace lbm

extern "C" int lbm_diagnostics_noalloc(lbm_lattice *h, lbm_diag *out, lbm_stream stream)
{
    using namespace lbm;
    if (!out)
        return api_fail(LBM_ERR_INVALID_ARG, "NULL output");
    LatticeView v;
    int rc = lattice_view(h, &v);
    if (rc)
        return rc;
    if (v.nr > kMaxRows)
        return api_fail(LBM_ERR_INVALID_ARG,
                        "lbm_diagnostics_noalloc handles at most 16384 lattice rows (nr); use lbm_diagnostics");
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev != v.device)
        return api_fail(LBM_ERR_INVALID_ARG, "make the lattice's device current before calling");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    double *scratch = nullptr;
    rc = scratch_on(dev, s, &scratch);
    if (rc)
        return rc;
    rc = lattice_enter(h, s);
    if (rc)
        return rc;
    switch (v.storage) {
    case LBM_F64: e = launch_rows<double, double>(v.pd, v.prev_valid, scratch, s); break;
    case LBM_F32: e = launch_rows<float, float>(v.pf, v.prev_valid, scratch, s); break;
    case LBM_F16: e = launch_rows<__half, float>(v.pf, v.prev_valid, scratch, s); break;
    case LBM_F16S: e = launch_rows<half_s, float>(v.pf, v.prev_valid, scratch, s); break;
    case LBM_BF16S: e = launch_rows<bf16_s, float>(v.pf, v.prev_valid, scratch, s); break;
    default: e = launch_rows<__nv_bfloat16, float>(v.pf, v.prev_valid, scratch, s); break;
    }
    double vals[DIAG_SLOTS];
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(vals, scratch + (size_t)kMaxRows * DIAG_SLOTS, sizeof(vals), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return api_fail(LBM_ERR_CUDA, "lbm_diagnostics_noalloc: a launch or the result copy failed");
    }
    rc = lattice_leave(h, s, LBM_OK);
    if (rc)
        return rc;
    return diag_finish(vals, v.prev_valid, out);
}
