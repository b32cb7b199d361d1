// Batches of AA-pattern lattices: the persistent multi-step launch of a
// table of (lattice, warp tile) entries, with the two-phase work item of
// the single-lattice AA kernel (lbm_aa.cuh).
#pragma once

#include "lbm_aa.cuh"

namespace lbm {

// ---- many AA lattices in one launch -------------------------------------------------------
// A batch of AA-pattern lattices runs like the two-buffer batch
// (batch_run_kernel): a table of (lattice, warp tile) entries, one work item
// per entry in step-major order, each lattice's entries consecutive, each
// warp copying its lattice's parameters to shared memory.  Each item is
// the two-phase item of aa_run_kernel.  ctl.flags holds the entries' step
// counters, then their edge counters.  An item waits on the edges of items
// at most one band of its lattice's tiles plus one away, so the host
// launches at least that many warps plus two for the widest member.
template <class S, class C>
__global__ void __launch_bounds__(256) aa_batch_run_kernel(const TileRef *__restrict__ tiles, int ntiles,
                                                           const StepParams<C> *__restrict__ lattices,
                                                           const RunCtl ctl)
{
    constexpr int NV = NodesPerLane<C>::value;
    constexpr int PW = (int)((sizeof(StepParams<C>) + 15) / 16);  // 16-byte words per parameter block
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int wpc = blockDim.x >> 5;
    StepParams<C> *pw = reinterpret_cast<StepParams<C> *>(smem_raw) + warp;
    S *wsm = reinterpret_cast<S *>(smem_raw + wpc * sizeof(StepParams<C>)) + (size_t)warp * Stages<NV>::value * Win<S, NV>::STAGE;
    static_assert(sizeof(StepParams<C>) % 16 == 0 && PW <= 32, "parameter block copy");
    const unsigned total = (unsigned)ctl.nsteps * (unsigned)ntiles;
    unsigned *done = ctl.flags, *pub = ctl.flags + ntiles;
    unsigned n = 0;
    if (lane == 0)
        n = atomicAdd(ctl.counter, 1u);
    n = __shfl_sync(0xffffffffu, n, 0);
    while (n < total) {
        const int k = (int)(n / (unsigned)ntiles);
        const int idx = (int)(n - (unsigned)k * (unsigned)ntiles);
        const TileRef t = tiles[idx];
        __syncwarp();  // every lane is done with the previous parameter block
        if (lane < PW)
            reinterpret_cast<uint4 *>(pw)[lane] = reinterpret_cast<const uint4 *>(lattices + t.lattice)[lane];
        __syncwarp();
        const StepParams<C> &p = *pw;
        const int b = t.tile / p.nstrips, g = t.tile % p.nstrips;
        const bool wrap = p.bc_in == IN_PERIODIC;
        const int first = idx - t.tile;  // the lattice's first entry
        if (k > 0 && !wait_neighbours<C>(p, done + first, p.nstrips, 1, wrap, b, g, k, ctl.spin_limit)) {
            if (lane == 0)
                atomicOr(p.status, STATUS_TIMEOUT);
            break;  // whole warp
        }
        const int P = (p.phase + k) & 1;
        S *buf = static_cast<S *>(const_cast<void *>(p.src));
        aa_edges_tile<S, NV, C>(p, P, buf, wsm, t.tile, lane);
        red_release_add(pub + idx, 1u);
        if (!wait_edges<C>(p, pub + first, p.nstrips, wrap, b, g, k + 1, ctl.spin_limit)) {
            if (lane == 0)
                atomicOr(p.status, STATUS_TIMEOUT);
            break;
        }
        unsigned next = 0;  // taken only after the wait, as in aa_run_kernel
        if (lane == 0)
            next = atomicAdd(ctl.counter, 1u);
        aa_collide_tile<S, NV, C>(p, P, buf, wsm, t.tile, lane, p.step + k, nullptr);
        red_release_add(done + idx, 1u);
        n = __shfl_sync(0xffffffffu, next, 0);
    }
}

// after an AA batch launch of nsteps steps: every lattice counts the steps
// and, for an odd count, switches representation
template <class C>
__global__ void aa_advance_kernel(StepParams<C> *lattices, int n, int nsteps)
{
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= n)
        return;
    lattices[m].phase ^= nsteps & 1;
    lattices[m].step += nsteps;
}

}  // namespace lbm
