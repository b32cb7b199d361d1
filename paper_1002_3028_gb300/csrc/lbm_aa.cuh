// The fused step in the AA layout: one population buffer, updated in place
// (the in-place "AA" access pattern of Bailey, Myre, Walsh, Lilja and
// Wilson, ICPP 2009), for the same update as the two-buffer step kernel
// (Eqs. 1-5, Section 2.3, the boundary rules).
//
// Layout.  The buffer has the 13 padded planes of the two-buffer layout.
// Every stored value is addressed as "population q arriving at node y",
// slot_P(q, y), in one of two representations P:
//   P = 0: cell(opp(q), y - e_q), the post-collision value of the node it
//          leaves, kept there in the plane of the opposite velocity;
//   P = 1: cell(q, y), the value already streamed to y.
// A step on a state in representation P reads slot_P(q, x) for every node
// x and every q (the populations streamed into x) and writes the
// post-collision population q of x to slot_{1-P}(q, x + e_q).  For P = 0
// both are the cells (x + e_q', q') over all q'; for P = 1 both are the 13
// cells of x: each node overwrites exactly what it read, and no two nodes
// share a cell.  The boundary value the rules give a ghost g for plane q
// (ghost_rules) goes to slot_{1-P}(q, g + e_q): a ghost cell for P = 0, for
// P = 1 a cell of the lattice node that will read it, which no node reads
// or writes in that step.  The post-collision value of node x is thus
// always slot_P(q, x + e_q), inside the lattice or in the ghost ring.
//
// Same-time moments.  The sources of Eq. 1 take central differences of the
// moments of neighbouring nodes at the same time level, formed from their
// streamed populations, which their own tiles overwrite in the same step.
// So a step is two passes over the warp tiles: pass A forms every node's
// Eq. 2 moments and stores them in 4 planes (rho - rho0, rho u_x, rho u_r,
// T - T0; the arithmetic type, padded like a population plane); pass B
// reads the streamed populations again, takes the moments beside the tile
// from those planes, collides and writes in place.  The moment planes also
// give the diagnostics the previous step's moments.
//
// Schedule.  Both passes of all steps run in one persistent launch.  Job u
// of the work counter is pass A of work item u / 2 (u even) or pass B of
// work item (u - 1) / 2 - L (u odd), items in step-major order: B trails A
// by the lag L, so the populations A loaded are still in L2 when B reads
// them.  A(k, i) waits for B(k - 1, j) of the items j around i (they wrote
// what A reads, and read the moments A overwrites).  B(k, i) waits for
// A(k, j) of the items around i and of i itself (the moments it reads, and
// A(k, i) must have read what B overwrites).  Item indices of neighbours
// differ by at most D (one band of items, plus one, or the wrap for
// periodic ends), so every job waited on precedes the waiting one in the
// counter order when D <= L <= items - 1 - D.  The host picks L there, or
// runs one step per launch (L = items) on lattices too small for that.
#pragma once

#include "lbm_kernels.cuh"

namespace lbm {

// element offset of slot_P(q, (i, j))
template <int P, class C>
__device__ __forceinline__ int64_t aa_slot(const StepParams<C> &p, int q, int i, int j)
{
    return P ? cell(p, q, i, j) : cell(p, opp_plane(q), i - qex(q), j - qey(q));
}

// Edge node (i, j), whose post-collision values are already stored in
// representation P, writes the boundary values the rules take from it.
template <class S, class C, int P>
__device__ __noinline__ void aa_write_ghosts(const StepParams<C> &p, S *buf, int i, int j, int64_t t)
{
    C fo[9], go[4];
#pragma unroll
    for (int k = 0; k < 9; ++k)
        fo[k] = load_as_shared<S, C>(buf + aa_slot<P>(p, k, i + ex9(k), j + ey9(k)));  // plain load: this thread stored it
#pragma unroll
    for (int k = 0; k < 4; ++k)
        go[k] = load_as_shared<S, C>(buf + aa_slot<P>(p, 9 + k, i + ex4(k), j + ey4(k)));
    ghost_rules<C>(p, fo, go, i, j, t, [&](int q, int ci, int cj, C v) {
        buf[aa_slot<P>(p, q, ci + qex(q), cj + qey(q))] = store_as<S, C>(v);
    });
}

// ---- staging ---------------------------------------------------------------------------
// The chunks one lane copies for every row of a tile: each plane's own
// 32 NV columns, and for P = 0 the 16-byte halo chunk on the side each of
// the eight axially moving populations streams from (f1, f5, f8, g0 from
// column x - 1; f3, f6, f7, g2 from x + 1).  Staged population q of node
// column c sits at window element c + H - e_qx (P = 0) or c + H (P = 1),
// as in the two-buffer staging.
template <class S, int NV, int P>
struct AACopyPlan {
    using Wn = Win<S, NV>;
    static constexpr int OPP = 32 * NV / Wn::E;
    static constexpr int OWN = 13 * OPP;
    static constexpr int TOTAL = OWN + (P ? 0 : 8);
    static constexpr int PER_LANE = (TOTAL + 31) / 32;
    static_assert(32 % OPP == 0, "own chunks of a plane must tile a warp's lanes");
    static_assert(32 * (PER_LANE - 1) <= OWN, "only the last copy of a lane may be a halo chunk");
    int goff[PER_LANE];
    int sbase;
    int slast;
};

// population of halo chunk h: left halos for h < 4, right halos for h >= 4
__device__ __forceinline__ int aa_halo_pop(int h)
{
    constexpr unsigned packed = 1u | (5u << 4) | (8u << 8) | (9u << 12) | (3u << 16) | (6u << 20) | (7u << 24) |
                                (11u << 28);
    return (int)((packed >> (4 * h)) & 15u);
}

template <class S, int NV, int P, class C>
__device__ __forceinline__ AACopyPlan<S, NV, P> aa_copy_plan(const StepParams<C> &p, int x0, int lane)
{
    using Wn = Win<S, NV>;
    using CP = AACopyPlan<S, NV, P>;
    CP cp;
#pragma unroll
    for (int m = 0; m < CP::PER_LANE; ++m) {
        const int t = min(lane + 32 * m, CP::TOTAL - 1);
        int q, c;
        if (t < CP::OWN) {
            q = t / CP::OPP;
            c = 1 + t % CP::OPP;
        } else {
            const int h = t - CP::OWN;
            q = aa_halo_pop(h);
            c = h < 4 ? 0 : Wn::CH - 1;
        }
        const int plane = P ? q : opp_plane(q);
        const int dy = P ? 0 : -qey(q);
        cp.goff[m] = plane * (int)p.plane + dy * p.pitch + (x0 - Wn::H + c * Wn::E + PAD_COLS);
        if (m == CP::PER_LANE - 1)
            cp.slast = q * Wn::W + c * Wn::E;
    }
    cp.sbase = (lane / CP::OPP) * Wn::W + (1 + lane % CP::OPP) * Wn::E;
    return cp;
}

template <class S, int NV, class C, int P>
__device__ __forceinline__ void aa_stage_pops(const S *stage, int lane, Vec<C, NV> (&f)[9], Vec<C, NV> (&g)[4])
{
#pragma unroll
    for (int c = 0; c < NV; ++c) {
#pragma unroll
        for (int k = 0; k < 9; ++k)
            f[k].set(c, sget<S, NV, C>(stage, k, P ? 0 : ex9(k), lane + 32 * c));
#pragma unroll
        for (int k = 0; k < 4; ++k)
            g[k].set(c, sget<S, NV, C>(stage, 9 + k, P ? 0 : ex4(k), lane + 32 * c));
    }
}

// moments of row j of the strip from the moment planes (the density is not needed)
template <int NV, class C>
__device__ __forceinline__ Mom<Vec<C, NV>> load_mom_row(const StepParams<C> &p, int x0, int lane, int j)
{
    Mom<Vec<C, NV>> m;
    const int row = (j + 1) * p.pitch + PAD_COLS + x0 + lane;
    const unsigned pl = (unsigned)p.plane;
#pragma unroll
    for (int c = 0; c < NV; ++c) {
        const unsigned o = (unsigned)(row + 32 * c);
        m.drho.set(c, C(0));
        m.jx.set(c, __ldcg(p.mom + pl + o));
        m.jr.set(c, __ldcg(p.mom + 2 * pl + o));
        m.dT.set(c, __ldcg(p.mom + 3 * pl + o));
    }
    return m;
}

// ---- pass A: moments of a warp tile ----------------------------------------------------
template <class S, int NV, class C, int P>
__device__ __forceinline__ void aa_moments_tile(const StepParams<C> &p, const S *__restrict__ buf, S *wsm, int tile,
                                                int lane)
{
    using Wn = Win<S, NV>;
    using V = Vec<C, NV>;
    constexpr int NSTAGE = Stages<NV>::value;
    constexpr int D = NSTAGE - 1;  // only the row being read occupies a stage
    const int x0 = (tile % p.nstrips) * 32 * NV;
    const int j0 = (tile / p.nstrips) * p.band;
    const int nrows = min(j0 + p.band, p.nr) - j0;
    const AACopyPlan<S, NV, P> plan = aa_copy_plan<S, NV, P, C>(p, x0, lane);
#pragma unroll
    for (int t = 0; t < D; ++t) {
        if (t < nrows)
            issue_row<S, NV, C>(p, buf, wsm + t * Wn::STAGE, plan, j0 + t, lane);
        cp_async_commit();
    }
    const unsigned pl = (unsigned)p.plane;
#pragma unroll 1
    for (int idx = 0; idx < nrows; ++idx) {
        __syncwarp();  // every lane is done with the stage refilled next (it held row idx - 1)
        if (idx + D < nrows)
            issue_row<S, NV, C>(p, buf, wsm + ((idx + D) % NSTAGE) * Wn::STAGE, plan, j0 + idx + D, lane);
        cp_async_commit();
        cp_async_wait<D>();
        __syncwarp();
        V f[9], g[4];
        aa_stage_pops<S, NV, C, P>(wsm + (idx % NSTAGE) * Wn::STAGE, lane, f, g);
        const Mom<V> m = moments<V>(f, g);
        const int row = (j0 + idx + 1) * p.pitch + PAD_COLS + x0 + lane;
#pragma unroll
        for (int c = 0; c < NV; ++c) {
            if (x0 + lane + 32 * c < p.nx) {
                const unsigned o = (unsigned)(row + 32 * c);
                p.mom[o] = m.drho[c];
                p.mom[pl + o] = m.jx[c];
                p.mom[2 * pl + o] = m.jr[c];
                p.mom[3 * pl + o] = m.dT[c];
            }
        }
    }
    cp_async_wait<0>();
    __syncwarp();
}

// ---- pass B: collide a warp tile in place ----------------------------------------------
// collide row j of the strip from its stage and write it (and its boundary values)
template <class S, int NV, class C, int P>
__device__ __forceinline__ void aa_collide_row(const StepParams<C> &p, S *__restrict__ buf, const S *st, int x0,
                                               int lane, int j, int64_t t, const Mom<Vec<C, NV>> &mp,
                                               const Mom<Vec<C, NV>> &mc, const Mom<Vec<C, NV>> &mn,
                                               const float2 *stab)
{
    using V = Vec<C, NV>;
    const C *mjr = p.mom + 2 * (int64_t)p.plane + (int64_t)(j + 1) * p.pitch + PAD_COLS;  // rho u_r of row j
    // rho u_r beside the strip from the moment planes: lanes 0..15 read the
    // left neighbour column, 16..31 the right one (in the padded row)
    const C beside = __ldcg(mjr + (lane < 16 ? x0 - 1 : x0 + 32 * NV));
    V left, right;
#pragma unroll
    for (int c = 0; c < NV; ++c) {
        const C up = __shfl_up_sync(0xffffffffu, mc.jr[c], 1);
        const C dn = __shfl_down_sync(0xffffffffu, mc.jr[c], 1);
        const C prev_last = __shfl_sync(0xffffffffu, mc.jr[(c + NV - 1) % NV], 31);
        const C next_first = __shfl_sync(0xffffffffu, mc.jr[(c + 1) % NV], 0);
        C l = up, r = dn;
        if (lane == 0)
            l = (c == 0) ? beside : prev_last;
        if (lane == 31)
            r = (c == NV - 1) ? beside : next_first;
        const int i = x0 + lane + 32 * c;
        if (i == 0)  // ghost moment beyond the inlet end (the periodic image: column nx - 1)
            l = p.bc_in == IN_INLET ? C(0) : __ldcg(mjr + (p.nx - 1));
        if (i == p.nx - 1)  // beyond the outlet end
            r = p.bc_out == OUT_OUTFLOW ? mc.jr[c] : (p.bc_out == OUT_WALL ? -mc.jr[c] : __ldcg(mjr));
        left.set(c, l);
        right.set(c, r);
    }
    if (x0 + lane >= p.nx)
        return;  // no active node in this lane
    V f[9], g[4], fo[9], go[4];
    aa_stage_pops<S, NV, C, P>(st, lane, f, g);
    const C inv_r = C(1) / (p.r0 + C(j) + C(0.5));
    collide<C, V>(p, f, g, mc, inv_r, C(0.5) * (mn.jx - mp.jx), C(0.5) * (mn.jr - mp.jr), C(0.5) * (right - left),
                  C(0.5) * (mn.dT - mp.dT), fo, go, stab);
    const int pl = (int)p.plane, pitch = p.pitch;
    // post-collision population q of node x goes to slot_{1-P}(q, x + e_q)
    auto dest = [&](int q) -> int { return P ? opp_plane(q) * pl : q * pl + qey(q) * pitch + qex(q); };
#pragma unroll
    for (int c = 0; c < NV; ++c) {
        const int i = x0 + lane + 32 * c;
        if (i < p.nx) {
            const int o = (j + 1) * pitch + i + PAD_COLS;
#pragma unroll
            for (int k = 0; k < 9; ++k)
                buf[o + dest(k)] = store_as<S, C>(fo[k][c]);
#pragma unroll
            for (int k = 0; k < 4; ++k)
                buf[o + dest(9 + k)] = store_as<S, C>(go[k][c]);
            if (i == 0 || i == p.nx - 1 || j == 0 || j == p.nr - 1)
                aa_write_ghosts<S, C, 1 - P>(p, buf, i, j, t + 1);
        }
    }
}

// Rows j0..j1-1 are staged in order; row j is collided once the moments of
// row j + 1 exist.  The moments above and below the tile come from the
// moment planes (or the boundary's ghost moments at the lattice edges).
template <class S, int NV, class C, int P>
__device__ __forceinline__ void aa_collide_tile(const StepParams<C> &p, S *__restrict__ buf, S *wsm, int tile,
                                                int lane, int64_t t, const float2 *stab)
{
    using Wn = Win<S, NV>;
    using V = Vec<C, NV>;
    constexpr int NSTAGE = Stages<NV>::value;
    constexpr int D = NSTAGE - 2;  // two stages are read at once
    const int x0 = (tile % p.nstrips) * 32 * NV;
    const int j0 = (tile / p.nstrips) * p.band;
    const int j1 = min(j0 + p.band, p.nr);
    const int nrows = j1 - j0;
    const AACopyPlan<S, NV, P> plan = aa_copy_plan<S, NV, P, C>(p, x0, lane);
#pragma unroll
    for (int r = 0; r < D; ++r) {
        if (r < nrows)
            issue_row<S, NV, C>(p, buf, wsm + r * Wn::STAGE, plan, j0 + r, lane);
        cp_async_commit();
    }
    Mom<V> mp, mc;
#pragma unroll 1
    for (int idx = 0; idx < nrows; ++idx) {
        __syncwarp();  // every lane is done with the stage refilled next (it held row idx - 2)
        if (idx + D < nrows)
            issue_row<S, NV, C>(p, buf, wsm + ((idx + D) % NSTAGE) * Wn::STAGE, plan, j0 + idx + D, lane);
        cp_async_commit();
        cp_async_wait<D>();
        __syncwarp();
        V f[9], g[4];
        aa_stage_pops<S, NV, C, P>(wsm + (idx % NSTAGE) * Wn::STAGE, lane, f, g);
        const Mom<V> mr = moments<V>(f, g);
        if (idx == 0) {
            mp = j0 == 0 ? ghost_bottom<C, V>(p, mr) : load_mom_row<NV, C>(p, x0, lane, j0 - 1);
        } else {
            aa_collide_row<S, NV, C, P>(p, buf, wsm + ((idx - 1) % NSTAGE) * Wn::STAGE, x0, lane, j0 + idx - 1, t, mp,
                                        mc, mr, stab);
            mp = mc;
        }
        mc = mr;
    }
    const Mom<V> mn = j1 == p.nr ? ghost_top<C, V>(p, mc) : load_mom_row<NV, C>(p, x0, lane, j1);
    aa_collide_row<S, NV, C, P>(p, buf, wsm + ((nrows - 1) % NSTAGE) * Wn::STAGE, x0, lane, j1 - 1, t, mp, mc, mn,
                                stab);
    cp_async_wait<0>();
    __syncwarp();
}

// ---- the persistent launch ---------------------------------------------------------------
// ctl.flags holds the pass A counters of the items, then those of pass B
// (32 per finished sub-step each); `lag` is L of the header comment.
template <class S, class C>
__global__ void __launch_bounds__(256) aa_run_kernel(const __grid_constant__ StepParams<C> p, const RunCtl ctl,
                                                     const int lag)
{
    constexpr int NV = NodesPerLane<C>::value;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    S *wsm = reinterpret_cast<S *>(smem_raw) + (size_t)warp * Stages<NV>::value * Win<S, NV>::STAGE;
    const float2 *stab = nullptr;
    if constexpr (UseSmemTable<S, C>::value) {
        if (p.ntab > 1 && p.ntab <= SMEM_TAB) {
            float2 *tab = reinterpret_cast<float2 *>(smem_raw + (blockDim.x >> 5) * step_smem_per_warp<S, C>());
            load_smem_table(p, tab);
            __syncthreads();
            stab = tab;
        }
    }
    S *buf = static_cast<S *>(const_cast<void *>(p.src));
    const int cols = item_cols(p.nstrips, ctl.group);
    const unsigned items = (unsigned)cols * (unsigned)((p.nr + p.band - 1) / p.band);
    const unsigned total = (unsigned)ctl.nsteps * items;
    const unsigned jobs = 2u * (total + (unsigned)lag);
    unsigned *flagsA = ctl.flags, *flagsB = ctl.flags + items;
    unsigned n = 0;
    if (lane == 0)
        n = atomicAdd(ctl.counter, 1u);
    n = __shfl_sync(0xffffffffu, n, 0);
    while (n < jobs) {
        unsigned next = 0;
        if (lane == 0)
            next = atomicAdd(ctl.counter, 1u);
        const bool passB = (n & 1u) != 0;
        const int64_t a = passB ? (int64_t)((n - 1u) >> 1) - lag : (int64_t)(n >> 1);
        if (a >= 0 && a < (int64_t)total) {
            const int k = (int)(a / items);
            const int item = (int)(a - (int64_t)k * items);
            const int b = item / cols, g = item - b * cols;
            const int P = (p.phase + k) & 1;
            bool ok = true;
            if (!passB) {
                if (k > 0)
                    ok = wait_neighbours<C>(p, flagsB, cols, 1, ctl.wrap != 0, b, g, k, ctl.spin_limit);
            } else {
                ok = wait_neighbours<C>(p, flagsA, cols, 1, ctl.wrap != 0, b, g, k + 1, ctl.spin_limit);
            }
            if (!ok) {
                if (lane == 0)
                    atomicOr(p.status, STATUS_TIMEOUT);
                break;  // whole warp
            }
            const int s1 = min((g + 1) * ctl.group, p.nstrips);
            for (int s = g * ctl.group; s < s1; ++s) {
                const int tile = b * p.nstrips + s;
                if (!passB) {
                    if (P)
                        aa_moments_tile<S, NV, C, 1>(p, buf, wsm, tile, lane);
                    else
                        aa_moments_tile<S, NV, C, 0>(p, buf, wsm, tile, lane);
                } else {
                    if (P)
                        aa_collide_tile<S, NV, C, 1>(p, buf, wsm, tile, lane, p.step + k, stab);
                    else
                        aa_collide_tile<S, NV, C, 0>(p, buf, wsm, tile, lane, p.step + k, stab);
                }
            }
            red_release_add((passB ? flagsB : flagsA) + item, 1u);
        }
        n = __shfl_sync(0xffffffffu, next, 0);
    }
}

// ---- state I/O and boundary values of a stored state ------------------------------------
// ghosts of the stored state in its representation (after it was set or the inlet changed)
template <class S, class C>
__global__ void aa_fill_ghosts_kernel(const __grid_constant__ StepParams<C> p)
{
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= (int64_t)p.nx * p.nr)
        return;
    const int i = (int)(n % p.nx), j = (int)(n / p.nx);
    if (!(i == 0 || i == p.nx - 1 || j == 0 || j == p.nr - 1))
        return;
    S *buf = static_cast<S *>(const_cast<void *>(p.src));
    if (p.phase)
        aa_write_ghosts<S, C, 1>(p, buf, i, j, p.step);
    else
        aa_write_ghosts<S, C, 0>(p, buf, i, j, p.step);
}

// post-collision population q of node (i, j) in a stored AA state of representation phase
__host__ __device__ __forceinline__ int64_t aa_post_cell(int phase, int q, int i, int j, int pitch, int64_t plane)
{
    const int pq = phase ? q : opp_plane(q);
    const int ci = phase ? i + qex(q) : i, cj = phase ? j + qey(q) : j;
    return (int64_t)pq * plane + (int64_t)(cj + 1) * pitch + (ci + PAD_COLS);
}

// absolute FP64 [q][j][i] <-> the stored deviations (written in representation 0)
template <class S>
__global__ void aa_state_in_kernel(S *buf, const double *f, const double *g, int nx, int nr, int pitch, int64_t plane,
                                   double rho0, double T0)
{
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t N = (int64_t)nx * nr;
    if (n >= 13 * N)
        return;
    const int q = (int)(n / N);
    const int64_t c = n % N;
    const int i = (int)(c % nx), j = (int)(c / nx);
    const double v = q < 9 ? f[(int64_t)q * N + c] - w9<double>(q) * rho0 : g[(int64_t)(q - 9) * N + c] - 0.25 * T0;
    buf[aa_post_cell(0, q, i, j, pitch, plane)] = store_as<S, compute_t<S>>(compute_t<S>(v));
}

template <class S>
__global__ void aa_state_out_kernel(const S *buf, int phase, double *f, double *g, int nx, int nr, int pitch,
                                    int64_t plane, double rho0, double T0)
{
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t N = (int64_t)nx * nr;
    if (n >= 13 * N)
        return;
    const int q = (int)(n / N);
    const int64_t c = n % N;
    const int i = (int)(c % nx), j = (int)(c / nx);
    const double v = (double)load_as<S, compute_t<S>>(buf + aa_post_cell(phase, q, i, j, pitch, plane));
    if (q < 9)
        f[(int64_t)q * N + c] = v + w9<double>(q) * rho0;
    else
        g[(int64_t)(q - 9) * N + c] = v + 0.25 * T0;
}

}  // namespace lbm
