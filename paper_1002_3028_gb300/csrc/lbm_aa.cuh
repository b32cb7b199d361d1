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
// So a warp tile is updated in two phases: phase 1 forms the Eq. 2 moments
// a neighbour tile needs from the tile's streamed populations (rho u_x,
// rho u_r, T - T0 of its bottom and top rows, rho u_r of its first and
// last columns) and publishes them in a small edge area;
// phase 2, once the four neighbour tiles have published theirs, stages the
// tile again (now from L2), collides it with the neighbours' edge moments
// and writes it in place.
//
// Schedule.  All steps run in one persistent launch; warps take work items
// (G adjacent tiles of one band) in step-major order, as the two-buffer
// step does.  An item of step k first waits until the items around it have
// finished step k - 1 (they wrote what it reads and read the edges it
// overwrites), runs phase 1 on its tiles, publishes, waits for the edges
// of its four direct neighbour items of step k, and only then takes its
// next item, then runs phase 2.  Deadlock freedom: take the lowest
// unfinished item x.  Its step k - 1 neighbours precede it, so they are
// done; the neighbours it waits on in step k lie within D items of it (one
// band of items, plus one; the wrap for periodic ends).  A warp holds an
// item it has not started only while it runs phase 2, which never waits.
// With at least D + 2 warps resident, every item up to x + D has been
// taken, so each of them has started (or will, once phase 2 of its warp's
// current item ends), passes its own wait on step k - 1 (earlier items)
// and publishes.  The host makes the items wide enough (G) for the
// resident warps to cover D.
//
// Edge area (arithmetic type C): rows [band][side][rho u_x, rho u_r,
// T - T0][epitch] for side 0 = the band's first row, 1 = its last, sized for
// bands of at least AA_BAND_MIN rows; then columns [strip][side][nr] of
// rho u_r for side 0 = the strip's first column, 1 = its last (nx - 1 in
// the last strip).
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
// as in the two-buffer staging.  P is a run-time value: one copy of the
// tile code serves both representations.
template <class S, int NV>
struct AACopyPlan {
    using Wn = Win<S, NV>;
    static constexpr int OPP = 32 * NV / Wn::E;
    static constexpr int OWN = 13 * OPP;
    static constexpr int TOTAL = OWN + 8;
    static constexpr int PER_LANE = (TOTAL + 31) / 32;
    static_assert(32 % OPP == 0, "own chunks of a plane must tile a warp's lanes");
    static_assert(32 * (PER_LANE - 1) <= OWN, "only the last copy of a lane may be a halo chunk");
    int goff[PER_LANE];
    int sbase;
    int slast;
    int total;  // chunks copied: OWN + 8 for P = 0, OWN for P = 1
};

// population of halo chunk h: left halos for h < 4, right halos for h >= 4
__device__ __forceinline__ int aa_halo_pop(int h)
{
    constexpr unsigned packed = 1u | (5u << 4) | (8u << 8) | (9u << 12) | (3u << 16) | (6u << 20) | (7u << 24) |
                                (11u << 28);
    return (int)((packed >> (4 * h)) & 15u);
}

template <class S, int NV, class C>
__device__ __forceinline__ AACopyPlan<S, NV> aa_copy_plan(const StepParams<C> &p, int P, int x0, int lane)
{
    using Wn = Win<S, NV>;
    using CP = AACopyPlan<S, NV>;
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
    cp.total = P ? CP::OWN : CP::TOTAL;
    return cp;
}

// start the copies of lattice row r into one stage
template <class S, int NV, class C>
__device__ __forceinline__ void aa_issue_row(const StepParams<C> &p, const S *src, S *stage,
                                             const AACopyPlan<S, NV> &cp, int r, int lane)
{
    using CP = AACopyPlan<S, NV>;
    const int row = (r + 1) * p.pitch;
#pragma unroll
    for (int m = 0; m < CP::PER_LANE; ++m) {
        const int so = (m < CP::PER_LANE - 1) ? cp.sbase + (32 * m / CP::OPP) * Win<S, NV>::W : cp.slast;
        if (m < CP::PER_LANE - 1 || lane + 32 * m < cp.total)
            cp_async16(stage + so, src + (unsigned)(row + cp.goff[m]));
    }
}

// the streamed populations of the lane's NV nodes from a stage (sh = 1 for P = 0, 0 for P = 1)
template <class S, int NV, class C>
__device__ __forceinline__ void aa_stage_pops(const S *stage, int lane, int sh, Vec<C, NV> (&f)[9],
                                              Vec<C, NV> (&g)[4])
{
#pragma unroll
    for (int c = 0; c < NV; ++c) {
        const S *col = stage + Win<S, NV>::H + lane + 32 * c;
#pragma unroll
        for (int k = 0; k < 9; ++k)
            f[k].set(c, load_as_shared<S, C>(col + k * Win<S, NV>::W - ex9(k) * sh));
#pragma unroll
        for (int k = 0; k < 4; ++k)
            g[k].set(c, load_as_shared<S, C>(col + (9 + k) * Win<S, NV>::W - ex4(k) * sh));
    }
}

// ---- edge area ----------------------------------------------------------------------------
constexpr int AA_BAND_MIN = 4;  // AA lattices use bands of at least this many rows (or nr)

__host__ __device__ constexpr int aa_band_cap(int nr) { return (nr + AA_BAND_MIN - 1) / AA_BAND_MIN; }

// elements of the edge area of a lattice
__host__ __device__ constexpr int64_t aa_edge_elems(int nr, int pitch, int max_strips)
{
    return (int64_t)6 * pitch * aa_band_cap(nr) + (int64_t)2 * max_strips * nr;
}

// quantity m (0: rho u_x, 1: rho u_r, 2: T - T0) of the edge row of band b, side 0/1, at column 0
template <class C>
__device__ __forceinline__ C *edge_row(const StepParams<C> &p, int b, int side, int m)
{
    return p.edge + ((int64_t)(b * 2 + side) * 3 + m) * p.epitch + PAD_COLS;
}

// rho u_r of the edge column of strip s, side 0/1, at row 0
template <class C>
__device__ __forceinline__ C *edge_col(const StepParams<C> &p, int s, int side)
{
    return p.edge + (int64_t)6 * p.epitch * aa_band_cap(p.nr) + (int64_t)(s * 2 + side) * p.nr;
}

// moments of the edge row of band b (side 0/1) for the strip's columns (the density is not needed)
template <int NV, class C>
__device__ __forceinline__ Mom<Vec<C, NV>> load_edge_row(const StepParams<C> &p, int b, int side, int x0, int lane)
{
    Mom<Vec<C, NV>> m;
    const C *rx = edge_row(p, b, side, 0), *rr = edge_row(p, b, side, 1), *rt = edge_row(p, b, side, 2);
#pragma unroll
    for (int c = 0; c < NV; ++c) {
        const int i = x0 + lane + 32 * c;
        m.drho.set(c, C(0));
        m.jx.set(c, __ldcg(rx + i));
        m.jr.set(c, __ldcg(rr + i));
        m.dT.set(c, __ldcg(rt + i));
    }
    return m;
}

// ---- phase 1: publish the edge moments of a warp tile -----------------------------------
// The tile's first and last rows are staged (moments of every column); the
// edge columns of the rows between need only rho u_r, from the six
// populations with a radial component, which lanes load one node each.
template <class S, int NV, class C>
__device__ __forceinline__ void aa_edges_tile(const StepParams<C> &p, int P, const S *__restrict__ buf, S *wsm,
                                              int tile, int lane)
{
    using Wn = Win<S, NV>;
    using V = Vec<C, NV>;
    const int s = tile % p.nstrips, b = tile / p.nstrips;
    const int x0 = s * 32 * NV;
    const int last = min(x0 + 32 * NV, p.nx) - 1;  // the strip's last column
    const int j0 = b * p.band;
    const int nrows = min(j0 + p.band, p.nr) - j0;
    C *col0 = edge_col(p, s, 0), *col1 = edge_col(p, s, 1);
    const AACopyPlan<S, NV> plan = aa_copy_plan<S, NV, C>(p, P, x0, lane);
    const int nedge = nrows > 1 ? 2 : 1;
    for (int e = 0; e < nedge; ++e) {
        aa_issue_row<S, NV, C>(p, buf, wsm + e * Wn::STAGE, plan, e ? j0 + nrows - 1 : j0, lane);
        cp_async_commit();
    }
    // interior rows: lane l takes node (edge column l % 2, row j0 + 1 + l / 2), 16 rows a round
    for (int r0 = 0; r0 < nrows - 2; r0 += 16) {
        const int r = r0 + (lane >> 1);
        if (r < nrows - 2) {
            const int j = j0 + 1 + r, i = (lane & 1) ? last : x0;
            auto ldq = [&](int q) -> C {
                return load_as<S, C>(buf + (P ? cell(p, q, i, j) : cell(p, opp_plane(q), i - qex(q), j - qey(q))));
            };
            const C jr = (ldq(2) - ldq(4)) + (ldq(5) - ldq(8)) + (ldq(6) - ldq(7));  // as in moments()
            ((lane & 1) ? col1 : col0)[j] = jr;
        }
    }
    cp_async_wait<0>();
    __syncwarp();
#pragma unroll 1
    for (int e = 0; e < nedge; ++e) {
        V f[9], g[4];
        aa_stage_pops<S, NV, C>(wsm + e * Wn::STAGE, lane, 1 - P, f, g);
        const Mom<V> m = moments<V>(f, g);
        const int j = e ? j0 + nrows - 1 : j0;
#pragma unroll
        for (int c = 0; c < NV; ++c) {
            const int i = x0 + lane + 32 * c;
            if (i == x0)
                col0[j] = m.jr[c];
            if (i == last)
                col1[j] = m.jr[c];
            if (i < p.nx) {
                // side 0 is the first row; side 1 the last (the same row for one-row tiles)
                for (int side = e; side < (nrows > 1 ? e + 1 : 2); ++side) {
                    edge_row(p, b, side, 0)[i] = m.jx[c];
                    edge_row(p, b, side, 1)[i] = m.jr[c];
                    edge_row(p, b, side, 2)[i] = m.dT[c];
                }
            }
        }
    }
    __syncwarp();  // the stages are reused by phase 2
}

// ---- phase 2: collide a warp tile in place -------------------------------------------------
// rho u_r beside the strip for the tile's first 16 rows, loaded once per
// tile: lane l < 16 holds row j0 + l of the neighbour column on the left,
// lane 16 + l that on the right (across the lattice ends for periodic
// lattices: column nx - 1 left of column 0, column 0 right of nx - 1)
template <class C>
__device__ __forceinline__ C aa_beside(const StepParams<C> &p, int s, int j0, int nrows, int lane, int r)
{
    const bool right = lane >= 16;
    int sn = right ? s + 1 : s - 1;
    if (p.bc_in == IN_PERIODIC)
        sn = sn < 0 ? p.nstrips - 1 : (sn >= p.nstrips ? 0 : sn);
    if (r >= nrows || sn < 0 || sn >= p.nstrips)
        return C(0);
    return __ldcg(edge_col(p, sn, right ? 0 : 1) + j0 + r);
}

// collide row j = j0 + r of the strip from its stage and write it (and its boundary values)
template <class S, int NV, class C>
__device__ __forceinline__ void aa_collide_row(const StepParams<C> &p, int P, S *__restrict__ buf, const S *st,
                                               int s, int lane, int j0, int r, int nrows, C bes, int64_t t,
                                               const Mom<Vec<C, NV>> &mp, const Mom<Vec<C, NV>> &mc,
                                               const Mom<Vec<C, NV>> &mn, const float2 *stab)
{
    using V = Vec<C, NV>;
    const int x0 = s * 32 * NV;
    const int j = j0 + r;
    C bl, br;  // beside values of this row (left, right)
    if (r < 16) {
        bl = __shfl_sync(0xffffffffu, bes, r);
        br = __shfl_sync(0xffffffffu, bes, 16 + r);
    } else {
        bl = aa_beside<C>(p, s, j0, nrows, 0, r);
        br = aa_beside<C>(p, s, j0, nrows, 16, r);
    }
    V left, right;
#pragma unroll
    for (int c = 0; c < NV; ++c) {
        const C up = __shfl_up_sync(0xffffffffu, mc.jr[c], 1);
        const C dn = __shfl_down_sync(0xffffffffu, mc.jr[c], 1);
        const C prev_last = __shfl_sync(0xffffffffu, mc.jr[(c + NV - 1) % NV], 31);
        const C next_first = __shfl_sync(0xffffffffu, mc.jr[(c + 1) % NV], 0);
        C l = up, rr = dn;
        if (lane == 0)
            l = (c == 0) ? bl : prev_last;
        if (lane == 31)
            rr = (c == NV - 1) ? br : next_first;
        const int i = x0 + lane + 32 * c;
        if (i == 0)  // ghost moment beyond the inlet end (periodic: the image held in bl)
            l = p.bc_in == IN_INLET ? C(0) : bl;
        if (i == p.nx - 1)  // beyond the outlet end (periodic: the image held in br)
            rr = p.bc_out == OUT_OUTFLOW ? mc.jr[c] : (p.bc_out == OUT_WALL ? -mc.jr[c] : br);
        left.set(c, l);
        right.set(c, rr);
    }
    if (x0 + lane >= p.nx)
        return;  // no active node in this lane
    V f[9], g[4], fo[9], go[4];
    aa_stage_pops<S, NV, C>(st, lane, 1 - P, f, g);
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
            if (i == 0 || i == p.nx - 1 || j == 0 || j == p.nr - 1) {
                if (P)
                    aa_write_ghosts<S, C, 0>(p, buf, i, j, t + 1);
                else
                    aa_write_ghosts<S, C, 1>(p, buf, i, j, t + 1);
            }
        }
    }
}

// Rows j0..j1-1 are staged in order; row j is collided once the moments of
// row j + 1 exist.  The moments below and above the tile are the edge rows
// of the neighbour bands (or the boundary's ghost moments at the lattice
// edges); they and the beside values are loaded ahead of their use.
template <class S, int NV, class C>
__device__ __forceinline__ void aa_collide_tile(const StepParams<C> &p, int P, S *__restrict__ buf, S *wsm, int tile,
                                                int lane, int64_t t, const float2 *stab)
{
    using Wn = Win<S, NV>;
    using V = Vec<C, NV>;
    constexpr int NSTAGE = Stages<NV>::value;
    constexpr int D = NSTAGE - 2;  // two stages are read at once
    const int s = tile % p.nstrips, b = tile / p.nstrips;
    const int x0 = s * 32 * NV;
    const int j0 = b * p.band;
    const int j1 = min(j0 + p.band, p.nr);
    const int nrows = j1 - j0;
    const AACopyPlan<S, NV> plan = aa_copy_plan<S, NV, C>(p, P, x0, lane);
    const C bes = aa_beside<C>(p, s, j0, nrows, lane, lane & 15);
    Mom<V> mp, mc, mn;
    if (j0 > 0)
        mp = load_edge_row<NV, C>(p, b - 1, 1, x0, lane);
#pragma unroll
    for (int r = 0; r < D; ++r) {
        if (r < nrows)
            aa_issue_row<S, NV, C>(p, buf, wsm + r * Wn::STAGE, plan, j0 + r, lane);
        cp_async_commit();
    }
    // one pass per staged row and one more for the last row: the collision
    // code appears once (the instruction cache is a limit of this kernel)
#pragma unroll 1
    for (int idx = 0; idx <= nrows; ++idx) {
        Mom<V> mr;
        if (idx < nrows) {
            __syncwarp();  // every lane is done with the stage refilled next (it held row idx - 2)
            if (idx + D < nrows)
                aa_issue_row<S, NV, C>(p, buf, wsm + ((idx + D) % NSTAGE) * Wn::STAGE, plan, j0 + idx + D, lane);
            cp_async_commit();
            if (idx == nrows - 1 && j1 < p.nr)
                mn = load_edge_row<NV, C>(p, b + 1, 0, x0, lane);
            cp_async_wait<D>();
            __syncwarp();
            V f[9], g[4];
            aa_stage_pops<S, NV, C>(wsm + (idx % NSTAGE) * Wn::STAGE, lane, 1 - P, f, g);
            mr = moments<V>(f, g);
            if (idx == 0) {
                if (j0 == 0)
                    mp = ghost_bottom<C, V>(p, mr);
                mc = mr;
                continue;
            }
        } else {
            mr = j1 == p.nr ? ghost_top<C, V>(p, mc) : mn;
        }
        aa_collide_row<S, NV, C>(p, P, buf, wsm + ((idx - 1) % NSTAGE) * Wn::STAGE, s, lane, j0, idx - 1, nrows, bes,
                                 t, mp, mc, mr, stab);
        mp = mc;
        mc = mr;
    }
    cp_async_wait<0>();
    __syncwarp();
}

// Every lane waits until the four direct neighbours of item (band b, column
// g) have published their edges of sub-step k - 1 (counters at 32 k or more);
// false if the wait runs out or another warp's did.
template <class C>
__device__ bool wait_edges(const StepParams<C> &p, const unsigned *pub, int cols, bool wrap, int b, int g, int k,
                           int spin_limit)
{
    const int nbands = (p.nr + p.band - 1) / p.band;
    const int lane = threadIdx.x & 31;
    const unsigned *f = nullptr;
    if (lane < 4) {
        const int bb = b + (lane == 0 ? -1 : (lane == 1 ? 1 : 0));
        int gg = g + (lane == 2 ? -1 : (lane == 3 ? 1 : 0));
        if (wrap)
            gg = gg < 0 ? gg + cols : (gg >= cols ? gg - cols : gg);
        if (bb >= 0 && bb < nbands && gg >= 0 && gg < cols)
            f = pub + bb * cols + gg;
    }
    const unsigned want = 32u * (unsigned)k;
    for (int it = 0;; ++it) {
        const bool ok = f == nullptr || (int)(ld_acquire(f) - want) >= 0;
        if (__all_sync(0xffffffffu, ok)) {
            __syncwarp();  // every lane now sees what its watcher acquired
            return true;
        }
        if (it >= spin_limit || (*static_cast<volatile int *>(p.status) & STATUS_TIMEOUT))
            return false;
        __nanosleep(it < 32 ? 32 : (it < 128 ? 256 : 2048));  // these waits are short: poll finely first
    }
}

// ---- the persistent launch ---------------------------------------------------------------
// ctl.flags holds the items' step counters (32 per finished step), then
// their edge counters (32 per published step).
template <class S, class C>
__global__ void __launch_bounds__(256) aa_run_kernel(const __grid_constant__ StepParams<C> p, const RunCtl ctl)
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
    unsigned *done = ctl.flags, *pub = ctl.flags + items;
    unsigned n = 0;
    if (lane == 0)
        n = atomicAdd(ctl.counter, 1u);
    n = __shfl_sync(0xffffffffu, n, 0);
    while (n < total) {
        const int k = (int)(n / items);
        const int item = (int)(n - (unsigned)k * items);
        const int b = item / cols, g = item - b * cols;
        const int P = (p.phase + k) & 1;
        if (k > 0 && !wait_neighbours<C>(p, done, cols, 1, ctl.wrap != 0, b, g, k, ctl.spin_limit)) {
            if (lane == 0)
                atomicOr(p.status, STATUS_TIMEOUT);
            break;  // whole warp
        }
        const int s1 = min((g + 1) * ctl.group, p.nstrips);
        for (int s = g * ctl.group; s < s1; ++s)
            aa_edges_tile<S, NV, C>(p, P, buf, wsm, b * p.nstrips + s, lane);
        red_release_add(pub + item, 1u);
        if (!wait_edges<C>(p, pub, cols, ctl.wrap != 0, b, g, k + 1, ctl.spin_limit)) {
            if (lane == 0)
                atomicOr(p.status, STATUS_TIMEOUT);
            break;
        }
        // the next item is taken only now: a warp never holds an item it has
        // not started while it waits
        unsigned next = 0;
        if (lane == 0)
            next = atomicAdd(ctl.counter, 1u);
        for (int s = g * ctl.group; s < s1; ++s)
            aa_collide_tile<S, NV, C>(p, P, buf, wsm, b * p.nstrips + s, lane, p.step + k, stab);
        red_release_add(done + item, 1u);
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
