// Device side of liblbm: the fused pull-stream + collide step of the
// axisymmetric thermal lattice Boltzmann LES model (Djebali et al.,
// arXiv:1002.3028, Eqs. 1-5 and Section 2.3), plus the small kernels that
// fill boundary ghosts, read fields and convert states.
//
// Storage.  13 planes (9 f, 4 g); each plane holds nr + 2 rows of `pitch`
// values: row -1 (ghost), rows 0..nr-1, row nr (ghost); in every row the
// lattice column i sits at element i + PAD_COLS, so columns -1 and nx are
// ghosts and every warp's strip starts on an aligned boundary.  Every value
// is the deviation from the rest state, f_k - w_k rho0 and g_k - T0/4 (the
// moment-split 2-byte types store FP32 moments beside the planes and each
// value as its deviation from the part of the equilibrium linear in them;
// see "moment-split storage").  The arithmetic type C is double for FP64
// storage and float for the others; all collision arithmetic runs on
// deviations, so the rounding of a stored value is relative to its (small)
// departure from rest.
//
// Boundaries as ghosts.  The boundary rules only ever pick, for a pulled
// source outside the lattice, a value computed from the post-collision
// populations of one node on the lattice edge (mirror, bounce-back, the
// rho0-held zero-gradient copy, the inlet equilibrium, the periodic image).
// So that node writes those values into the ghost cells right after its own
// collision (write_ghosts), and the next step's pull is 13 plain loads for
// every node, with no branch.  The radial rule is applied before the axial
// one, exactly as in the rules' definition.
//
// Work split of the step kernel.  One warp owns a strip of 32 NV consecutive
// columns (NV = 2 nodes per lane, at columns x0 + lane and x0 + 32 + lane,
// computed together with the paired FP32x2 instructions, or NV = 1: a launch
// parameter in FP32 arithmetic; NV = 1 in FP64) and marches along a band of
// rows (FP32 storage: up in even bands, down in odd ones).  The populations each row
// pulls are staged in the warp's shared-memory ring by asynchronous copies
// issued one row ahead (two in FP64); from a landed row the warp forms the
// Eq. 2 moments and collides the row below, whose radial neighbours' moments
// (same time level) it already holds.  The axial neighbours' rho u_r come
// from the adjacent columns by warp shuffle and, for the two columns beside
// the strip, from the staged window's halo.
//
// Launches.  All steps of one lbm_step call run in one persistent launch
// (step_run_kernel; batches: batch_run_kernel): warps take warp tiles in
// step-major order, and a tile of step t + 1 starts once the tiles around it
// have finished step t (see "many steps of one lattice in one launch").
// Lattices kept in one buffer updated in place use the kernels of
// lbm_aa.cuh and lbm_aa_batch.cuh, built from the same staging, moment,
// collision and boundary code.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

namespace lbm {

enum : int { IN_INLET = 0, IN_PERIODIC = 1 };
enum : int { OUT_OUTFLOW = 0, OUT_WALL = 1, OUT_PERIODIC = 2 };
enum : int { TOP_WALL = 0, TOP_OPEN = 1 };
enum : int { BOTTOM_AXIS = 0, BOTTOM_WALL = 1 };

constexpr int PAD_COLS = 32;  // element offset of lattice column 0 within a row

// ---- lattice: D2Q9 (k = 0..8) and D2Q4 (k = 0..3) --------------------------
__host__ __device__ constexpr int ex9(int k) { return (k == 1 || k == 5 || k == 8) ? 1 : ((k == 3 || k == 6 || k == 7) ? -1 : 0); }
__host__ __device__ constexpr int ey9(int k) { return (k == 2 || k == 5 || k == 6) ? 1 : ((k == 4 || k == 7 || k == 8) ? -1 : 0); }
__host__ __device__ constexpr int ex4(int k) { return k == 0 ? 1 : (k == 2 ? -1 : 0); }
__host__ __device__ constexpr int ey4(int k) { return k == 1 ? 1 : (k == 3 ? -1 : 0); }
template <class C> __host__ __device__ constexpr C w9(int k) { return k == 0 ? C(4) / C(9) : (k <= 4 ? C(1) / C(9) : C(1) / C(36)); }
// plane q = 0..12: f_0..f_8, then g_0..g_3; its velocity and the plane of the opposite velocity
__host__ __device__ constexpr int qex(int q) { return q < 9 ? ex9(q) : ex4(q - 9); }
__host__ __device__ constexpr int qey(int q) { return q < 9 ? ey9(q) : ey4(q - 9); }
__host__ __device__ constexpr int opp_plane(int q)
{
    return q == 0 ? 0 : (q < 5 ? 1 + (q + 1) % 4 : (q < 9 ? 5 + (q - 3) % 4 : 9 + (q - 7) % 4));
}

// nodes per lane of the step kernel for an arithmetic type
template <class C> struct NodesPerLane { static constexpr int value = 1; };
template <> struct NodesPerLane<float> { static constexpr int value = 2; };

// ---- kernel parameters -------------------------------------------------------
// (16-byte aligned so a warp can copy a block from a batch table in 16-byte words)
template <class C>
struct alignas(16) StepParams {
    const void *src;  // post-collision state of the previous step (with its ghosts)
    void *dst;        // post-collision state written by this step (with its ghosts)
    int64_t plane;    // elements from one population plane to the next
    int nx, nr;
    int pitch;        // elements from one row of a plane to the next (planes interleaved by row:
                      // 13 padded rows; whole planes: one)
    int bc_in, bc_out, bc_top, bc_bottom, axisym;
    int band;         // rows per warp tile
    int nstrips;      // ceil(nx / (32 NV))
    int ntiles;       // nstrips * ceil(nr / band)
    int ntab;
    int64_t step;     // time index of the step that reads src
    uint64_t seed;
    double noise_amp;
    C r0, rho0, T0;
    C cs2_18;         // 18 Cs^2 (Eq. 4 with filter width 1)
    C inv_prt;        // 1 / Pr_t (Eq. 5)
    C dT_top, dT_bottom, dT_out;  // wall temperature minus T0
    C T_lo, tab_scale;            // table position s = (T - T_lo) * tab_scale
    C hir0;                       // 1 / (2 rho0) (moment-split storage)
    const C *u_in, *T_in;         // inlet profiles, nr values
    const C *nu_tab, *al_tab;     // property tables, ntab values
    int *status;                  // error flags of the lattice
    C *edge;                      // AA layout: moments at the warp tiles' edges (see lbm_aa.cuh)
    int aa;                       // 1: one buffer in the AA layout (src == dst); 0: two buffers
    int phase;                    // AA layout: representation of the stored state
    int epitch;                   // AA layout: elements per row of the edge area (one padded row)
};

// ---- storage conversions -----------------------------------------------------
// Population loads go through L2 (ld.global.cg): a multi-step launch reads
// buffers that other warps of the same launch wrote, which the read-only
// and L1 paths may not see.
template <class S, class C> __device__ __forceinline__ C load_as(const S *p);
template <> __device__ __forceinline__ double load_as<double, double>(const double *p) { return __ldcg(p); }
template <> __device__ __forceinline__ float load_as<float, float>(const float *p) { return __ldcg(p); }
template <> __device__ __forceinline__ float load_as<__half, float>(const __half *p) { return __half2float(__ldcg(p)); }
template <> __device__ __forceinline__ float load_as<__nv_bfloat16, float>(const __nv_bfloat16 *p) { return __bfloat162float(__ldcg(p)); }

template <class S, class C> __device__ __forceinline__ C load_as_shared(const S *p);
template <> __device__ __forceinline__ double load_as_shared<double, double>(const double *p) { return *p; }
template <> __device__ __forceinline__ float load_as_shared<float, float>(const float *p) { return *p; }
template <> __device__ __forceinline__ float load_as_shared<__half, float>(const __half *p) { return __half2float(*p); }
template <> __device__ __forceinline__ float load_as_shared<__nv_bfloat16, float>(const __nv_bfloat16 *p) { return __bfloat162float(*p); }

template <class S, class C> __device__ __forceinline__ S store_as(C v);
template <> __device__ __forceinline__ double store_as<double, double>(double v) { return v; }
template <> __device__ __forceinline__ float store_as<float, float>(float v) { return v; }
template <> __device__ __forceinline__ __half store_as<__half, float>(float v) { return __float2half_rn(v); }
template <> __device__ __forceinline__ __nv_bfloat16 store_as<__nv_bfloat16, float>(float v) { return __float2bfloat16_rn(v); }

// ---- moment-split storage of 2-byte types ------------------------------------
// Storage types half_s and bf16_s keep, for every cell, the moments
// j_x = rho u_x, j_r = rho u_r and T - T0 in FP32 (after the 13 population
// planes of the buffer, at byte offset split_moff(plane): a plane of
// (j_x, j_r) pairs, 2 plane floats, then a plane of T - T0), and
// each population as its 2-byte deviation d from the part of the equilibrium
// that is linear in those moments:
//   f_k - w_k rho0 = 3 w_k e_k.j + d_k,
//   g_k - T0/4     = (T - T0)/4 + T e_k.j / (2 rho0) + d_k.
// A node stores its own pre-collision moments and the deviations of its
// post-collision populations from their linear parts at those moments; a
// pull adds back the linear part at the moments stored with the pulled
// value.  Both sides evaluate it with the same FP32 expression, so the only
// loss is the 2-byte rounding of d, which holds the non-equilibrium and
// quadratic parts only: its rounding no longer scales with the velocity or
// the temperature excess of the jet.
struct half_s {
    __half v;
};
struct bf16_s {
    __nv_bfloat16 v;
};
template <class S> struct IsSplit { static constexpr bool value = false; };
template <> struct IsSplit<half_s> { static constexpr bool value = true; };
template <> struct IsSplit<bf16_s> { static constexpr bool value = true; };
constexpr int SPLIT_MOMENTS = 3;  // j_x, j_r, T - T0

// byte offset of the first moment plane in a buffer of 13 planes of `plane` 2-byte values
__host__ __device__ constexpr int64_t split_moff(int64_t plane) { return (13 * plane * 2 + 255) / 256 * 256; }

template <> __device__ __forceinline__ float load_as<half_s, float>(const half_s *p) { return __half2float(__ldcg(&p->v)); }
template <> __device__ __forceinline__ float load_as<bf16_s, float>(const bf16_s *p) { return __bfloat162float(__ldcg(&p->v)); }
template <> __device__ __forceinline__ float load_as_shared<half_s, float>(const half_s *p) { return __half2float(p->v); }
template <> __device__ __forceinline__ float load_as_shared<bf16_s, float>(const bf16_s *p) { return __bfloat162float(p->v); }
template <> __device__ __forceinline__ half_s store_as<half_s, float>(float v) { return half_s{__float2half_rn(v)}; }
template <> __device__ __forceinline__ bf16_s store_as<bf16_s, float>(float v) { return bf16_s{__float2bfloat16_rn(v)}; }

// the moments of cell offset o (an element offset within a plane) in a moment area M
struct MomRef {
    float *M;
    int64_t plane;
    __device__ __forceinline__ float2 &j(int64_t o) const { return reinterpret_cast<float2 *>(M)[o]; }
    __device__ __forceinline__ float &T(int64_t o) const { return M[2 * plane + o]; }
};

template <class S>
__device__ __forceinline__ float *split_m(S *buf, int64_t plane)
{
    return reinterpret_cast<float *>(reinterpret_cast<char *>(buf) + split_moff(plane));
}
template <class S>
__device__ __forceinline__ const float *split_m(const S *buf, int64_t plane)
{
    return reinterpret_cast<const float *>(reinterpret_cast<const char *>(buf) + split_moff(plane));
}

// linear part of population q (deviation from rest) at moments (jx, jr, dT)
// e.j for a lattice velocity e with components in {-1, 0, 1} (no product with a zero component)
template <class C>
__device__ __forceinline__ C edot(int ex, int ey, C jx, C jr)
{
    const C a = ex > 0 ? jx : -jx, b = ey > 0 ? jr : -jr;
    return ex == 0 ? (ey == 0 ? C(0) : b) : (ey == 0 ? a : a + b);
}

template <class C>
__device__ __forceinline__ C lin_part(const StepParams<C> &p, int q, C jx, C jr, C dT)
{
    if (q == 0)
        return C(0);
    if (q < 9)
        return (C(3) * w9<C>(q)) * edot<C>(ex9(q), ey9(q), jx, jr);
    return C(0.25) * dT + (p.T0 + dT) * p.hir0 * edot<C>(ex4(q - 9), ey4(q - 9), jx, jr);
}

// Moments a ghost cell (ci, cj) carries when node (i, j), with moments
// (jx, jr, dT), writes it: the one node whose rule fills an axis, open-top,
// inlet, outflow or periodic ghost cell writes its own moments there
// (mirrored across the axis; the prescribed inflow at the inlet).  The
// lattice corners and the cells beyond walls, which several nodes fill,
// carry zero moments and their populations whole.  Returns false for those.
template <class C>
__device__ __forceinline__ bool ghost_moments(const StepParams<C> &p, int ci, int cj, C jx, C jr, C dT, C &gx, C &gr,
                                              C &gT)
{
    const bool col_in = ci >= 0 && ci < p.nx, row_in = cj >= 0 && cj < p.nr;
    gx = jx;
    gr = jr;
    gT = dT;
    if (col_in && cj == -1) {
        gr = -jr;
        return p.bc_bottom == BOTTOM_AXIS;
    }
    if (col_in && cj == p.nr)
        return p.bc_top == TOP_OPEN;
    if (row_in && ci == -1) {
        if (p.bc_in == IN_INLET) {
            gx = p.rho0 * p.u_in[cj];
            gr = C(0);
            gT = p.T_in[cj] - p.T0;
        }
        return true;
    }
    if (row_in && ci == p.nx)
        return p.bc_out != OUT_WALL;
    return false;
}

template <class C>
__device__ __forceinline__ int64_t cell(const StepParams<C> &p, int q, int i, int j)
{
    return (int64_t)q * p.plane + (int64_t)(j + 1) * p.pitch + (i + PAD_COLS);
}

template <class S, class C>
__device__ __forceinline__ C ld(const StepParams<C> &p, const S *src, int q, int i, int j)
{
    return load_as<S, C>(src + cell(p, q, i, j));
}

// ---- NV nodes of one lane as one value ---------------------------------------
// Vec<C, 1> is a scalar; Vec<float, 2> holds two nodes and maps +, -, * and
// fma onto the paired FP32x2 instructions of sm_100 and later.
template <class C, int N> struct Vec;

template <class C>
struct Vec<C, 1> {
    C x;
    __device__ __forceinline__ Vec() {}
    __device__ __forceinline__ explicit Vec(C s) : x(s) {}
    __device__ __forceinline__ C operator[](int) const { return x; }
    __device__ __forceinline__ void set(int, C v) { x = v; }
};
// One rounding per operation, exactly as the paired instructions round each
// of their two lanes: the compiler may not fuse a product into a following
// sum across these operators (it would for plain a * b + c), so a node gives
// the same bits at either strip width.
__device__ __forceinline__ float rn_add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float rn_sub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float rn_mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float rn_fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double rn_add(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double rn_sub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double rn_mul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double rn_fma(double a, double b, double c) { return __fma_rn(a, b, c); }

template <class C> __device__ __forceinline__ Vec<C, 1> operator+(Vec<C, 1> a, Vec<C, 1> b) { return Vec<C, 1>(rn_add(a.x, b.x)); }
template <class C> __device__ __forceinline__ Vec<C, 1> operator-(Vec<C, 1> a, Vec<C, 1> b) { return Vec<C, 1>(rn_sub(a.x, b.x)); }
template <class C> __device__ __forceinline__ Vec<C, 1> operator*(Vec<C, 1> a, Vec<C, 1> b) { return Vec<C, 1>(rn_mul(a.x, b.x)); }
template <class C> __device__ __forceinline__ Vec<C, 1> operator-(Vec<C, 1> a) { return Vec<C, 1>(-a.x); }
template <class C> __device__ __forceinline__ Vec<C, 1> vfma(Vec<C, 1> a, Vec<C, 1> b, Vec<C, 1> c) { return Vec<C, 1>(rn_fma(a.x, b.x, c.x)); }

template <>
struct Vec<float, 2> {
    float2 v;
    __device__ __forceinline__ Vec() {}
    __device__ __forceinline__ explicit Vec(float s) : v(make_float2(s, s)) {}
    __device__ __forceinline__ explicit Vec(float2 a) : v(a) {}
    __device__ __forceinline__ float operator[](int c) const { return c ? v.y : v.x; }
    __device__ __forceinline__ void set(int c, float a)
    {
        if (c)
            v.y = a;
        else
            v.x = a;
    }
};
using F2 = Vec<float, 2>;
__device__ __forceinline__ F2 operator+(F2 a, F2 b) { return F2(__fadd2_rn(a.v, b.v)); }
__device__ __forceinline__ F2 operator-(F2 a, F2 b) { return F2(__ffma2_rn(b.v, make_float2(-1.f, -1.f), a.v)); }
__device__ __forceinline__ F2 operator*(F2 a, F2 b) { return F2(__fmul2_rn(a.v, b.v)); }
__device__ __forceinline__ F2 operator-(F2 a) { return F2(make_float2(-a.v.x, -a.v.y)); }
__device__ __forceinline__ F2 vfma(F2 a, F2 b, F2 c) { return F2(__ffma2_rn(a.v, b.v, c.v)); }

template <class C, int N> __device__ __forceinline__ Vec<C, N> operator*(C s, Vec<C, N> a) { return Vec<C, N>(s) * a; }
template <class C, int N> __device__ __forceinline__ Vec<C, N> operator+(C s, Vec<C, N> a) { return Vec<C, N>(s) + a; }
template <class C, int N> __device__ __forceinline__ Vec<C, N> operator-(Vec<C, N> a, C s) { return a - Vec<C, N>(s); }
template <class C, int N> __device__ __forceinline__ Vec<C, N> operator-(C s, Vec<C, N> a) { return Vec<C, N>(s) - a; }

// component-wise reciprocal and square root
template <class C, int N>
__device__ __forceinline__ Vec<C, N> vrcp(Vec<C, N> a)
{
    Vec<C, N> r;
#pragma unroll
    for (int c = 0; c < N; ++c)
        r.set(c, C(1) / a[c]);
    return r;
}

template <class C, int N>
__device__ __forceinline__ Vec<C, N> vsqrt(Vec<C, N> a)
{
    Vec<C, N> r;
#pragma unroll
    for (int c = 0; c < N; ++c)
        r.set(c, sqrt(a[c]));
    return r;
}

// ---- inlet noise: SplitMix64 (Steele, Lea, Flood, OOPSLA 2014) ---------------
__device__ __forceinline__ uint64_t splitmix64(uint64_t x)
{
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// prescribed inlet velocity of row j at time index t: profile, plus the
// noise xi = amp (2U - 1) where the profile is non-zero
template <class C>
__device__ __forceinline__ C inlet_velocity(const StepParams<C> &p, int j, int64_t t)
{
    C u = p.u_in[j];
    if (u != C(0) && p.noise_amp != 0.0) {
        const uint64_t c = ((uint64_t)t << 20) + (uint64_t)j;
        const uint64_t h = splitmix64(p.seed ^ splitmix64(c));
        const double U = (double)(h >> 11) * (1.0 / 9007199254740992.0);
        u += C(p.noise_amp * (2.0 * U - 1.0));
    }
    return u;
}

// ---- equilibria (deviation form) ---------------------------------------------
// f_eq_k(rho, u) - w_k rho0 = w_k (drho + rho (3 e.u + 9/2 (e.u)^2 - 3/2 u.u))
template <class C>
__device__ __forceinline__ C feq_dev(int k, C drho, C rho, C ux, C ur)
{
    const C eu = C(ex9(k)) * ux + C(ey9(k)) * ur;
    const C uu = ux * ux + ur * ur;
    return w9<C>(k) * (drho + rho * (C(3) * eu + C(4.5) * eu * eu - C(1.5) * uu));
}

// unit-density equilibrium w_k (1 + 3 e.u + 9/2 (e.u)^2 - 3/2 u.u)
template <class C>
__device__ __forceinline__ C feq_unit(int k, C ux, C ur)
{
    const C eu = C(ex9(k)) * ux + C(ey9(k)) * ur;
    const C uu = ux * ux + ur * ur;
    return w9<C>(k) * (C(1) + C(3) * eu + C(4.5) * eu * eu - C(1.5) * uu);
}

// ---- boundary ghosts -------------------------------------------------------------
// The boundary rules of node (i, j) on the lattice edge, given its
// post-collision deviations fo, go: W(q, ci, cj, v) is called for every
// ghost cell (ci, cj) of plane q whose value the rules take from this node
// (v is that value).  t is the time index of the step that will pull these
// ghosts (inlet noise).  Writers of distinct ghost cells are distinct
// nodes, except where two rules give the same bounce-back value to the same
// cell.
template <class C, class Wr>
__device__ __forceinline__ void ghost_rules(const StepParams<C> &p, const C (&fo)[9], const C (&go)[4], int i, int j,
                                            int64_t t, Wr W)
{
    const int nx = p.nx, nr = p.nr;
    C drho = C(0), jx = C(0), jr = C(0);
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        drho += fo[k];
        jx += C(ex9(k)) * fo[k];
        jr += C(ey9(k)) * fo[k];
    }
    const C rho = p.rho0 + drho;
    const C ux = jx / rho, ur = jr / rho;
    // zero-gradient copy of this node held at rho0
    auto openc = [&](int k) -> C { return fo[k] - drho * feq_unit<C>(k, ux, ur); };
    // inlet equilibrium at this node's density, this row's prescribed velocity
    auto inlet_f = [&](int k) -> C { return feq_dev<C>(k, drho, rho, inlet_velocity<C>(p, j, t), C(0)); };
    auto inlet_g0 = [&]() -> C {
        const C T = p.T_in[j];
        return C(0.25) * (T - p.T0) + C(0.5) * T * inlet_velocity<C>(p, j, t);
    };

    // radial edges (and the corner cells the radial rule reaches first)
    if (j == 0) {
        if (p.bc_bottom == BOTTOM_AXIS) {  // specular mirror
            W(2, i, -1, fo[4]);
            W(5, i, -1, fo[8]);
            W(6, i, -1, fo[7]);
            W(9 + 1, i, -1, go[3]);
            if (i == 0) {
                if (p.bc_in == IN_INLET)
                    W(5, -1, -1, inlet_f(8));
                else
                    W(6, nx, -1, fo[7]);
            }
            if (i == nx - 1) {
                if (p.bc_out == OUT_OUTFLOW)
                    W(6, nx, -1, openc(7));
                else if (p.bc_out == OUT_PERIODIC)
                    W(5, -1, -1, fo[8]);
            }
        } else {  // half-way bounce-back, thermal anti-bounce-back
            W(2, i, -1, fo[4]);
            W(5, i - 1, -1, fo[7]);
            W(6, i + 1, -1, fo[8]);
            W(9 + 1, i, -1, -go[3] + C(0.5) * p.dT_bottom);
        }
    }
    if (j == nr - 1) {
        if (p.bc_top == TOP_WALL) {
            W(4, i, nr, fo[2]);
            W(7, i + 1, nr, fo[5]);
            W(8, i - 1, nr, fo[6]);
            W(9 + 3, i, nr, -go[1] + C(0.5) * p.dT_top);
        } else {
            W(4, i, nr, openc(4));
            W(7, i, nr, openc(7));
            W(8, i, nr, openc(8));
            W(9 + 3, i, nr, go[3]);
            if (i == 0) {
                if (p.bc_in == IN_INLET)
                    W(8, -1, nr, inlet_f(8));
                else
                    W(7, nx, nr, openc(7));
            }
            if (i == nx - 1) {
                if (p.bc_out == OUT_OUTFLOW)
                    W(7, nx, nr, openc(7));
                else if (p.bc_out == OUT_PERIODIC)
                    W(8, -1, nr, openc(8));
            }
        }
    }
    // axial edges
    if (i == 0) {
        if (p.bc_in == IN_INLET) {
            W(1, -1, j, inlet_f(1));
            W(5, -1, j, inlet_f(5));
            W(8, -1, j, inlet_f(8));
            W(9 + 0, -1, j, inlet_g0());
        } else {  // periodic image of column 0 beyond the outlet
            W(3, nx, j, fo[3]);
            W(6, nx, j, fo[6]);
            W(7, nx, j, fo[7]);
            W(9 + 2, nx, j, go[2]);
        }
    }
    if (i == nx - 1) {
        if (p.bc_out == OUT_OUTFLOW) {
            W(3, nx, j, openc(3));
            W(6, nx, j, openc(6));
            W(7, nx, j, openc(7));
            W(9 + 2, nx, j, go[2]);
        } else if (p.bc_out == OUT_WALL) {
            W(3, nx, j, fo[1]);
            W(6, nx, j - 1, fo[8]);
            W(7, nx, j + 1, fo[5]);
            W(9 + 2, nx, j, -go[0] + C(0.5) * p.dT_out);
        } else {  // periodic image of column nx - 1 before the inlet
            W(1, -1, j, fo[1]);
            W(5, -1, j, fo[5]);
            W(8, -1, j, fo[8]);
            W(9 + 0, -1, j, go[0]);
        }
    }
}

// Two-buffer layout: node (i, j) on the lattice edge, whose post-collision
// deviations are already stored in buf, writes the ghost cells of buf that
// the rules take from it.
template <class S, class C>
__device__ __noinline__ void write_ghosts(const StepParams<C> &p, S *buf, int i, int j, int64_t t)
{
    C fo[9], go[4];
    if constexpr (IsSplit<S>::value) {
        // the node's stored populations (its moments plus the stored deviations), then each
        // ghost value as a deviation from the linear part at the ghost cell's own moments
        const MomRef M{split_m(buf, p.plane), p.plane};
        const int64_t o = cell(p, 0, i, j);
        const float2 jj = M.j(o);  // plain loads: this thread stored them
        const C jx = jj.x, jr = jj.y, dT = M.T(o);
#pragma unroll
        for (int k = 0; k < 9; ++k)
            fo[k] = lin_part<C>(p, k, jx, jr, dT) + load_as_shared<S, C>(buf + cell(p, k, i, j));
#pragma unroll
        for (int k = 0; k < 4; ++k)
            go[k] = lin_part<C>(p, 9 + k, jx, jr, dT) + load_as_shared<S, C>(buf + cell(p, 9 + k, i, j));
        ghost_rules<C>(p, fo, go, i, j, t, [&](int q, int ci, int cj, C v) {
            C gx, gr, gT;
            const int64_t oc = cell(p, 0, ci, cj);
            if (ghost_moments<C>(p, ci, cj, jx, jr, dT, gx, gr, gT)) {
                M.j(oc) = make_float2(gx, gr);
                M.T(oc) = gT;
                v -= lin_part<C>(p, q, gx, gr, gT);
            }
            buf[cell(p, q, ci, cj)] = store_as<S, C>(v);
        });
        return;
    }
#pragma unroll
    for (int k = 0; k < 9; ++k)
        fo[k] = load_as_shared<S, C>(buf + cell(p, k, i, j));  // plain load: this thread stored it
#pragma unroll
    for (int k = 0; k < 4; ++k)
        go[k] = load_as_shared<S, C>(buf + cell(p, 9 + k, i, j));
    ghost_rules<C>(p, fo, go, i, j, t, [&](int q, int ci, int cj, C v) { buf[cell(p, q, ci, cj)] = store_as<S, C>(v); });
}

// ---- pull and moments -------------------------------------------------------------
// element offset of population q streamed into node (i, j) from a stored
// state: the post-collision value of node (i, j) - e_q (two buffers), or
// the AA layout's slot for that population in the state's representation
template <class C>
__device__ __forceinline__ int64_t stream_cell(const StepParams<C> &p, int q, int i, int j)
{
    if (p.aa && p.phase)
        return cell(p, q, i, j);
    return cell(p, p.aa ? opp_plane(q) : q, i - qex(q), j - qey(q));
}

// population q streamed into node (i, j) from a stored state (deviation from rest)
template <class S, class C>
__device__ __forceinline__ C pulled(const StepParams<C> &p, const S *src, int q, int i, int j)
{
    const int64_t c = stream_cell(p, q, i, j);
    C v = load_as<S, C>(src + c);
    if constexpr (IsSplit<S>::value) {  // plus the linear part at the source cell's moments
        const float *M = split_m(src, p.plane);
        const int64_t o = c - (int64_t)q * p.plane;
        const float2 jj = __ldcg(reinterpret_cast<const float2 *>(M) + o);
        v += lin_part<C>(p, q, jj.x, jj.y, __ldcg(M + 2 * p.plane + o));
    }
    return v;
}

template <class S, class C>
__device__ __forceinline__ void pull(const StepParams<C> &p, const S *src, int i, int j, C (&f)[9], C (&g)[4])
{
#pragma unroll
    for (int k = 0; k < 9; ++k)
        f[k] = pulled<S, C>(p, src, k, i, j);
#pragma unroll
    for (int k = 0; k < 4; ++k)
        g[k] = pulled<S, C>(p, src, 9 + k, i, j);
}

template <class V>
struct Mom {
    V drho, jx, jr, dT;  // rho - rho0, rho u_x, rho u_r, T - T0
};

template <class V>
__device__ __forceinline__ Mom<V> moments(const V (&f)[9], const V (&g)[4])
{
    Mom<V> m;
    m.drho = ((f[0] + f[1]) + (f[2] + f[3])) + ((f[4] + f[5]) + (f[6] + f[7])) + f[8];
    m.jx = (f[1] - f[3]) + (f[5] - f[6]) + (f[8] - f[7]);
    m.jr = (f[2] - f[4]) + (f[5] - f[8]) + (f[6] - f[7]);
    m.dT = (g[0] + g[1]) + (g[2] + g[3]);
    return m;
}

// moments of the ghost row below row 0 / above row nr - 1 (central differences)
template <class C, class V>
__device__ __forceinline__ Mom<V> ghost_bottom(const StepParams<C> &p, Mom<V> m)
{
    if (p.bc_bottom == BOTTOM_AXIS) {
        m.jr = -m.jr;  // rho u_r odd, rho u_x and T even across the axis
    } else {
        m.jx = -m.jx;
        m.jr = -m.jr;
        m.dT = V(C(2) * p.dT_bottom) - m.dT;
    }
    return m;
}

template <class C, class V>
__device__ __forceinline__ Mom<V> ghost_top(const StepParams<C> &p, Mom<V> m)
{
    if (p.bc_top == TOP_WALL) {
        m.jx = -m.jx;
        m.jr = -m.jr;
        m.dT = V(C(2) * p.dT_top) - m.dT;
    }
    return m;
}

// Eq. 2 moments at node (i, j) (deviations from rest) of the populations
// streamed from the stored state, or (previous, two-buffer layout only) of
// those streamed from the other buffer, the state one step earlier
template <class S, class C>
__device__ __forceinline__ Mom<Vec<C, 1>> node_moments(const StepParams<C> &p, int i, int j, bool previous)
{
    using V1 = Vec<C, 1>;
    C f[9], g[4];
    pull<S, C>(p, static_cast<const S *>(previous ? p.dst : p.src), i, j, f, g);
    V1 vf[9], vg[4];
#pragma unroll
    for (int k = 0; k < 9; ++k)
        vf[k] = V1(f[k]);
#pragma unroll
    for (int k = 0; k < 4; ++k)
        vg[k] = V1(g[k]);
    return moments<V1>(vf, vg);
}

// rho u_r of the streamed populations at lattice node (i, j): the six
// populations with a radial component
template <class S, class C>
__device__ __forceinline__ C jr_at(const StepParams<C> &p, const S *src, int i, int j)
{
    if constexpr (IsSplit<S>::value)
        return (pulled<S, C>(p, src, 2, i, j) - pulled<S, C>(p, src, 4, i, j)) +
               (pulled<S, C>(p, src, 5, i, j) - pulled<S, C>(p, src, 8, i, j)) +
               (pulled<S, C>(p, src, 6, i, j) - pulled<S, C>(p, src, 7, i, j));
    return (ld<S, C>(p, src, 2, i, j - 1) - ld<S, C>(p, src, 4, i, j + 1)) +
           (ld<S, C>(p, src, 5, i - 1, j - 1) - ld<S, C>(p, src, 8, i - 1, j + 1)) +
           (ld<S, C>(p, src, 6, i + 1, j - 1) - ld<S, C>(p, src, 7, i + 1, j + 1));
}

// ---- properties (Section 2.3) ------------------------------------------------------
// Property tables copied to shared memory by a persistent CTA (2-byte
// storage, up to SMEM_TAB entries) as (nu_m, alpha_m) pairs: two 8-byte
// loads a node instead of four global ones, and the same interpolation.
// Measured on the 4096 x 1024 jet: FP16 62.4 GLUPS against 61.0.  FP32
// storage keeps the global path: its staging rings already fill most of the
// shared memory, and 2 KB more per CTA left too little L1 (49.0 against 52.2).
constexpr int SMEM_TAB = 256;
template <class S, class C>
struct UseSmemTable {
    static constexpr bool value = std::is_same<C, float>::value && sizeof(S) == 2;
};

__device__ __forceinline__ void load_smem_table(const StepParams<float> &p, float2 *tab)
{
    for (int m = threadIdx.x; m < p.ntab; m += blockDim.x)
        tab[m] = make_float2(__ldg(p.nu_tab + m), __ldg(p.al_tab + m));
}

template <class C>
__device__ __forceinline__ void properties(const StepParams<C> &p, C T, C &nu, C &al, const float2 *stab)
{
    if (p.ntab == 1) {
        nu = __ldg(p.nu_tab);
        al = __ldg(p.al_tab);
        return;
    }
    C s = (T - p.T_lo) * p.tab_scale;
    if (!(s > C(0)))
        s = C(0);
    const C smax = C(p.ntab - 1);
    if (s > smax)
        s = smax;
    int m = (int)floor(s);
    if (m > p.ntab - 2)
        m = p.ntab - 2;
    const C fr = s - C(m);
    if constexpr (std::is_same<C, float>::value) {
        if (stab != nullptr) {
            const float2 e0 = stab[m], e1 = stab[m + 1];
            nu = e0.x + fr * (e1.x - e0.x);
            al = e0.y + fr * (e1.y - e0.y);
            return;
        }
    }
    const C n0 = __ldg(p.nu_tab + m), n1 = __ldg(p.nu_tab + m + 1);
    const C a0 = __ldg(p.al_tab + m), a1 = __ldg(p.al_tab + m + 1);
    nu = n0 + fr * (n1 - n0);
    al = a0 + fr * (a1 - a0);
}

// ---- collision of NV nodes (right-hand side of Eq. 1) -------------------------------
// d_* are central differences: d_r(rho u_x), d_r(rho u_r), d_x(rho u_r), d_r T.
// Equilibrium deviations are formed pairwise: with j = rho u,
//   f_eq_k - w_k rho0 = w_k (A + 3 e_k.j + 9/2 (e_k.j)(e_k.u)),  A = drho - 3/2 j.u,
// and opposite directions share the quadratic term.
template <class C, class V>
__device__ __forceinline__ void collide(const StepParams<C> &p, const V (&f)[9], const V (&g)[4], const Mom<V> &m,
                                        C inv_r, V d_rjx, V d_rjr, V d_xjr, V d_rT, V (&fo)[9], V (&go)[4],
                                        const float2 *stab)
{
    constexpr int N = sizeof(V) / sizeof(C);
    constexpr C third = C(1) / C(3);
    constexpr C sixth = C(1) / C(6);
    constexpr C w0 = C(4) / C(9), w1 = C(1) / C(9), w2 = C(1) / C(36);
    const V rho = p.rho0 + m.drho;
    const V inv_rho = vrcp(rho);
    const V ux = m.jx * inv_rho, ur = m.jr * inv_rho;
    const V T = p.T0 + m.dT;
    V nu, al;
#pragma unroll
    for (int c = 0; c < N; ++c) {
        C a, b;
        properties<C>(p, T[c], a, b, stab);
        nu.set(c, a);
        al.set(c, b);
    }
    const V tau_nu = vfma(V(C(3)), nu, V(C(0.5)));

    const V A = m.drho - C(1.5) * vfma(m.jx, ux, m.jr * ur);
    const V jp = m.jx + m.jr, up = ux + ur, jm = m.jx - m.jr, um = ux - ur;
    const V qx = vfma(C(4.5) * m.jx, ux, A), qr = vfma(C(4.5) * m.jr, ur, A);
    const V qp = vfma(C(4.5) * jp, up, A), qm = vfma(C(4.5) * jm, um, A);
    const V jx3 = C(3) * m.jx, jr3 = C(3) * m.jr, jp3 = C(3) * jp, jm3 = C(3) * jm;
    V fneq[9];
    fneq[0] = f[0] - w0 * A;
    fneq[1] = f[1] - w1 * (qx + jx3);
    fneq[3] = f[3] - w1 * (qx - jx3);
    fneq[2] = f[2] - w1 * (qr + jr3);
    fneq[4] = f[4] - w1 * (qr - jr3);
    fneq[5] = f[5] - w2 * (qp + jp3);  // e = (1, 1)
    fneq[7] = f[7] - w2 * (qp - jp3);  // e = (-1, -1)
    fneq[8] = f[8] - w2 * (qm + jm3);  // e = (1, -1)
    fneq[6] = f[6] - w2 * (qm - jm3);  // e = (-1, 1)

    // stress Q_ij of Eq. 4 and the Smagorinsky relaxation time
    const V dsum = (fneq[5] + fneq[6]) + (fneq[7] + fneq[8]);
    const V Qxx = (fneq[1] + fneq[3]) + dsum;
    const V Qrr = (fneq[2] + fneq[4]) + dsum;
    const V Qxr = (fneq[5] - fneq[6]) + (fneq[7] - fneq[8]);
    const V Qn = vsqrt(C(2) * vfma(Qxx, Qxx, vfma(C(2) * Qxr, Qxr, Qrr * Qrr)));
    const V tau = C(0.5) * (tau_nu + vsqrt(vfma(tau_nu, tau_nu, V(p.cs2_18) * Qn * inv_rho)));  // Eq. 4
    const V nu_t = (tau - tau_nu) * V(third);                                                   // Eq. 3
    const V al_tot = vfma(nu_t, V(p.inv_prt), al);                                              // Eq. 5
    const V tau_a = vfma(V(C(2)), al_tot, V(C(0.5)));
    const V nu_tot = (tau - C(0.5)) * V(third);

    // axisymmetric sources
    V F1(C(0)), F2x(C(0)), F2r(C(0)), S(C(0));
    if (p.axisym) {
        const V ir(inv_r);
        const V nr_ = nu_tot * ir;
        F1 = -(m.jr * ir);
        F2x = vfma(nr_, d_rjx + d_xjr, -(m.jx * ur * ir));
        F2r = vfma(nr_, (d_rjr + d_rjr) - C(2) * m.jr * ir, -(m.jr * ur * ir));
        S = vfma(al_tot * ir, d_rT, -(T * ur * ir));
    }

    const V omega = vrcp(tau);
    const V omega_a = vrcp(tau_a);
    const V sx = F2x * V(sixth), sr = F2r * V(sixth);
    const V s1 = w1 * F1, s2 = w2 * F1;
    const V nomega = -omega;
    fo[0] = vfma(nomega, fneq[0], vfma(V(w0), F1, f[0]));  // one rounding at every strip width
    fo[1] = vfma(nomega, fneq[1], f[1] + (s1 + sx));
    fo[3] = vfma(nomega, fneq[3], f[3] + (s1 - sx));
    fo[2] = vfma(nomega, fneq[2], f[2] + (s1 + sr));
    fo[4] = vfma(nomega, fneq[4], f[4] + (s1 - sr));
    fo[5] = vfma(nomega, fneq[5], f[5] + (s2 + (sx + sr)));
    fo[7] = vfma(nomega, fneq[7], f[7] + (s2 - (sx + sr)));
    fo[8] = vfma(nomega, fneq[8], f[8] + (s2 + (sx - sr)));
    fo[6] = vfma(nomega, fneq[6], f[6] + (s2 - (sx - sr)));

    // D2Q4: g_eq_k - T0/4 = dT/4 + (T/2) e_k.u
    const V gd = C(0.25) * m.dT;
    const V hT = C(0.5) * T;
    const V hx = hT * ux, hr = hT * ur;
    const V qS = C(0.25) * S;
    const V nomega_a = -omega_a;
    go[0] = vfma(nomega_a, g[0] - (gd + hx), g[0] + qS);
    go[2] = vfma(nomega_a, g[2] - (gd - hx), g[2] + qS);
    go[1] = vfma(nomega_a, g[1] - (gd + hr), g[1] + qS);
    go[3] = vfma(nomega_a, g[3] - (gd - hr), g[3] + qS);
}

// rho u_r just beyond the inlet end (ghost moment of the central difference)
template <class S, class C>
__device__ __forceinline__ C jr_beyond_inlet(const StepParams<C> &p, const S *src, int j)
{
    if (p.bc_in == IN_INLET)
        return C(0);  // the imposed inflow has no radial component
    return jr_at<S, C>(p, src, p.nx - 1, j);
}

// rho u_r just beyond the outlet end; jr_last is that of column nx - 1
template <class S, class C>
__device__ __forceinline__ C jr_beyond_outlet(const StepParams<C> &p, const S *src, int j, C jr_last)
{
    if (p.bc_out == OUT_OUTFLOW)
        return jr_last;
    if (p.bc_out == OUT_WALL)
        return -jr_last;
    return jr_at<S, C>(p, src, 0, j);
}

// ---- shared-memory staging of pulled rows -------------------------------------------
// Each warp owns a ring of NSTAGE<NV> stages (3 for two nodes per lane, 4
// for one: the stage sizes differ, the shared memory per SM does not).  A
// stage holds, for one lattice row
// r and each plane q, the window of source row r - e_qy over source columns
// x0 - H .. x0 + 32 NV - 1 + H (H = one 16-byte chunk of elements), copied
// with asynchronous 16-byte copies spread over the warp's lanes.  Node
// column c of the strip (0 .. 32 NV - 1) reads population q at window index
// c + H - e_qx.
template <int NV> struct Stages { static constexpr int value = NV == 1 ? 4 : 3; };
// the step kernels' ring: moment-split storage keeps three stages (populations one row
// ahead, which its moment ring assumes) at every width
template <class S, int NV>
constexpr int step_stages()
{
    return IsSplit<S>::value ? 3 : Stages<NV>::value;
}

template <class S, int NV>
struct Win {
    static constexpr int E = 16 / (int)sizeof(S);  // elements per 16-byte chunk
    static constexpr int H = E;                    // halo elements on each side
    static constexpr int W = 32 * NV + 2 * H;      // window length
    static constexpr int CH = W / E;               // chunks per plane
    static constexpr int STAGE = 13 * W;           // elements per stage
};

// e_y of plane q (9 D2Q9 planes, then 4 D2Q4 planes)
__device__ __forceinline__ int plane_ey(int q)
{
    // (e_y + 1) packed two bits per plane
    constexpr unsigned packed = (1u << 0) | (1u << 2) | (2u << 4) | (1u << 6) | (0u << 8) | (2u << 10) | (2u << 12) |
                                (0u << 14) | (0u << 16) | (1u << 18) | (2u << 20) | (1u << 22) | (0u << 24);
    return (int)((packed >> (2 * q)) & 3u) - 1;
}

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }

template <int N>
__device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// The chunks one lane copies for every row of a tile.  Every plane copies
// its 32 NV own columns (OPP chunks); the 16-byte halo chunk on the left is
// copied only for the six planes that read it (f1, f5, f8, g0 pull from
// x - 1; f2, f4, f5, f8 enter rho u_r at column -1), the one on the right
// only for f3, f6, f7, g2 and f2, f4, f6, f7 likewise: 13 OPP + 12 chunks a
// row instead of 13 (OPP + 2).  Chunk t = lane + 32 m is an own chunk for
// t < 13 OPP (plane t / OPP, window chunk 1 + t % OPP), else halo chunk
// t - 13 OPP of the table below.  It lands at window element
// plane * W + chunk * E of the stage; unused halo slots are never read.
// Global offsets are 32-bit (the library caps the lattice so that 13 planes
// stay below 2^31 elements).
template <class S, int NV>
struct CopyPlan {
    using Wn = Win<S, NV>;
    static constexpr int OPP = 32 * NV / Wn::E;  // own chunks per plane
    static constexpr int OWN = 13 * OPP;
    static constexpr int TOTAL = OWN + 12;
    static constexpr int PER_LANE = (TOTAL + 31) / 32;
    static_assert(32 % OPP == 0, "own chunks of a plane must tile a warp's lanes");
    static_assert(32 * (PER_LANE - 1) <= OWN, "only the last copy of a lane may be a halo chunk");
    int goff[PER_LANE];  // element offset in the source buffer (row 0)
    int sbase;           // stage element of this lane's own chunk in copy 0
    int slast;           // stage element of this lane's chunk in copy PER_LANE - 1
};

// plane of halo chunk h: left halos (window chunk 0) for h < 6, right halos
// (last window chunk) for h >= 6
__device__ __forceinline__ int halo_plane(int h)
{
    constexpr unsigned long long packed = 1ull | (2ull << 4) | (4ull << 8) | (5ull << 12) | (8ull << 16) |
                                          (9ull << 20) | (2ull << 24) | (3ull << 28) | (4ull << 32) |
                                          (6ull << 36) | (7ull << 40) | (11ull << 44);
    return (int)((packed >> (4 * h)) & 15ull);
}

template <class S, int NV>
__device__ __forceinline__ void chunk_of(int t, int &q, int &c)
{
    using CP = CopyPlan<S, NV>;
    if (t < CP::OWN) {
        q = t / CP::OPP;
        c = 1 + t % CP::OPP;
    } else {
        const int h = t - CP::OWN;
        q = halo_plane(h);
        c = h < 6 ? 0 : Win<S, NV>::CH - 1;
    }
}

template <class S, int NV, class C>
__device__ __forceinline__ CopyPlan<S, NV> make_copy_plan(const StepParams<C> &p, int x0, int lane)
{
    using Wn = Win<S, NV>;
    using CP = CopyPlan<S, NV>;
    CP cp;
#pragma unroll
    for (int m = 0; m < CP::PER_LANE; ++m) {
        int q, c;
        chunk_of<S, NV>(min(lane + 32 * m, CP::TOTAL - 1), q, c);
        cp.goff[m] = q * (int)p.plane - plane_ey(q) * p.pitch + (x0 - Wn::H + c * Wn::E + PAD_COLS);
        if (m == CP::PER_LANE - 1)
            cp.slast = q * Wn::W + c * Wn::E;
    }
    cp.sbase = (lane / CP::OPP) * Wn::W + (1 + lane % CP::OPP) * Wn::E;
    return cp;
}

// start the copies of lattice row r into one stage (CP: a copy plan with
// the members of CopyPlan)
template <class S, int NV, class C, class CP>
__device__ __forceinline__ void issue_row(const StepParams<C> &p, const S *src, S *stage, const CP &cp, int r, int lane)
{
    const int row = (r + 1) * p.pitch;
#pragma unroll
    for (int m = 0; m < CP::PER_LANE; ++m) {
        // copies before the last hold own chunks only: 32 m / OPP whole planes further on
        const int so = (m < CP::PER_LANE - 1) ? cp.sbase + (32 * m / CP::OPP) * Win<S, NV>::W : cp.slast;
        if (m < CP::PER_LANE - 1 || lane + 32 * m < CP::TOTAL)
            cp_async16(stage + so, src + (unsigned)(row + cp.goff[m]));
    }
}

// population q of strip column col (-1 and 32 NV are the columns beside the strip)
template <class S, int NV, class C>
__device__ __forceinline__ C sget(const S *stage, int q, int ex, int col)
{
    using Wn = Win<S, NV>;
    return load_as_shared<S, C>(stage + q * Wn::W + col + Wn::H - ex);
}

// Moment-split storage: the moment rows are staged too, each lattice row
// once, into a per-warp ring of MSLOTS slots; a slot holds one row's
// (j_x, j_r) pairs and its T - T0 over the strip's columns and MH columns
// on each side.  A row's populations come from sources in rows r - 1, r and
// r + 1, so the pull of row r reads three slots: the (j_x, j_r) pairs of
// the eight neighbours and T - T0 of the four axis neighbours, twelve
// shared-memory loads per node.
template <int NV> struct MWin {
    static constexpr int H = 4;                // halo columns on each side
    static constexpr int W = 32 * NV + 2 * H;  // window length (columns)
    static constexpr int JCH = W / 2;          // 16-byte chunks of the (j_x, j_r) window
    static constexpr int TCH = W / 4;          // 16-byte chunks of the T window
    static constexpr int SLOT = 3 * W;         // floats per slot: W pairs, then W values of T
};
constexpr int MSLOTS = 5;  // moment rows r - 2 .. r + 2 around the row whose moments are formed

// this lane's view of the staged moment windows of rows r - 1, r, r + 1
// (null for other storage types): element col of a window is strip column
// lane + col
template <int NV>
struct MRows {
    const float2 *j[3];
    const float *T[3];
};

template <int NV>
__device__ __forceinline__ MRows<NV> mrows_at(const float *const (&slot)[3], int lane)
{
    MRows<NV> m;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        m.j[k] = reinterpret_cast<const float2 *>(slot[k]) + lane + MWin<NV>::H;
        m.T[k] = slot[k] + 2 * MWin<NV>::W + lane + MWin<NV>::H;
    }
    return m;
}

// start the copies of moment row r into a slot
template <int NV, class C>
__device__ __forceinline__ void issue_mrow(const StepParams<C> &p, const float *M, float *slot, int x0, int r, int lane)
{
    using MW = MWin<NV>;
    const int c0 = (r + 1) * p.pitch + x0 - MW::H + PAD_COLS;  // element offset of the window's first cell
#pragma unroll
    for (int t0 = 0; t0 < MW::JCH + MW::TCH; t0 += 32) {
        const int t = t0 + lane;
        if (t < MW::JCH)
            cp_async16(slot + 4 * t, M + (unsigned)(2 * c0 + 4 * t));
        else if (t < MW::JCH + MW::TCH)
            cp_async16(slot + 2 * MW::W + 4 * (t - MW::JCH), M + (unsigned)(2 * (int)p.plane + c0 + 4 * (t - MW::JCH)));
    }
}

// population q of strip column lane + off pulled from the stage, with (moment-split
// storage) its linear part at the source's moments
template <class S, int NV, class C>
__device__ __forceinline__ C spop(const StepParams<C> &p, const S *stage, const MRows<NV> &mr, int q, int lane, int off)
{
    const int ex = qex(q), ey = qey(q);
    C v = sget<S, NV, C>(stage, q, ex, lane + off);
    if constexpr (IsSplit<S>::value) {
        const float2 jj = mr.j[1 - ey][off - ex];
        v += lin_part<C>(p, q, jj.x, jj.y, q < 9 ? C(0) : mr.T[1 - ey][off - ex]);
    }
    return v;
}

template <class S, int NV, class C>
__device__ __forceinline__ void stage_pops(const StepParams<C> &p, const S *stage, const MRows<NV> &mr, int lane,
                                           Vec<C, NV> (&f)[9], Vec<C, NV> (&g)[4])
{
    using V = Vec<C, NV>;
#pragma unroll
    for (int c = 0; c < NV; ++c) {
#pragma unroll
        for (int k = 0; k < 9; ++k)
            f[k].set(c, sget<S, NV, C>(stage, k, ex9(k), lane + 32 * c));
#pragma unroll
        for (int k = 0; k < 4; ++k)
            g[k].set(c, sget<S, NV, C>(stage, 9 + k, ex4(k), lane + 32 * c));
    }
    if constexpr (IsSplit<S>::value) {
        // the linear parts, from the (j_x, j_r) pairs of the eight neighbours and T - T0 of
        // the four axis neighbours (row index 0: r - 1, the source of upward populations)
        V wx, ex_, sy, ny, swx, swy, sex, sey, nex, ney, nwx, nwy, tw, ts, te, tn;
#pragma unroll
        for (int c = 0; c < NV; ++c) {
            const int o = 32 * c;
            const float2 w = mr.j[1][o - 1], e = mr.j[1][o + 1], sj = mr.j[0][o], nj = mr.j[2][o];
            const float2 sw = mr.j[0][o - 1], se = mr.j[0][o + 1], ne = mr.j[2][o + 1], nw = mr.j[2][o - 1];
            wx.set(c, w.x);
            ex_.set(c, e.x);
            sy.set(c, sj.y);
            ny.set(c, nj.y);
            swx.set(c, sw.x);
            swy.set(c, sw.y);
            sex.set(c, se.x);
            sey.set(c, se.y);
            nex.set(c, ne.x);
            ney.set(c, ne.y);
            nwx.set(c, nw.x);
            nwy.set(c, nw.y);
            tw.set(c, mr.T[1][o - 1]);
            te.set(c, mr.T[1][o + 1]);
            ts.set(c, mr.T[0][o]);
            tn.set(c, mr.T[2][o]);
        }
        constexpr C a1 = C(3) * w9<C>(1), a2 = C(3) * w9<C>(5);
        f[1] = vfma(V(a1), wx, f[1]);                    // e = (1, 0), from x - 1
        f[3] = vfma(V(-a1), ex_, f[3]);                  // e = (-1, 0), from x + 1
        f[2] = vfma(V(a1), sy, f[2]);                    // e = (0, 1), from r - 1
        f[4] = vfma(V(-a1), ny, f[4]);                   // e = (0, -1), from r + 1
        f[5] = vfma(V(a2), swx + swy, f[5]);             // e = (1, 1)
        f[6] = vfma(V(a2), sey - sex, f[6]);             // e = (-1, 1)
        f[7] = vfma(V(-a2), nex + ney, f[7]);            // e = (-1, -1)
        f[8] = vfma(V(a2), nwx - nwy, f[8]);             // e = (1, -1)
        const V T0(p.T0), h(p.hir0), q4(C(0.25));
        g[0] = vfma(q4, tw, vfma((T0 + tw) * h, wx, g[0]));    // e = (1, 0)
        g[1] = vfma(q4, ts, vfma((T0 + ts) * h, sy, g[1]));    // e = (0, 1)
        g[2] = vfma(q4, te, vfma(-((T0 + te) * h), ex_, g[2]));  // e = (-1, 0)
        g[3] = vfma(q4, tn, vfma(-((T0 + tn) * h), ny, g[3]));   // e = (0, -1)
    }
}

// rho u_r of the streamed populations in strip column lane + off of a stage
template <class S, int NV, class C>
__device__ __forceinline__ C stage_jr(const StepParams<C> &p, const S *stage, const MRows<NV> &mr, int lane, int off)
{
    return (spop<S, NV, C>(p, stage, mr, 2, lane, off) - spop<S, NV, C>(p, stage, mr, 4, lane, off)) +
           (spop<S, NV, C>(p, stage, mr, 5, lane, off) - spop<S, NV, C>(p, stage, mr, 8, lane, off)) +
           (spop<S, NV, C>(p, stage, mr, 6, lane, off) - spop<S, NV, C>(p, stage, mr, 7, lane, off));
}

// ---- the fused step kernel ------------------------------------------------------------
// collide row j of the tile from its stage and write it (and its ghosts); kf, kg
// are the row's populations when the caller already pulled them
template <class S, int NV, class C>
__device__ __forceinline__ void collide_row(const StepParams<C> &p, const S *src, S *__restrict__ dst, const S *st,
                                            const MRows<NV> &mr, int x0, int lane, int j, int64_t t,
                                            const Mom<Vec<C, NV>> &mp, const Mom<Vec<C, NV>> &mc,
                                            const Mom<Vec<C, NV>> &mn, const float2 *stab,
                                            const Vec<C, NV> *kf = nullptr, const Vec<C, NV> *kg = nullptr)
{
    using V = Vec<C, NV>;
    // axial neighbours of rho u_r: the strip's columns form one sequence
    // c = lane + 32 v; its ends read the staged halo, the lattice ends the
    // boundary's ghost moments
    V left, right;
    // rho u_r beside the strip, computed by every lane for its half's side
    // (lanes 0..15 the left, 16..31 the right) in one warp-uniform pass
    const C beside = stage_jr<S, NV, C>(p, st, mr, lane, (lane < 16 ? -1 : 32 * NV) - lane);
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
        if (i == 0)
            l = jr_beyond_inlet<S, C>(p, src, j);
        if (i == p.nx - 1)
            r = jr_beyond_outlet<S, C>(p, src, j, mc.jr[c]);
        left.set(c, l);
        right.set(c, r);
    }
    if (x0 + lane >= p.nx)
        return;  // no active node in this lane
    V f[9], g[4], fo[9], go[4];
    if (kf) {
#pragma unroll
        for (int k = 0; k < 9; ++k)
            f[k] = kf[k];
#pragma unroll
        for (int k = 0; k < 4; ++k)
            g[k] = kg[k];
    } else {
        stage_pops<S, NV, C>(p, st, mr, lane, f, g);
    }
    const C inv_r = C(1) / (p.r0 + C(j) + C(0.5));
    collide<C, V>(p, f, g, mc, inv_r, C(0.5) * (mn.jx - mp.jx), C(0.5) * (mn.jr - mp.jr), C(0.5) * (right - left),
                  C(0.5) * (mn.dT - mp.dT), fo, go, stab);
    const unsigned pl = (unsigned)p.plane;
#pragma unroll
    for (int c = 0; c < NV; ++c) {
        const int i = x0 + lane + 32 * c;
        if (i < p.nx) {
            const unsigned o = (unsigned)((j + 1) * p.pitch + i + PAD_COLS);
            if constexpr (IsSplit<S>::value) {
                // the node's pre-collision moments, and every population as its deviation
                // from the linear part at them
                const C jx = mc.jx[c], jr = mc.jr[c], dT = mc.dT[c];
                const MomRef M{split_m(dst, p.plane), p.plane};
                M.j(o) = make_float2(jx, jr);
                M.T(o) = dT;
#pragma unroll
                for (int k = 0; k < 9; ++k)
                    dst[o + k * pl] = store_as<S, C>(fo[k][c] - lin_part<C>(p, k, jx, jr, dT));
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    dst[o + (9 + k) * pl] = store_as<S, C>(go[k][c] - lin_part<C>(p, 9 + k, jx, jr, dT));
            } else {
#pragma unroll
                for (int k = 0; k < 9; ++k)
                    dst[o + k * pl] = store_as<S, C>(fo[k][c]);
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    dst[o + (9 + k) * pl] = store_as<S, C>(go[k][c]);
            }
            if (i == 0 || i == p.nx - 1 || j == 0 || j == p.nr - 1)
                write_ghosts<S, C>(p, dst, i, j, t + 1);
        }
    }
}

// One warp tile: columns x0..x0+32 NV-1 of rows j0..j1-1.  Rows j0-1 (if
// any) through min(j1, nr-1) are staged one after the other, NSTAGE - 2
// rows ahead of the one whose moments are being formed; a row is collided
// once the moments of the rows on both sides of it exist.  (The stage being
// refilled is never one of the two being read: it held row idx - 2.)
//
// FP32 storage: even bands march upwards and odd bands downwards.  The two
// rows that neighbouring bands share (each one's last own row and the
// other's halo row) are then staged by both tiles at the same end of their
// work, a fraction of a microsecond apart (the tiles of one strip are one
// band of work items apart), so the second read finds them in L2.  With
// one direction the second read came a whole tile later, after some 90 MB
// of other traffic, and about a fifth of them went to DRAM again.  The
// 2-byte kernels, bound by instruction issue, keep one direction.
//
// Moment-split storage also stages moment rows rfirst - 1 .. min(j1, nr -
// 1) + 1 into the warp's ring msm, one row further ahead (row r + 1 lands
// with the populations of row r); the slot refilled held row r - 3.
template <class S, int NV, class C>
__device__ __forceinline__ void step_tile(const StepParams<C> &p, const S *__restrict__ src, S *__restrict__ dst,
                                          S *wsm, int tile, int lane, int64_t t, const float2 *stab = nullptr,
                                          float *msm = nullptr)
{
    using Wn = Win<S, NV>;
    using V = Vec<C, NV>;
    constexpr int NSTAGE = step_stages<S, NV>();
    constexpr int D = NSTAGE - 2;
    constexpr bool SPLIT = IsSplit<S>::value;
    constexpr bool ALT = std::is_same<S, float>::value;  // alternating band directions
    static_assert(!SPLIT || D == 1, "the moment ring assumes populations staged one row ahead");
    const int strip = tile % p.nstrips;
    const int band = tile / p.nstrips;
    const int x0 = strip * 32 * NV;
    const int j0 = band * p.band;
    const int j1 = min(j0 + p.band, p.nr);
    const int rlo = j0 > 0 ? j0 - 1 : j0;  // rows staged: rlo .. rhi
    const int rhi = min(j1, p.nr - 1);
    const int nrows = rhi - rlo + 1;
    const bool down = ALT && (band & 1) != 0;
    const int rstart = down ? rhi : rlo;
    const int dr = down ? -1 : 1;
    const int first_own = down ? j1 - 1 : j0;            // first row of the band reached
    const bool edge_first = down ? j1 == p.nr : j0 == 0;  // the lattice ends beyond it
    const bool edge_last = down ? j0 == 0 : j1 == p.nr;   // ... beyond the last one
    const CopyPlan<S, NV> plan = make_copy_plan<S, NV, C>(p, x0, lane);
    const float *M = nullptr;
    if constexpr (SPLIT)
        M = split_m(src, p.plane);
    // moment row m lives in slot (m - rlo + 1) % MSLOTS
    auto mslot = [&](int m) { return msm + ((m - rlo + 1) % MSLOTS) * MWin<NV>::SLOT; };
    auto mrows = [&](int r) {
        MRows<NV> mr = {};
        if constexpr (SPLIT) {
            const float *sl[3] = {mslot(r - 1), mslot(r), mslot(r + 1)};
            mr = mrows_at<NV>(sl, lane);
        }
        return mr;
    };

    if constexpr (SPLIT) {  // moment rows rlo - 1 .. rlo + 1 join the first group
        for (int m = rlo - 1; m <= rlo + 1; ++m)
            issue_mrow<NV, C>(p, M, mslot(m), x0, m, lane);
    }
#pragma unroll
    for (int t = 0; t < D; ++t) {
        if (t < nrows)
            issue_row<S, NV, C>(p, src, wsm + t * Wn::STAGE, plan, rstart + dr * t, lane);
        cp_async_commit();
    }
    Mom<V> mb, mc;  // moments of the row passed before the current one, and of the current one
    // Moment-split tiles keep the populations decoded for a row's moments in
    // registers for its collision one row later, instead of decoding the staged
    // row a second time.  It costs registers (two nodes per lane: 164, so 12
    // warps per SM instead of 16) and saves more: the ragged 256-jet ensemble
    // with one node per lane 721 -> 648 us per step, the 4096 x 1024 jet with
    // two 95 -> 89 us.
    constexpr bool KEEP = SPLIT;
    V kf[9], kg[4];  // the populations of the row passed last (KEEP)
#pragma unroll 1
    for (int idx = 0; idx < nrows; ++idx) {
        __syncwarp();  // every lane is done with the stage refilled next
        if (idx + D < nrows)
            issue_row<S, NV, C>(p, src, wsm + ((idx + D) % NSTAGE) * Wn::STAGE, plan, rstart + dr * (idx + D), lane);
        if constexpr (SPLIT) {
            if (idx + D < nrows)  // moment rows up to the last staged row + 1 (at most the ghost row nr)
                issue_mrow<NV, C>(p, M, mslot(rlo + idx + D + 1), x0, rlo + idx + D + 1, lane);
        }
        cp_async_commit();
        cp_async_wait<D>();
        __syncwarp();  // row idx has landed for every lane
        const int r = rstart + dr * idx;
        const S *st = wsm + (idx % NSTAGE) * Wn::STAGE;
        V f[9], g[4];
        stage_pops<S, NV, C>(p, st, mrows(r), lane, f, g);
        const Mom<V> mr = moments<V>(f, g);
        if (r == first_own) {
            if (edge_first)
                mb = down ? ghost_top<C, V>(p, mr) : ghost_bottom<C, V>(p, mr);
            mc = mr;
        } else if (idx == 0) {  // the halo row
            mb = mr;
        } else {
            collide_row<S, NV, C>(p, src, dst, wsm + ((idx - 1) % NSTAGE) * Wn::STAGE, mrows(r - dr), x0, lane,
                                  r - dr, t, down ? mr : mb, mc, down ? mb : mr, stab, KEEP ? kf : nullptr,
                                  KEEP ? kg : nullptr);
            mb = mc;
            mc = mr;
        }
        if constexpr (KEEP) {
#pragma unroll
            for (int k = 0; k < 9; ++k)
                kf[k] = f[k];
#pragma unroll
            for (int k = 0; k < 4; ++k)
                kg[k] = g[k];
        }
    }
    if (edge_last)
        collide_row<S, NV, C>(p, src, dst, wsm + ((nrows - 1) % NSTAGE) * Wn::STAGE, mrows(down ? 0 : p.nr - 1), x0,
                              lane, down ? 0 : p.nr - 1, t, down ? ghost_bottom<C, V>(p, mc) : mb, mc,
                              down ? mb : ghost_top<C, V>(p, mc), stab, KEEP ? kf : nullptr, KEEP ? kg : nullptr);
    cp_async_wait<0>();
    __syncwarp();
}

template <class S, class C, int NV = NodesPerLane<C>::value>
constexpr int pop_ring_bytes()
{
    return step_stages<S, NV>() * Win<S, NV>::STAGE * (int)sizeof(S);
}

template <class S, class C, int NV = NodesPerLane<C>::value>
constexpr int step_smem_per_warp()
{
    return pop_ring_bytes<S, C, NV>() + (IsSplit<S>::value ? MSLOTS * MWin<NV>::SLOT * (int)sizeof(float) : 0);
}

// shared memory of a step_run_kernel CTA: the warps' rings, then (2-byte
// storage) the property table
template <class S, class C, int NV = NodesPerLane<C>::value>
constexpr int run_smem(int warps)
{
    return warps * step_smem_per_warp<S, C, NV>() + (UseSmemTable<S, C>::value ? SMEM_TAB * (int)sizeof(float2) : 0);
}

// ---- many steps of one lattice in one launch ----------------------------------------
// lbm_step runs all its steps in one persistent launch.  A work item is a
// group of G adjacent warp tiles of one band (strips g G .. g G + G - 1);
// warps take items from a counter in step-major order (item n = k * items
// + i for sub-step k) and run the group's tiles one after the other.  An
// item of sub-step k > 0 reads what the items around it wrote in sub-step
// k - 1 and overwrites what they read there: rows within one band (two
// bands for one-row bands) and columns within one strip beyond the group
// (wrapping around for periodic ends).  So before starting it waits until
// those neighbour items count sub-step k - 1 as done.  Each lane adds one
// to its item's counter with release semantics after its last store, so an
// item is done with sub-step k - 1 once its counter reaches 32 k.  To wait,
// lane l watches one neighbour counter with acquire loads; a warp barrier
// (which orders memory among its lanes) then hands the acquired view to
// every lane.  Every neighbour item precedes the waiting one in the counter
// order, so it was taken by a warp that is already running; a warp works on
// its items in counter order, and the lowest unfinished item never waits on
// a later one, so the waits end.  Each wait is bounded all the same; a
// wait that runs out raises LBM_STATUS_TIMEOUT in the lattice's status
// word and the warps stop taking work.
constexpr int STATUS_TIMEOUT = 1;
constexpr int RUN_SPIN_LIMIT = 1 << 21;  // polls of at most ~2 us: a few seconds

struct RunCtl {
    unsigned *counter;  // work items taken (zeroed before the launch; step_run_kernel: at cbase)
    unsigned *flags;    // per work item: 32 x sub-steps done (zeroed before the launch; step_run_kernel: at fbase)
    int nsteps;         // sub-steps of this launch
    int radius;         // neighbour bands an item depends on
    int wrap;           // strips wrap around (periodic axial ends; a batch reads each lattice's ends)
    int group;          // G: warp tiles (adjacent strips of one band) per work item
    int spin_limit;     // polls before a wait gives up (RUN_SPIN_LIMIT; smaller in the self-test)
    // step_run_kernel only.  Its counters carry on from launch to launch: the work
    // counter ends a launch advanced by exactly nsteps x items + the grid's warps
    // (below), and every item's completion counter by 32 (nsteps - 1), since nothing
    // in a launch waits for its last sub-step.  The host tracks both, so consecutive
    // launches need no reset between them.
    unsigned cbase = 0;  // the work counter's value at the start of the launch
    unsigned fbase = 0;  // every completion counter's value at the start of the launch
    unsigned first = 0;  // the first work item of the launch (0; the self-test starts at sub-step 1)
};

// work items per band of a lattice with nstrips strips
__host__ __device__ __forceinline__ int item_cols(int nstrips, int group) { return (nstrips + group - 1) / group; }

__device__ __forceinline__ unsigned ld_acquire(const unsigned *a)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];\n" : "=r"(v) : "l"(a) : "memory");
    return v;
}

__device__ __forceinline__ void red_release_add(unsigned *a, unsigned v)
{
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;\n" ::"l"(a), "r"(v) : "memory");
}

// Every lane waits until the items around item (band b, column g) of a
// lattice (its counters start at `flags`, `cols` items per band, each at
// `base` before sub-step 0) have
// finished sub-step k - 1: radius bands and one item column on each side,
// and also the items two columns out when `far`.  Returns false if the
// wait runs out or another warp's wait ran out (the status word is read
// only while waiting).
template <class C>
__device__ bool wait_neighbours(const StepParams<C> &p, const unsigned *flags, int cols, int radius, bool wrap, int b,
                                int g, int k, int spin_limit, bool far = false, unsigned base = 0)
{
    // lane l < 3 (2 radius + 1) watches neighbour (band b + l / 3 - radius, column g + l % 3 - 1);
    // when far, lane 16 + m < 16 + 2 (2 radius + 1) watches (band b + m / 2 - radius, column g -+ 2)
    const int nbands = (p.nr + p.band - 1) / p.band;
    const int lane = threadIdx.x & 31;
    const unsigned *f = nullptr;
    if (lane < 3 * (2 * radius + 1)) {
        const int bb = b + lane / 3 - radius;
        int gg = g + lane % 3 - 1;
        if (wrap)
            gg = gg < 0 ? gg + cols : (gg >= cols ? gg - cols : gg);
        if (bb >= 0 && bb < nbands && gg >= 0 && gg < cols)
            f = flags + bb * cols + gg;
    } else if (far && lane >= 16 && lane < 16 + 2 * (2 * radius + 1)) {
        const int bb = b + (lane - 16) / 2 - radius;
        int gg = g + ((lane & 1) ? 2 : -2);
        gg = gg < 0 ? gg + cols : (gg >= cols ? gg - cols : gg);
        if (bb >= 0 && bb < nbands && gg >= 0 && gg < cols)
            f = flags + bb * cols + gg;
    }
    const unsigned want = base + 32u * (unsigned)k;
    for (int it = 0;; ++it) {
        const bool ok = f == nullptr || (int)(ld_acquire(f) - want) >= 0;
        if (__all_sync(0xffffffffu, ok)) {
            __syncwarp();  // orders memory among the lanes: every lane now sees what its watcher acquired
            return true;
        }
        if (it >= spin_limit || (*static_cast<volatile int *>(p.status) & STATUS_TIMEOUT))
            return false;
        __nanosleep(it < 8 ? 64 : (it < 64 ? 512 : 2048));
    }
}

// With periodic ends and a last strip of one column (nx - 1 a multiple of
// the strip width), the pulled moments of column nx - 1 read column nx - 2
// and the periodic ghost column nx, which strip 0 writes.  The strip before
// the last one takes them for its right neighbour column, strip 0 for the
// periodic neighbour of column 0: with four strips or more these tiles are
// two strips apart across the wrap, so their items also wait for the items
// two columns out.  The step kernels take this path only in their FAR
// instantiation, which the host launches for such lattices alone: every
// other launch runs the one-column wait unchanged.
__host__ __device__ constexpr bool far_wrap(int bc_in, int nx, int nstrips, int strip_cols)
{
    return bc_in == IN_PERIODIC && (nx - 1) % strip_cols == 0 && nstrips >= 4;
}

template <int NV, class C>
__device__ __forceinline__ bool far_wrap(const StepParams<C> &p)
{
    return far_wrap(p.bc_in, p.nx, p.nstrips, 32 * NV);
}

template <class S, class C, bool FAR = false, int NV = NodesPerLane<C>::value>
__global__ void __launch_bounds__(256) step_run_kernel(const __grid_constant__ StepParams<C> p, const RunCtl ctl)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    unsigned char *wbase = smem_raw + (size_t)warp * step_smem_per_warp<S, C, NV>();
    S *wsm = reinterpret_cast<S *>(wbase);
    float *msm = IsSplit<S>::value ? reinterpret_cast<float *>(wbase + pop_ring_bytes<S, C, NV>()) : nullptr;
    const float2 *stab = nullptr;
    if constexpr (UseSmemTable<S, C>::value) {
        if (p.ntab > 1 && p.ntab <= SMEM_TAB) {
            float2 *tab = reinterpret_cast<float2 *>(smem_raw + (blockDim.x >> 5) * step_smem_per_warp<S, C, NV>());
            load_smem_table(p, tab);
            __syncthreads();
            stab = tab;
        }
    }
    const int cols = item_cols(p.nstrips, ctl.group);
    const unsigned items = (unsigned)cols * (unsigned)((p.nr + p.band - 1) / p.band);
    const unsigned total = (unsigned)ctl.nsteps * items;
    // Every warp draws from the counter once, then once per item it runs (its
    // last draw is past the end), so the counter ends the launch at
    // cbase + total + the grid's warps.  (Handing each warp its first item by
    // its index instead put the 4096 x 1024 jet into a steady schedule 8%
    // slower: which warps meet which items first shapes the whole launch.)
    unsigned n = 0;
    if (lane == 0)
        n = ctl.first + (atomicAdd(ctl.counter, 1u) - ctl.cbase);
    n = __shfl_sync(0xffffffffu, n, 0);
    while (n < total) {
        // take the next item now: its latency hides behind this one
        unsigned next = 0;
        if (lane == 0)
            next = ctl.first + (atomicAdd(ctl.counter, 1u) - ctl.cbase);
        const int k = (int)(n / items);
        const int item = (int)(n - (unsigned)k * items);
        const int b = item / cols, g = item - b * cols;
        if (k > 0 && !wait_neighbours<C>(p, ctl.flags, cols, ctl.radius, ctl.wrap != 0, b, g, k, ctl.spin_limit,
                                         FAR && far_wrap<NV>(p), ctl.fbase)) {
            if (lane == 0)
                atomicOr(p.status, STATUS_TIMEOUT);
            break;  // whole warp
        }
        const S *src = static_cast<const S *>((k & 1) ? p.dst : p.src);
        S *dst = static_cast<S *>((k & 1) ? const_cast<void *>(p.src) : p.dst);
        const int s1 = min((g + 1) * ctl.group, p.nstrips);
        for (int s = g * ctl.group; s < s1; ++s)
            step_tile<S, NV, C>(p, src, dst, wsm, b * p.nstrips + s, lane, p.step + k, stab, msm);
        if (k + 1 < ctl.nsteps)  // no item of this launch waits for the last sub-step
            red_release_add(ctl.flags + item, 1u);
        n = __shfl_sync(0xffffffffu, next, 0);
    }
}

// ---- many lattices in one launch --------------------------------------------------------
// A batch of independent lattices of any sizes (same storage type) runs
// many steps in one persistent launch, exactly like one lattice: a table
// lists every warp tile of every member as (lattice, tile of that lattice),
// and work item n of a launch is sub-step n / T (T table entries) of entry
// n % T.  Each entry has its own completion counter; the counters of one
// lattice are consecutive (its entries are), so a tile finds its
// neighbours' counters from its own entry index.  Each warp copies its
// lattice's parameters from the batch's parameter table into shared memory.
// After the launch the parameters (buffers, step counter) advance on the
// device (advance_kernel), so a captured launch can be replayed.
struct TileRef {
    int lattice;  // index in the batch's parameter table
    int tile;     // warp tile index within that lattice
};

template <class S, class C, bool FAR = false, int NV = NodesPerLane<C>::value>
__global__ void __launch_bounds__(256) batch_run_kernel(const TileRef *__restrict__ tiles, int ntiles,
                                                        const StepParams<C> *__restrict__ lattices, const RunCtl ctl)
{
    constexpr int PW = (int)((sizeof(StepParams<C>) + 15) / 16);  // 16-byte words per parameter block
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int wpc = blockDim.x >> 5;
    // parameter blocks of all warps first, then the warps' staging rings
    StepParams<C> *pw = reinterpret_cast<StepParams<C> *>(smem_raw) + warp;
    unsigned char *wbase = smem_raw + wpc * sizeof(StepParams<C>) + (size_t)warp * step_smem_per_warp<S, C, NV>();
    S *wsm = reinterpret_cast<S *>(wbase);
    float *msm = IsSplit<S>::value ? reinterpret_cast<float *>(wbase + pop_ring_bytes<S, C, NV>()) : nullptr;
    static_assert(sizeof(StepParams<C>) % 16 == 0 && PW <= 32, "parameter block copy");
    const unsigned total = (unsigned)ctl.nsteps * (unsigned)ntiles;
    unsigned n = 0;
    if (lane == 0)
        n = atomicAdd(ctl.counter, 1u);
    n = __shfl_sync(0xffffffffu, n, 0);
    while (n < total) {
        unsigned next = 0;
        if (lane == 0)
            next = atomicAdd(ctl.counter, 1u);
        const int k = (int)(n / (unsigned)ntiles);
        const int idx = (int)(n - (unsigned)k * (unsigned)ntiles);
        const TileRef t = tiles[idx];
        __syncwarp();  // every lane is done with the previous parameter block
        if (lane < PW)
            reinterpret_cast<uint4 *>(pw)[lane] = reinterpret_cast<const uint4 *>(lattices + t.lattice)[lane];
        __syncwarp();
        const StepParams<C> &p = *pw;
        if (k > 0 && !wait_neighbours<C>(p, ctl.flags + (idx - t.tile), p.nstrips, ctl.radius, p.bc_in == IN_PERIODIC,
                                         t.tile / p.nstrips, t.tile % p.nstrips, k, ctl.spin_limit,
                                         FAR && far_wrap<NV>(p))) {
            if (lane == 0)
                atomicOr(p.status, STATUS_TIMEOUT);
            break;  // whole warp
        }
        const S *src = static_cast<const S *>((k & 1) ? p.dst : p.src);
        S *dst = static_cast<S *>((k & 1) ? const_cast<void *>(p.src) : p.dst);
        step_tile<S, NV, C>(p, src, dst, wsm, t.tile, lane, p.step + k, nullptr, msm);
        red_release_add(ctl.flags + idx, 1u);
        n = __shfl_sync(0xffffffffu, next, 0);
    }
}

template <class S, class C, int NV = NodesPerLane<C>::value>
constexpr int batch_smem_per_warp()
{
    return step_smem_per_warp<S, C, NV>() + (int)sizeof(StepParams<C>);
}

// after a batch launch of nsteps steps: every lattice counts the steps and,
// for an odd count, swaps its buffers
template <class C>
__global__ void advance_kernel(StepParams<C> *lattices, int n, int nsteps)
{
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= n)
        return;
    StepParams<C> &p = lattices[m];
    if (nsteps & 1) {
        const void *s = p.src;
        p.src = p.dst;
        p.dst = const_cast<void *>(s);
    }
    p.step += nsteps;
}

// ---- ghosts of a stored state (after it is set from outside) ------------------------
template <class S, class C>
__global__ void fill_ghosts_kernel(const __grid_constant__ StepParams<C> p)
{
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= (int64_t)p.nx * p.nr)
        return;
    const int i = (int)(n % p.nx), j = (int)(n / p.nx);
    if (!(i == 0 || i == p.nx - 1 || j == 0 || j == p.nr - 1))
        return;
    write_ghosts<S, C>(p, static_cast<S *>(p.dst), i, j, p.step);
}

// ---- fields at the current time: Eq. 2 moments of the streamed populations ---------------
template <class S, class C, class O>
__global__ void fields_kernel(const __grid_constant__ StepParams<C> p, O *out)
{
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t N = (int64_t)p.nx * p.nr;
    if (n >= N)
        return;
    const int i = (int)(n % p.nx), j = (int)(n / p.nx);
    const Mom<Vec<C, 1>> m = node_moments<S, C>(p, i, j, false);
    const C rho = p.rho0 + m.drho.x;
    out[n] = O(rho);
    out[N + n] = O(m.jx.x / rho);
    out[2 * N + n] = O(m.jr.x / rho);
    out[3 * N + n] = O(p.T0 + m.dT.x);
}

// ---- FP64 diagnostics: mass, heat, steady residual, divergence -------------------------
// Per node, from the populations streamed from the current state (and from
// the previous state in the other buffer): rho, u, T of Eq. 2.  Sums run in
// FP64: Σ rho, Σ r rho, Σ T, Σ r T, Σ |u(t) - u(t-1)|^2, Σ |u(t)|^2,
// max |u(t) - u(t-1)|, max |u(t)|, and the count of nodes whose rho is not
// finite and positive or whose T is not finite.  Block partials go to
// `partials` (DIAG_SLOTS doubles per block); diag_final_kernel folds them.
constexpr int DIAG_SLOTS = 9;
constexpr int DIAG_THREADS = 256;

__device__ __forceinline__ void diag_combine(double *a, const double *b)
{
    for (int k = 0; k < 5; ++k)
        a[k] += b[k];
    a[5] = fmax(a[5], b[5]);
    a[6] = fmax(a[6], b[6]);
    a[7] += b[7];
    a[8] += b[8];
}

// block-wide combine of per-thread slots through shared memory; thread 0 ends with the result
__device__ __forceinline__ void diag_block_reduce(double (&v)[DIAG_SLOTS])
{
    __shared__ double sh[DIAG_THREADS / 32][DIAG_SLOTS];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int off = 16; off > 0; off >>= 1) {
        double o[DIAG_SLOTS];
        for (int k = 0; k < DIAG_SLOTS; ++k)
            o[k] = __shfl_down_sync(0xffffffffu, v[k], off);
        diag_combine(v, o);
    }
    if (lane == 0)
        for (int k = 0; k < DIAG_SLOTS; ++k)
            sh[warp][k] = v[k];
    __syncthreads();
    if (threadIdx.x == 0)
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
            diag_combine(v, sh[w]);
}

// adds node (i, j) to the per-thread slots
template <class S, class C>
__device__ __forceinline__ void diag_node(const StepParams<C> &p, int have_prev, int i, int j, double (&v)[DIAG_SLOTS])
{
    const Mom<Vec<C, 1>> m = node_moments<S, C>(p, i, j, false);
    const double rho = (double)p.rho0 + (double)m.drho.x;
    const double T = (double)p.T0 + (double)m.dT.x;
    const double ux = (double)m.jx.x / rho, ur = (double)m.jr.x / rho;
    const double r = (double)p.r0 + j + 0.5;
    if (!(rho > 0.0) || !isfinite(rho) || !isfinite(T) || !isfinite(ux) || !isfinite(ur)) {
        v[7] += 1.0;
        return;
    }
    v[0] += rho;
    v[1] += r * rho;
    v[2] += T;
    v[3] += r * T;
    const double uu = ux * ux + ur * ur;
    v[8] += uu;
    v[6] = fmax(v[6], sqrt(uu));
    if (have_prev) {
        const Mom<Vec<C, 1>> q = node_moments<S, C>(p, i, j, true);
        const double rp = (double)p.rho0 + (double)q.drho.x;
        const double dx = ux - (double)q.jx.x / rp, dr = ur - (double)q.jr.x / rp;
        v[4] += dx * dx + dr * dr;
        v[5] = fmax(v[5], sqrt(dx * dx + dr * dr));
    }
}

template <class S, class C>
__global__ void __launch_bounds__(DIAG_THREADS) diag_kernel(const __grid_constant__ StepParams<C> p, int have_prev,
                                                            double *partials)
{
    double v[DIAG_SLOTS] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    const int64_t N = (int64_t)p.nx * p.nr;
    for (int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; n < N; n += (int64_t)gridDim.x * blockDim.x)
        diag_node<S, C>(p, have_prev, (int)(n % p.nx), (int)(n / p.nx), v);
    diag_block_reduce(v);
    if (threadIdx.x == 0)
        for (int k = 0; k < DIAG_SLOTS; ++k)
            partials[(int64_t)blockIdx.x * DIAG_SLOTS + k] = v[k];
}

// one block folds nblocks partials into out[0 .. DIAG_SLOTS-1]
static __global__ void __launch_bounds__(DIAG_THREADS) diag_final_kernel(const double *partials, int nblocks, double *out)
{
    double v[DIAG_SLOTS] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x)
        diag_combine(v, partials + (int64_t)b * DIAG_SLOTS);
    diag_block_reduce(v);
    if (threadIdx.x == 0)
        for (int k = 0; k < DIAG_SLOTS; ++k)
            out[k] = v[k];
}

// ---- state conversion: absolute FP64 [q][j][i] <-> stored deviations -----------------
template <class S>
using compute_t = typename std::conditional<std::is_same<S, double>::value, double, float>::type;

template <class S>
__global__ void state_in_kernel(S *buf, const double *f, const double *g, int nx, int nr, int pitch, int64_t plane,
                                double rho0, double T0)
{
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t N = (int64_t)nx * nr;
    if (n >= 13 * N)
        return;
    const int q = (int)(n / N);
    const int64_t c = n % N;
    const int i = (int)(c % nx), j = (int)(c / nx);
    double v;
    if (q < 9)
        v = f[(int64_t)q * N + c] - w9<double>(q) * rho0;
    else
        v = g[(int64_t)(q - 9) * N + c] - 0.25 * T0;
    buf[(int64_t)q * plane + (int64_t)(j + 1) * pitch + (i + PAD_COLS)] = store_as<S, compute_t<S>>(compute_t<S>(v));
}

template <class S>
__global__ void state_out_kernel(const S *buf, double *f, double *g, int nx, int nr, int pitch, int64_t plane,
                                 double rho0, double T0)
{
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t N = (int64_t)nx * nr;
    if (n >= 13 * N)
        return;
    const int q = (int)(n / N);
    const int64_t c = n % N;
    const int i = (int)(c % nx), j = (int)(c / nx);
    const double v =
        (double)load_as<S, compute_t<S>>(buf + (int64_t)q * plane + (int64_t)(j + 1) * pitch + (i + PAD_COLS));
    if (q < 9)
        f[(int64_t)q * N + c] = v + w9<double>(q) * rho0;
    else
        g[(int64_t)(q - 9) * N + c] = v + 0.25 * T0;
}

// ---- moment-split storage: state conversion, one node per thread ----------------------
// A minimal parameter block for lin_part: T0 and 1 / (2 rho0), formed exactly as the host
// forms them for the step kernels.
__device__ __forceinline__ StepParams<float> lin_params(double rho0, double T0)
{
    StepParams<float> p;
    p.T0 = float(T0);
    p.hir0 = float(0.5 / rho0);
    return p;
}

template <class S>
__global__ void split_state_in_kernel(S *buf, const double *f, const double *g, int nx, int nr, int pitch,
                                      int64_t plane, double rho0, double T0)
{
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t N = (int64_t)nx * nr;
    if (n >= N)
        return;
    const int i = (int)(n % nx), j = (int)(n / nx);
    const StepParams<float> lp = lin_params(rho0, T0);
    double dev[13], jx = 0.0, jr = 0.0, dT = 0.0;
    for (int k = 0; k < 9; ++k) {
        dev[k] = f[(int64_t)k * N + n] - w9<double>(k) * rho0;
        jx += ex9(k) * dev[k];
        jr += ey9(k) * dev[k];
    }
    for (int k = 0; k < 4; ++k) {
        dev[9 + k] = g[(int64_t)k * N + n] - 0.25 * T0;
        dT += dev[9 + k];
    }
    const float mx = float(jx), mr = float(jr), mT = float(dT);
    const int64_t o = (int64_t)(j + 1) * pitch + (i + PAD_COLS);
    const MomRef M{split_m(buf, plane), plane};
    M.j(o) = make_float2(mx, mr);
    M.T(o) = mT;
    for (int q = 0; q < 13; ++q)
        buf[(int64_t)q * plane + o] = store_as<S, float>(float(dev[q]) - lin_part<float>(lp, q, mx, mr, mT));
}

template <class S>
__global__ void split_state_out_kernel(const S *buf, double *f, double *g, int nx, int nr, int pitch, int64_t plane,
                                       double rho0, double T0)
{
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t N = (int64_t)nx * nr;
    if (n >= N)
        return;
    const int i = (int)(n % nx), j = (int)(n / nx);
    const StepParams<float> lp = lin_params(rho0, T0);
    const int64_t o = (int64_t)(j + 1) * pitch + (i + PAD_COLS);
    const float *M = split_m(buf, plane);
    const float2 jj = reinterpret_cast<const float2 *>(M)[o];
    const float mx = jj.x, mr = jj.y, mT = M[2 * plane + o];
    for (int q = 0; q < 13; ++q) {
        const double v = double(lin_part<float>(lp, q, mx, mr, mT) + load_as<S, float>(buf + (int64_t)q * plane + o));
        if (q < 9)
            f[(int64_t)q * N + n] = v + w9<double>(q) * rho0;
        else
            g[(int64_t)(q - 9) * N + n] = v + 0.25 * T0;
    }
}

}  // namespace lbm
