// Device side of liblbm: the fused pull-stream + collide step of the
// axisymmetric thermal lattice Boltzmann LES model (Djebali et al.,
// arXiv:1002.3028, Eqs. 1-5 and Section 2.3), plus the small kernels that
// fill boundary ghosts, read fields and convert states.
//
// Storage.  13 planes (9 f, 4 g); each plane holds nr + 2 rows of `pitch`
// values: row -1 (ghost), rows 0..nr-1, row nr (ghost); in every row the
// lattice column i sits at element i + PAD_COLS, so columns -1 and nx are
// ghosts and every warp's 32-column segment starts on an aligned boundary.
// Every value is the deviation from the rest state, f_k - w_k rho0 and
// g_k - T0/4.  The arithmetic type C is double for FP64 storage and float
// for FP32/FP16/BF16; all collision arithmetic runs on deviations, so the
// rounding of a stored value is relative to its (small) departure from rest.
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
// Work split of the step kernel.  One warp owns a strip of 32 consecutive
// columns and marches up a band of rows.  The populations each row pulls are
// staged in the warp's shared-memory ring by asynchronous copies issued two
// rows ahead; from a landed row the warp forms the Eq. 2 moments and
// collides the row below, whose radial neighbours' moments (same time level)
// it already holds.  The axial neighbours' rho u_r comes from the adjacent
// lanes by warp shuffle and, for the two columns beside the strip, from the
// staged window's halo.
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

// ---- kernel parameters -------------------------------------------------------
template <class C>
struct StepParams {
    const void *src;  // post-collision state of the previous step (with its ghosts)
    void *dst;        // post-collision state written by this step (with its ghosts)
    int64_t plane;    // elements per population plane ((nr + 2) * pitch)
    int nx, nr, pitch;
    int bc_in, bc_out, bc_top, bc_bottom, axisym;
    int band;         // rows per warp tile
    int nstrips;      // ceil(nx / 32)
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
    const C *u_in, *T_in;         // inlet profiles, nr values
    const C *nu_tab, *al_tab;     // property tables, ntab values
};

// ---- storage conversions -----------------------------------------------------
template <class S, class C> __device__ __forceinline__ C load_as(const S *p);
template <> __device__ __forceinline__ double load_as<double, double>(const double *p) { return __ldg(p); }
template <> __device__ __forceinline__ float load_as<float, float>(const float *p) { return __ldg(p); }
template <> __device__ __forceinline__ float load_as<__half, float>(const __half *p) { return __half2float(__ldg(p)); }
template <> __device__ __forceinline__ float load_as<__nv_bfloat16, float>(const __nv_bfloat16 *p) { return __bfloat162float(__ldg(p)); }

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
// Node (i, j) on the lattice edge, with post-collision deviations fo/go,
// writes every ghost cell whose value the boundary rules take from it.
// t is the time index of the step that will pull these ghosts (inlet noise).
// Writers of distinct ghost cells are distinct nodes, except where two
// rules give the same bounce-back value to the same cell.
template <class S, class C>
__device__ __noinline__ void write_ghosts(const StepParams<C> &p, S *dst, int i, int j, const C *fo, const C *go,
                                          int64_t t)
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
    auto W = [&](int q, int ci, int cj, C v) { dst[cell(p, q, ci, cj)] = store_as<S, C>(v); };
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

// ---- pull and moments -------------------------------------------------------------
template <class S, class C>
__device__ __forceinline__ void pull(const StepParams<C> &p, const S *src, int i, int j, C (&f)[9], C (&g)[4])
{
#pragma unroll
    for (int k = 0; k < 9; ++k)
        f[k] = ld<S, C>(p, src, k, i - ex9(k), j - ey9(k));
#pragma unroll
    for (int k = 0; k < 4; ++k)
        g[k] = ld<S, C>(p, src, 9 + k, i - ex4(k), j - ey4(k));
}

template <class C>
struct Mom {
    C drho, jx, jr, dT;  // rho - rho0, rho u_x, rho u_r, T - T0
};

template <class C>
__device__ __forceinline__ Mom<C> moments(const C (&f)[9], const C (&g)[4])
{
    Mom<C> m;
    m.drho = ((f[0] + f[1]) + (f[2] + f[3])) + ((f[4] + f[5]) + (f[6] + f[7])) + f[8];
    m.jx = (f[1] - f[3]) + (f[5] - f[6]) + (f[8] - f[7]);
    m.jr = (f[2] - f[4]) + (f[5] - f[8]) + (f[6] - f[7]);
    m.dT = (g[0] + g[1]) + (g[2] + g[3]);
    return m;
}

// moments of the ghost row below row 0 / above row nr - 1 (central differences)
template <class C>
__device__ __forceinline__ Mom<C> ghost_bottom(const StepParams<C> &p, Mom<C> m)
{
    if (p.bc_bottom == BOTTOM_AXIS) {
        m.jr = -m.jr;  // rho u_r odd, rho u_x and T even across the axis
    } else {
        m.jx = -m.jx;
        m.jr = -m.jr;
        m.dT = C(2) * p.dT_bottom - m.dT;
    }
    return m;
}

template <class C>
__device__ __forceinline__ Mom<C> ghost_top(const StepParams<C> &p, Mom<C> m)
{
    if (p.bc_top == TOP_WALL) {
        m.jx = -m.jx;
        m.jr = -m.jr;
        m.dT = C(2) * p.dT_top - m.dT;
    }
    return m;
}

// rho u_r of the streamed populations at lattice node (i, j): the six
// populations with a radial component
template <class S, class C>
__device__ __forceinline__ C jr_at(const StepParams<C> &p, const S *src, int i, int j)
{
    return (ld<S, C>(p, src, 2, i, j - 1) - ld<S, C>(p, src, 4, i, j + 1)) +
           (ld<S, C>(p, src, 5, i - 1, j - 1) - ld<S, C>(p, src, 8, i - 1, j + 1)) +
           (ld<S, C>(p, src, 6, i + 1, j - 1) - ld<S, C>(p, src, 7, i + 1, j + 1));
}

// ---- properties (Section 2.3) ------------------------------------------------------
template <class C>
__device__ __forceinline__ void properties(const StepParams<C> &p, C T, C &nu, C &al)
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
    const C n0 = __ldg(p.nu_tab + m), n1 = __ldg(p.nu_tab + m + 1);
    const C a0 = __ldg(p.al_tab + m), a1 = __ldg(p.al_tab + m + 1);
    nu = n0 + fr * (n1 - n0);
    al = a0 + fr * (a1 - a0);
}

// ---- collision of one node (right-hand side of Eq. 1) -------------------------------
// d_* are central differences: d_r(rho u_x), d_r(rho u_r), d_x(rho u_r), d_r T.
// Equilibrium deviations are formed pairwise: with j = rho u,
//   f_eq_k - w_k rho0 = w_k (A + 3 e_k.j + 9/2 (e_k.j)(e_k.u)),  A = drho - 3/2 j.u,
// and opposite directions share the quadratic term.
template <class C>
__device__ __forceinline__ void collide(const StepParams<C> &p, const C (&f)[9], const C (&g)[4], const Mom<C> &m,
                                        C inv_r, C d_rjx, C d_rjr, C d_xjr, C d_rT, C (&fo)[9], C (&go)[4])
{
    constexpr C third = C(1) / C(3);
    constexpr C sixth = C(1) / C(6);
    constexpr C w0 = C(4) / C(9), w1 = C(1) / C(9), w2 = C(1) / C(36);
    const C rho = p.rho0 + m.drho;
    const C inv_rho = C(1) / rho;
    const C ux = m.jx * inv_rho, ur = m.jr * inv_rho;
    const C T = p.T0 + m.dT;
    C nu, al;
    properties<C>(p, T, nu, al);
    const C tau_nu = C(0.5) + C(3) * nu;

    const C A = m.drho - C(1.5) * (m.jx * ux + m.jr * ur);
    const C jp = m.jx + m.jr, up = ux + ur, jm = m.jx - m.jr, um = ux - ur;
    const C qx = A + C(4.5) * m.jx * ux, qr = A + C(4.5) * m.jr * ur;
    const C qp = A + C(4.5) * jp * up, qm = A + C(4.5) * jm * um;
    C fneq[9];
    fneq[0] = f[0] - w0 * A;
    fneq[1] = f[1] - w1 * (qx + C(3) * m.jx);
    fneq[3] = f[3] - w1 * (qx - C(3) * m.jx);
    fneq[2] = f[2] - w1 * (qr + C(3) * m.jr);
    fneq[4] = f[4] - w1 * (qr - C(3) * m.jr);
    fneq[5] = f[5] - w2 * (qp + C(3) * jp);  // e = (1, 1)
    fneq[7] = f[7] - w2 * (qp - C(3) * jp);  // e = (-1, -1)
    fneq[8] = f[8] - w2 * (qm + C(3) * jm);  // e = (1, -1)
    fneq[6] = f[6] - w2 * (qm - C(3) * jm);  // e = (-1, 1)

    // stress Q_ij of Eq. 4 and the Smagorinsky relaxation time
    const C dsum = (fneq[5] + fneq[6]) + (fneq[7] + fneq[8]);
    const C Qxx = (fneq[1] + fneq[3]) + dsum;
    const C Qrr = (fneq[2] + fneq[4]) + dsum;
    const C Qxr = (fneq[5] - fneq[6]) + (fneq[7] - fneq[8]);
    const C Qn = sqrt(C(2) * (Qxx * Qxx + C(2) * Qxr * Qxr + Qrr * Qrr));
    const C tau = C(0.5) * (tau_nu + sqrt(tau_nu * tau_nu + p.cs2_18 * Qn * inv_rho));  // Eq. 4
    const C nu_t = (tau - tau_nu) * third;                                               // Eq. 3
    const C al_tot = al + nu_t * p.inv_prt;                                              // Eq. 5
    const C tau_a = C(0.5) + C(2) * al_tot;
    const C nu_tot = (tau - C(0.5)) * third;

    // axisymmetric sources
    C F1 = C(0), F2x = C(0), F2r = C(0), S = C(0);
    if (p.axisym) {
        const C nr_ = nu_tot * inv_r;
        F1 = -m.jr * inv_r;
        F2x = -m.jx * ur * inv_r + nr_ * (d_rjx + d_xjr);
        F2r = -m.jr * ur * inv_r + nr_ * (d_rjr + d_rjr) - C(2) * nr_ * m.jr * inv_r;
        S = -T * ur * inv_r + al_tot * inv_r * d_rT;
    }

    const C omega = C(1) / tau;
    const C omega_a = C(1) / tau_a;
    const C sx = F2x * sixth, sr = F2r * sixth;
    const C s1 = w1 * F1, s2 = w2 * F1;
    fo[0] = f[0] - omega * fneq[0] + w0 * F1;
    fo[1] = f[1] - omega * fneq[1] + (s1 + sx);
    fo[3] = f[3] - omega * fneq[3] + (s1 - sx);
    fo[2] = f[2] - omega * fneq[2] + (s1 + sr);
    fo[4] = f[4] - omega * fneq[4] + (s1 - sr);
    fo[5] = f[5] - omega * fneq[5] + (s2 + (sx + sr));
    fo[7] = f[7] - omega * fneq[7] + (s2 - (sx + sr));
    fo[8] = f[8] - omega * fneq[8] + (s2 + (sx - sr));
    fo[6] = f[6] - omega * fneq[6] + (s2 - (sx - sr));

    // D2Q4: g_eq_k - T0/4 = dT/4 + (T/2) e_k.u
    const C gd = C(0.25) * m.dT;
    const C hx = C(0.5) * T * ux, hr = C(0.5) * T * ur;
    const C qS = C(0.25) * S;
    go[0] = g[0] - omega_a * (g[0] - (gd + hx)) + qS;
    go[2] = g[2] - omega_a * (g[2] - (gd - hx)) + qS;
    go[1] = g[1] - omega_a * (g[1] - (gd + hr)) + qS;
    go[3] = g[3] - omega_a * (g[3] - (gd - hr)) + qS;
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
// Each warp owns a ring of NSTAGE stages.  A stage holds, for one lattice row
// r and each plane q, the window of source row r - e_qy over source columns
// x0 - H .. x0 + 31 + H (H = one 16-byte chunk of elements), copied with
// asynchronous 16-byte copies spread over the warp's lanes.  Lane l then
// reads population q of node (x0 + l, r) at window index l + H - e_qx.
constexpr int NSTAGE = 4;

template <class S>
struct Win {
    static constexpr int E = 16 / (int)sizeof(S);  // elements per 16-byte chunk
    static constexpr int H = E;                    // halo elements on each side
    static constexpr int W = 32 + 2 * H;           // window length
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

// start the copies of lattice row r into one stage
template <class S, class C>
__device__ __forceinline__ void issue_row(const StepParams<C> &p, const S *src, S *stage, int x0, int r, int lane)
{
    using Wn = Win<S>;
    constexpr int total = 13 * Wn::CH;
#pragma unroll
    for (int m = 0; m < (total + 31) / 32; ++m) {
        const int t = lane + 32 * m;
        if (t < total) {
            const int q = t / Wn::CH;
            const int c = t - q * Wn::CH;
            cp_async16(stage + q * Wn::W + c * Wn::E, src + cell(p, q, x0 - Wn::H + c * Wn::E, r - plane_ey(q)));
        }
    }
}

// population q of lane `col` (0..31, or -1 / 32 for the columns beside the strip)
template <class S, class C>
__device__ __forceinline__ C sget(const S *stage, int q, int ex, int col)
{
    using Wn = Win<S>;
    return load_as_shared<S, C>(stage + q * Wn::W + col + Wn::H - ex);
}

template <class S, class C>
__device__ __forceinline__ void stage_pops(const S *stage, int lane, C (&f)[9], C (&g)[4])
{
#pragma unroll
    for (int k = 0; k < 9; ++k)
        f[k] = sget<S, C>(stage, k, ex9(k), lane);
#pragma unroll
    for (int k = 0; k < 4; ++k)
        g[k] = sget<S, C>(stage, 9 + k, ex4(k), lane);
}

// rho u_r of the streamed populations in window column col of a stage
template <class S, class C>
__device__ __forceinline__ C stage_jr(const S *stage, int col)
{
    return (sget<S, C>(stage, 2, 0, col) - sget<S, C>(stage, 4, 0, col)) +
           (sget<S, C>(stage, 5, 1, col) - sget<S, C>(stage, 8, 1, col)) +
           (sget<S, C>(stage, 6, -1, col) - sget<S, C>(stage, 7, -1, col));
}

// ---- the fused step kernel ------------------------------------------------------------
// collide row j of the tile from its stage and write it (and its ghosts)
template <class S, class C>
__device__ __forceinline__ void collide_row(const StepParams<C> &p, const S *src, S *__restrict__ dst, const S *st,
                                            int x0, int lane, int j, const Mom<C> &mp, const Mom<C> &mc,
                                            const Mom<C> &mn)
{
    const int i = x0 + lane;
    const bool active = i < p.nx;
    // axial neighbours of rho u_r on row j
    C left = __shfl_up_sync(0xffffffffu, mc.jr, 1);
    C right = __shfl_down_sync(0xffffffffu, mc.jr, 1);
    if (lane == 0)
        left = (i == 0) ? jr_beyond_inlet<S, C>(p, src, j) : stage_jr<S, C>(st, -1);
    if (active && (lane == 31 || i == p.nx - 1))
        right = (i == p.nx - 1) ? jr_beyond_outlet<S, C>(p, src, j, mc.jr) : stage_jr<S, C>(st, 32);
    if (!active)
        return;
    C f[9], g[4], fo[9], go[4];
    stage_pops<S, C>(st, lane, f, g);
    const C inv_r = C(1) / (p.r0 + C(j) + C(0.5));
    collide<C>(p, f, g, mc, inv_r, C(0.5) * (mn.jx - mp.jx), C(0.5) * (mn.jr - mp.jr), C(0.5) * (right - left),
               C(0.5) * (mn.dT - mp.dT), fo, go);
    S *o = dst + cell(p, 0, i, j);
#pragma unroll
    for (int k = 0; k < 9; ++k)
        o[(int64_t)k * p.plane] = store_as<S, C>(fo[k]);
#pragma unroll
    for (int k = 0; k < 4; ++k)
        o[(int64_t)(9 + k) * p.plane] = store_as<S, C>(go[k]);
    if (i == 0 || i == p.nx - 1 || j == 0 || j == p.nr - 1) {
        C tf[9], tg[4];
#pragma unroll
        for (int k = 0; k < 9; ++k)
            tf[k] = fo[k];
#pragma unroll
        for (int k = 0; k < 4; ++k)
            tg[k] = go[k];
        write_ghosts<S, C>(p, dst, i, j, tf, tg, p.step + 1);
    }
}

// One warp tile: columns x0..x0+31 of rows j0..j1-1.  Rows j0-1 (if any)
// through min(j1, nr-1) are staged in order, NSTAGE - 2 rows ahead of the
// one whose moments are being formed; row j is collided once the moments of
// row j + 1 exist.
template <class S, class C>
__device__ __forceinline__ void step_tile(const StepParams<C> &p, const S *__restrict__ src, S *__restrict__ dst,
                                          S *wsm, int tile, int lane)
{
    using Wn = Win<S>;
    constexpr int D = NSTAGE - 2;
    const int strip = tile % p.nstrips;
    const int band = tile / p.nstrips;
    const int x0 = strip << 5;
    const int j0 = band * p.band;
    const int j1 = min(j0 + p.band, p.nr);
    const int rfirst = j0 > 0 ? j0 - 1 : j0;
    const int nrows = min(j1, p.nr - 1) - rfirst + 1;

#pragma unroll
    for (int t = 0; t < D; ++t) {
        if (t < nrows)
            issue_row<S, C>(p, src, wsm + t * Wn::STAGE, x0, rfirst + t, lane);
        cp_async_commit();
    }
    Mom<C> mp, mc;
#pragma unroll 1
    for (int idx = 0; idx < nrows; ++idx) {
        __syncwarp();  // every lane is done with the stage refilled next
        if (idx + D < nrows)
            issue_row<S, C>(p, src, wsm + ((idx + D) % NSTAGE) * Wn::STAGE, x0, rfirst + idx + D, lane);
        cp_async_commit();
        cp_async_wait<D>();
        __syncwarp();  // row idx has landed for every lane
        const int r = rfirst + idx;
        const S *st = wsm + (idx % NSTAGE) * Wn::STAGE;
        C f[9], g[4];
        stage_pops<S, C>(st, lane, f, g);
        const Mom<C> mr = moments<C>(f, g);
        if (r < j0) {
            mp = mr;
        } else if (r == j0) {
            if (j0 == 0)
                mp = ghost_bottom<C>(p, mr);
            mc = mr;
        } else {
            collide_row<S, C>(p, src, dst, wsm + ((idx - 1) % NSTAGE) * Wn::STAGE, x0, lane, r - 1, mp, mc, mr);
            mp = mc;
            mc = mr;
        }
    }
    if (j1 == p.nr)
        collide_row<S, C>(p, src, dst, wsm + ((nrows - 1) % NSTAGE) * Wn::STAGE, x0, lane, p.nr - 1, mp, mc,
                          ghost_top<C>(p, mc));
    cp_async_wait<0>();
    __syncwarp();
}

template <class S>
constexpr int step_smem_per_warp()
{
    return NSTAGE * Win<S>::STAGE * (int)sizeof(S);
}

template <class S, class C>
__global__ void __launch_bounds__(256) step_kernel(const __grid_constant__ StepParams<C> p)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int wpc = blockDim.x >> 5;
    const int tile = blockIdx.x * wpc + warp;
    if (tile >= p.ntiles)
        return;  // whole warp
    S *wsm = reinterpret_cast<S *>(smem_raw) + (size_t)warp * NSTAGE * Win<S>::STAGE;
    step_tile<S, C>(p, static_cast<const S *>(p.src), static_cast<S *>(p.dst), wsm, tile, lane);
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
    S *buf = static_cast<S *>(p.dst);
    C tf[9], tg[4];
#pragma unroll
    for (int k = 0; k < 9; ++k)
        tf[k] = load_as<S, C>(buf + cell(p, k, i, j));
#pragma unroll
    for (int k = 0; k < 4; ++k)
        tg[k] = load_as<S, C>(buf + cell(p, 9 + k, i, j));
    write_ghosts<S, C>(p, buf, i, j, tf, tg, p.step);
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
    const S *src = static_cast<const S *>(p.src);
    C f[9], g[4];
    pull<S, C>(p, src, i, j, f, g);
    const Mom<C> m = moments<C>(f, g);
    const C rho = p.rho0 + m.drho;
    out[n] = O(rho);
    out[N + n] = O(m.jx / rho);
    out[2 * N + n] = O(m.jr / rho);
    out[3 * N + n] = O(p.T0 + m.dT);
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

}  // namespace lbm
