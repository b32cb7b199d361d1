/*
 * FP64 CPU oracle of the axisymmetric thermal lattice Boltzmann LES update
 * (Djebali, Calve, Pateyron, El Ganaoui, Sammouda: "Les methodes de
 * resolution de type Lattice Boltzmann sont-elles utilisables pour simuler
 * les jets plasmas ...", arXiv:1002.3028).
 *
 * TEST INFRASTRUCTURE.  Only the tests, the smoke check and the CPU-baseline
 * leg of the benchmark load this library.  It shares no source, header,
 * table or helper with the CUDA path; both are written from the paper.
 *
 * One time step is computed as three plain passes over the whole lattice,
 * in the order the paper's equations use them:
 *   pass 1  pull-streaming (left-hand side of Eq. 1) with the boundary
 *           rules applied to every source outside the lattice;
 *   pass 2  macroscopic moments of the streamed populations (Eq. 2);
 *   pass 3  per node: temperature-dependent nu(T), alpha(T) (Section 2.3),
 *           Smagorinsky relaxation time (Eqs. 3-4), turbulent diffusivity
 *           (Eq. 5), axisymmetric source terms F1, F2i, S (named in Eq. 1),
 *           BGK collision (right-hand side of Eq. 1).
 *
 * Readings of what the paper leaves open (all fixed identically on the CUDA
 * side, written down in the design notes):
 *   - D2Q9 e_k = (0,0),(1,0),(0,1),(-1,0),(0,-1),(1,1),(-1,1),(-1,-1),(1,-1),
 *     weights 4/9, 1/9 x4, 1/36 x4; D2Q4 e_k = (1,0),(0,1),(-1,0),(0,-1),
 *     weight 1/4 (consistent with alpha = (tau_alpha - 1/2)/2 in Section 2.1).
 *   - x is axial (index i), y = r radial (index j); node j sits at
 *     r_j = r0 + j + 1/2 (r0 = 0 puts the axis half a cell below row 0).
 *   - f_eq = w rho (1 + 3 e.u + 9/2 (e.u)^2 - 3/2 u.u), g_eq = T/4 (1 + 2 e.u),
 *     with u the Eq. 2 velocity.
 *   - the source "dt F1" in Eq. 1 carries the lattice weight w_k, the
 *     thermal source "dt S" carries 1/4, "(dt/6) e_ki F2i" is as printed.
 *   - F1  = -rho u_r / r
 *     F2i = -rho u_i u_r / r + (nu_tot / r)(d_r(rho u_i) + d_i(rho u_r))
 *           - 2 nu_tot rho u_r delta_ir / r^2
 *     S   = -T u_r / r + (alpha_tot / r) d_r T
 *     (Zhou's axisymmetric model, the paper's ref. [4]); derivatives are
 *     second-order central differences of the moments of the same time level.
 *   - |Q| = sqrt(2 Q_ij Q_ij), the norm under which Eq. 4 is the positive
 *     root of the quadratic that Eq. 3 leads to.
 *   - nu(T), alpha(T): linear interpolation in uniform tables on
 *     [T_lo, T_hi], T clamped to the range.
 *   - boundaries: axis = specular mirror, walls = half-way bounce-back for f
 *     and anti-bounce-back for g, inlet = equilibrium ghost with the prescribed profile (Eq. 7) plus a
 *     counter-based noise, at the density of the first column; open top and
 *     outflow = zero-gradient copy held at rho0; the radial rule is applied
 *     before the axial one.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_EXPORT __attribute__((visibility("default")))

/* ---- lattice (standard D2Q9 / D2Q4, reading of Section 2.1) ---- */
static const int EX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int EY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const double W9[9] = {4.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0,
                             1.0 / 9.0,  1.0 / 9.0,  1.0 / 36.0,
                             1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
/* population with the opposite velocity, and with the radial component negated */
static const int OPP9[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
static const int MIR9[9] = {0, 1, 4, 3, 2, 8, 7, 6, 5};

static const int GX[4] = {1, 0, -1, 0};
static const int GY[4] = {0, 1, 0, -1};
static const int OPP4[4] = {2, 3, 0, 1};
static const int MIR4[4] = {0, 3, 2, 1};

/* boundary kinds (this file's own numbering) */
enum { ORC_IN_INLET = 0, ORC_IN_PERIODIC = 1 };
enum { ORC_OUT_OUTFLOW = 0, ORC_OUT_WALL = 1, ORC_OUT_PERIODIC = 2 };
enum { ORC_TOP_WALL = 0, ORC_TOP_OPEN = 1 };
enum { ORC_BOTTOM_AXIS = 0, ORC_BOTTOM_WALL = 1 };

typedef struct {
    int nx, nr;
    int bc_in, bc_out, bc_top, bc_bottom;
    int axisym; /* 1: axisymmetric source terms on; 0: plain planar model */
    int nthreads;
    double r0;
    double rho0, T0;
    double Cs, Pr_t;
    double T_top, T_bottom, T_out;
    double noise_amp;
    uint64_t seed;
} orc_params;

typedef struct {
    orc_params p;
    long long step;
    double *f, *g;   /* post-collision state: f[k][j][i], g[k][j][i] */
    double *fs, *gs; /* streamed (pulled) populations of the current step */
    double *m;       /* moments rho, rho u_x, rho u_r, T: m[c][j][i] */
    double *u_in, *T_in;
    double *nu_tab, *al_tab;
    int ntab;
    double T_lo, T_hi;
} orc_sim;

#define IDX(s, k, i, j) (((size_t)(k) * (size_t)(s)->p.nr + (size_t)(j)) * (size_t)(s)->p.nx + (size_t)(i))

/* ---- counter-based inlet noise: SplitMix64 (Steele, Lea, Flood 2014) ---- */
ORC_EXPORT uint64_t orc_splitmix64(uint64_t x)
{
    uint64_t z = x + 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* xi_{j,t} = amp (2U - 1), U = top 53 bits of splitmix64(seed ^ splitmix64(t 2^20 + j)) / 2^53 */
ORC_EXPORT double orc_inlet_noise(uint64_t seed, long long step, int j, double amp)
{
    uint64_t c = ((uint64_t)step << 20) + (uint64_t)j;
    uint64_t h = orc_splitmix64(seed ^ orc_splitmix64(c));
    double U = (double)(h >> 11) * (1.0 / 9007199254740992.0);
    return amp * (2.0 * U - 1.0);
}

/* ---- equilibria (reading of Eq. 1 / Eq. 2) ---- */
ORC_EXPORT void orc_feq(double rho, double ux, double ur, double *out)
{
    double uu = ux * ux + ur * ur;
    for (int k = 0; k < 9; ++k) {
        double eu = EX[k] * ux + EY[k] * ur;
        out[k] = W9[k] * rho * (1.0 + 3.0 * eu + 4.5 * eu * eu - 1.5 * uu);
    }
}

ORC_EXPORT void orc_geq(double T, double ux, double ur, double *out)
{
    for (int k = 0; k < 4; ++k) {
        double eu = GX[k] * ux + GY[k] * ur;
        out[k] = 0.25 * T * (1.0 + 2.0 * eu);
    }
}

/* ---- moments, Eq. 2: out = {rho, rho u_x, rho u_r, T} ---- */
ORC_EXPORT void orc_moments(const double *f, const double *g, double *out)
{
    double rho = 0.0, jx = 0.0, jr = 0.0, T = 0.0;
    for (int k = 0; k < 9; ++k) {
        rho += f[k];
        jx += EX[k] * f[k];
        jr += EY[k] * f[k];
    }
    for (int k = 0; k < 4; ++k)
        T += g[k];
    out[0] = rho;
    out[1] = jx;
    out[2] = jr;
    out[3] = T;
}

/* ---- Smagorinsky total relaxation time, Eqs. 3-4 ---- */
ORC_EXPORT double orc_tau_total(double tau_nu, double Cs, const double *f)
{
    double mom[4], g0[4] = {0, 0, 0, 0}, feq[9];
    orc_moments(f, g0, mom);
    double rho = mom[0];
    orc_feq(rho, mom[1] / rho, mom[2] / rho, feq);
    double Qxx = 0.0, Qxr = 0.0, Qrr = 0.0;
    for (int k = 0; k < 9; ++k) {
        double fneq = f[k] - feq[k];
        Qxx += EX[k] * EX[k] * fneq;
        Qxr += EX[k] * EY[k] * fneq;
        Qrr += EY[k] * EY[k] * fneq;
    }
    double Qn = sqrt(2.0 * (Qxx * Qxx + 2.0 * Qxr * Qxr + Qrr * Qrr));
    return 0.5 * (tau_nu + sqrt(tau_nu * tau_nu + 18.0 * Cs * Cs * Qn / rho));
}

/* ---- property tables, Section 2.3: linear interpolation, T clamped ---- */
ORC_EXPORT double orc_property(const double *tab, int n, double T_lo, double T_hi, double T)
{
    if (n == 1)
        return tab[0];
    double s = (T - T_lo) / (T_hi - T_lo) * (double)(n - 1);
    if (!(s > 0.0))
        s = 0.0;
    if (s > (double)(n - 1))
        s = (double)(n - 1);
    int m = (int)floor(s);
    if (m > n - 2)
        m = n - 2;
    double fr = s - (double)m;
    return tab[m] + fr * (tab[m + 1] - tab[m]);
}

/*
 * Collision of one node (right-hand side of Eq. 1), given its streamed
 * populations, its radius, and the central differences
 *   d[0] = d_r(rho u_x), d[1] = d_r(rho u_r), d[2] = d_x(rho u_r), d[3] = d_r T.
 * props = {nu, alpha}; cfg = {Cs, Pr_t, axisym}.  Writes the post-collision
 * populations and, if diag != NULL, {tau_tot, tau_alpha_tot, F1, F2x, F2r, S}.
 */
ORC_EXPORT void orc_collide_node(const double *fs, const double *gs, double r, const double *d,
                                 double nu, double alpha, double Cs, double Pr_t, int axisym,
                                 double *fpost, double *gpost, double *diag)
{
    double mom[4];
    orc_moments(fs, gs, mom);
    double rho = mom[0], jx = mom[1], jr = mom[2], T = mom[3];
    double ux = jx / rho, ur = jr / rho;

    /* relaxation times from nu(T), alpha(T) (Section 2.1 relations) */
    double tau_nu = 0.5 + 3.0 * nu;

    /* Eq. 4 */
    double tau_tot = orc_tau_total(tau_nu, Cs, fs);
    /* Eq. 3 and Eq. 5 */
    double nu_t = (tau_tot - tau_nu) / 3.0;
    double alpha_tot = alpha + nu_t / Pr_t;
    double tau_al_tot = 0.5 + 2.0 * alpha_tot;
    double nu_tot = (tau_tot - 0.5) / 3.0;

    /* axisymmetric sources */
    double F1 = 0.0, F2x = 0.0, F2r = 0.0, S = 0.0;
    if (axisym) {
        F1 = -jr / r;
        F2x = -jx * ur / r + nu_tot / r * (d[0] + d[2]);
        F2r = -jr * ur / r + nu_tot / r * (d[1] + d[1]) - 2.0 * nu_tot * jr / (r * r);
        S = -T * ur / r + alpha_tot / r * d[3];
    }

    double feq[9], geq[4];
    orc_feq(rho, ux, ur, feq);
    orc_geq(T, ux, ur, geq);
    for (int k = 0; k < 9; ++k)
        fpost[k] = fs[k] - (fs[k] - feq[k]) / tau_tot + W9[k] * F1 + (EX[k] * F2x + EY[k] * F2r) / 6.0;
    for (int k = 0; k < 4; ++k)
        gpost[k] = gs[k] - (gs[k] - geq[k]) / tau_al_tot + 0.25 * S;

    if (diag) {
        diag[0] = tau_tot;
        diag[1] = tau_al_tot;
        diag[2] = F1;
        diag[3] = F2x;
        diag[4] = F2r;
        diag[5] = S;
    }
}

/* ---- creation / configuration ---- */
ORC_EXPORT orc_sim *orc_create(const orc_params *p)
{
    if (!p || p->nx < 1 || p->nr < 1)
        return NULL;
    if ((p->bc_in == ORC_IN_PERIODIC) != (p->bc_out == ORC_OUT_PERIODIC))
        return NULL;
    if (p->bc_bottom == ORC_BOTTOM_AXIS && p->r0 != 0.0)
        return NULL;
    orc_sim *s = (orc_sim *)calloc(1, sizeof(orc_sim));
    if (!s)
        return NULL;
    s->p = *p;
    size_t N = (size_t)p->nx * (size_t)p->nr;
    s->f = (double *)calloc(9 * N, sizeof(double));
    s->g = (double *)calloc(4 * N, sizeof(double));
    s->fs = (double *)calloc(9 * N, sizeof(double));
    s->gs = (double *)calloc(4 * N, sizeof(double));
    s->m = (double *)calloc(4 * N, sizeof(double));
    s->u_in = (double *)calloc((size_t)p->nr, sizeof(double));
    s->T_in = (double *)calloc((size_t)p->nr, sizeof(double));
    s->nu_tab = (double *)calloc(1, sizeof(double));
    s->al_tab = (double *)calloc(1, sizeof(double));
    if (!s->f || !s->g || !s->fs || !s->gs || !s->m || !s->u_in || !s->T_in || !s->nu_tab || !s->al_tab) {
        free(s->f); free(s->g); free(s->fs); free(s->gs); free(s->m);
        free(s->u_in); free(s->T_in); free(s->nu_tab); free(s->al_tab);
        free(s);
        return NULL;
    }
    /* defaults: nu = alpha = 0.1 (tau = 0.8 / 0.7), T range [T0, T0 + 1] */
    s->ntab = 1;
    s->nu_tab[0] = 0.1;
    s->al_tab[0] = 0.1;
    s->T_lo = p->T0;
    s->T_hi = p->T0 + 1.0;
    for (int j = 0; j < p->nr; ++j)
        s->T_in[j] = p->T0;
    /* rest state at rho0, T0 */
    double feq[9], geq[4];
    orc_feq(p->rho0, 0.0, 0.0, feq);
    orc_geq(p->T0, 0.0, 0.0, geq);
    for (int k = 0; k < 9; ++k)
        for (size_t n = 0; n < N; ++n)
            s->f[(size_t)k * N + n] = feq[k];
    for (int k = 0; k < 4; ++k)
        for (size_t n = 0; n < N; ++n)
            s->g[(size_t)k * N + n] = geq[k];
    return s;
}

ORC_EXPORT void orc_destroy(orc_sim *s)
{
    if (!s)
        return;
    free(s->f); free(s->g); free(s->fs); free(s->gs); free(s->m);
    free(s->u_in); free(s->T_in); free(s->nu_tab); free(s->al_tab);
    free(s);
}

ORC_EXPORT void orc_set_inlet(orc_sim *s, const double *u_in, const double *T_in)
{
    memcpy(s->u_in, u_in, (size_t)s->p.nr * sizeof(double));
    memcpy(s->T_in, T_in, (size_t)s->p.nr * sizeof(double));
}

ORC_EXPORT int orc_set_properties(orc_sim *s, const double *nu, const double *alpha, int n, double T_lo,
                                  double T_hi)
{
    if (n < 1 || (n > 1 && !(T_hi > T_lo)))
        return -1;
    double *a = (double *)malloc((size_t)n * sizeof(double));
    double *b = (double *)malloc((size_t)n * sizeof(double));
    if (!a || !b) {
        free(a); free(b);
        return -1;
    }
    memcpy(a, nu, (size_t)n * sizeof(double));
    memcpy(b, alpha, (size_t)n * sizeof(double));
    free(s->nu_tab);
    free(s->al_tab);
    s->nu_tab = a;
    s->al_tab = b;
    s->ntab = n;
    s->T_lo = T_lo;
    s->T_hi = T_hi;
    return 0;
}

ORC_EXPORT void orc_set_state(orc_sim *s, const double *f, const double *g, long long step)
{
    size_t N = (size_t)s->p.nx * (size_t)s->p.nr;
    memcpy(s->f, f, 9 * N * sizeof(double));
    memcpy(s->g, g, 4 * N * sizeof(double));
    s->step = step;
}

ORC_EXPORT void orc_get_state(const orc_sim *s, double *f, double *g)
{
    size_t N = (size_t)s->p.nx * (size_t)s->p.nr;
    memcpy(f, s->f, 9 * N * sizeof(double));
    memcpy(g, s->g, 4 * N * sizeof(double));
}

ORC_EXPORT long long orc_get_step(const orc_sim *s) { return s->step; }

/* ---- pass 1: pull-streaming with the boundary rules ---- */

/* prescribed inlet velocity at row j and step t: profile plus noise where the profile is non-zero */
static double inlet_velocity(const orc_sim *s, int j, long long t)
{
    double u = s->u_in[j];
    if (u != 0.0 && s->p.noise_amp != 0.0)
        u += orc_inlet_noise(s->p.seed, t, j, s->p.noise_amp);
    return u;
}

/* density and velocity of the post-collision populations stored at (i, j) */
static void post_moments(const orc_sim *s, int i, int j, double *rho, double *ux, double *ur)
{
    double d = 0.0, jx = 0.0, jr = 0.0;
    for (int k = 0; k < 9; ++k) {
        double v = s->f[IDX(s, k, i, j)];
        d += v;
        jx += EX[k] * v;
        jr += EY[k] * v;
    }
    *rho = d;
    *ux = jx / d;
    *ur = jr / d;
}

/*
 * f_k at node (i, j) after streaming from the post-collision state.
 * Inlet: equilibrium ghost at the prescribed velocity, density of the
 * first column.  Open top and outflow: zero-gradient copy of the last
 * row / column, with its density shifted back to rho0 along the
 * equilibrium direction (f + (rho0 - rho) f_eq(1, u)).
 */
static double pull_f(const orc_sim *s, int k, int i, int j, long long t)
{
    const orc_params *p = &s->p;
    int is = i - EX[k], js = j - EY[k], kk = k, open = 0;
    /* radial rule first */
    if (js < 0) {
        if (p->bc_bottom == ORC_BOTTOM_AXIS) {
            js = 0;
            kk = MIR9[k];
        } else {
            return s->f[IDX(s, OPP9[k], i, j)];
        }
    } else if (js >= p->nr) {
        if (p->bc_top == ORC_TOP_WALL)
            return s->f[IDX(s, OPP9[k], i, j)];
        js = p->nr - 1;
        open = 1;
    }
    /* then the axial rule, on the (possibly mirrored) source */
    if (is < 0) {
        if (p->bc_in == ORC_IN_INLET) {
            double rb, ub, vb, feq[9];
            post_moments(s, 0, js, &rb, &ub, &vb);
            orc_feq(rb, inlet_velocity(s, js, t), 0.0, feq);
            return feq[kk];
        }
        is = p->nx - 1;
    } else if (is >= p->nx) {
        if (p->bc_out == ORC_OUT_WALL)
            return s->f[IDX(s, OPP9[k], i, j)];
        if (p->bc_out == ORC_OUT_PERIODIC) {
            is = 0;
        } else {
            is = p->nx - 1;
            open = 1;
        }
    }
    double v = s->f[IDX(s, kk, is, js)];
    if (open) {
        double rb, ub, vb, feq[9];
        post_moments(s, is, js, &rb, &ub, &vb);
        orc_feq(1.0, ub, vb, feq);
        v += (p->rho0 - rb) * feq[kk];
    }
    return v;
}

/* g_k at node (i, j) after streaming; walls hold their temperature by anti-bounce-back */
static double pull_g(const orc_sim *s, int k, int i, int j, long long t)
{
    const orc_params *p = &s->p;
    int is = i - GX[k], js = j - GY[k], kk = k;
    if (js < 0) {
        if (p->bc_bottom == ORC_BOTTOM_AXIS) {
            js = 0;
            kk = MIR4[k];
        } else {
            return -s->g[IDX(s, OPP4[k], i, j)] + 0.5 * p->T_bottom;
        }
    } else if (js >= p->nr) {
        if (p->bc_top == ORC_TOP_WALL)
            return -s->g[IDX(s, OPP4[k], i, j)] + 0.5 * p->T_top;
        js = p->nr - 1;
    }
    if (is < 0) {
        if (p->bc_in == ORC_IN_INLET) {
            double geq[4];
            orc_geq(s->T_in[js], inlet_velocity(s, js, t), 0.0, geq);
            return geq[kk];
        }
        is = p->nx - 1;
    } else if (is >= p->nx) {
        if (p->bc_out == ORC_OUT_WALL)
            return -s->g[IDX(s, OPP4[k], i, j)] + 0.5 * p->T_out;
        is = (p->bc_out == ORC_OUT_PERIODIC) ? 0 : p->nx - 1;
    }
    return s->g[IDX(s, kk, is, js)];
}

static void stream_and_moments(orc_sim *s)
{
    const int nx = s->p.nx, nr = s->p.nr;
    const long long t = s->step;
#pragma omp parallel for schedule(static) num_threads(s->p.nthreads > 0 ? s->p.nthreads : 1)
    for (int j = 0; j < nr; ++j) {
        for (int i = 0; i < nx; ++i) {
            double fl[9], gl[4], mom[4];
            for (int k = 0; k < 9; ++k) {
                fl[k] = pull_f(s, k, i, j, t);
                s->fs[IDX(s, k, i, j)] = fl[k];
            }
            for (int k = 0; k < 4; ++k) {
                gl[k] = pull_g(s, k, i, j, t);
                s->gs[IDX(s, k, i, j)] = gl[k];
            }
            /* pass 2: moments, Eq. 2 */
            orc_moments(fl, gl, mom);
            for (int c = 0; c < 4; ++c)
                s->m[IDX(s, c, i, j)] = mom[c];
        }
    }
}

/*
 * Moment c (0 rho, 1 rho u_x, 2 rho u_r, 3 T) at a face neighbour that may
 * lie one cell outside the lattice: the ghost values that make the central
 * differences consistent with each boundary rule.
 */
static double moment_at(const orc_sim *s, int c, int i, int j, long long t)
{
    const orc_params *p = &s->p;
    if (j < 0) {
        double v = s->m[IDX(s, c, i, 0)];
        if (p->bc_bottom == ORC_BOTTOM_AXIS)
            return (c == 2) ? -v : v;                 /* rho u_r odd, others even */
        if (c == 1 || c == 2) return -v;              /* no slip */
        if (c == 3) return 2.0 * p->T_bottom - v;     /* wall temperature */
        return v;
    }
    if (j >= p->nr) {
        double v = s->m[IDX(s, c, i, p->nr - 1)];
        if (p->bc_top == ORC_TOP_OPEN)
            return v;
        if (c == 1 || c == 2) return -v;
        if (c == 3) return 2.0 * p->T_top - v;
        return v;
    }
    if (i < 0) {
        if (p->bc_in == ORC_IN_PERIODIC)
            return s->m[IDX(s, c, p->nx - 1, j)];
        if (c == 0) return p->rho0;
        if (c == 1) return p->rho0 * inlet_velocity(s, j, t);
        if (c == 2) return 0.0;
        return s->T_in[j];
    }
    if (i >= p->nx) {
        if (p->bc_out == ORC_OUT_PERIODIC)
            return s->m[IDX(s, c, 0, j)];
        double v = s->m[IDX(s, c, p->nx - 1, j)];
        if (p->bc_out == ORC_OUT_OUTFLOW)
            return v;
        if (c == 1 || c == 2) return -v;
        if (c == 3) return 2.0 * p->T_out - v;
        return v;
    }
    return s->m[IDX(s, c, i, j)];
}

/* ---- pass 3: properties, LES relaxation, sources, collision ---- */
static void collide_all(orc_sim *s)
{
    const int nx = s->p.nx, nr = s->p.nr;
    const long long t = s->step;
#pragma omp parallel for schedule(static) num_threads(s->p.nthreads > 0 ? s->p.nthreads : 1)
    for (int j = 0; j < nr; ++j) {
        double r = s->p.r0 + (double)j + 0.5;
        for (int i = 0; i < nx; ++i) {
            double fl[9], gl[4], fo[9], go[4], d[4];
            for (int k = 0; k < 9; ++k)
                fl[k] = s->fs[IDX(s, k, i, j)];
            for (int k = 0; k < 4; ++k)
                gl[k] = s->gs[IDX(s, k, i, j)];
            d[0] = 0.5 * (moment_at(s, 1, i, j + 1, t) - moment_at(s, 1, i, j - 1, t));
            d[1] = 0.5 * (moment_at(s, 2, i, j + 1, t) - moment_at(s, 2, i, j - 1, t));
            d[2] = 0.5 * (moment_at(s, 2, i + 1, j, t) - moment_at(s, 2, i - 1, j, t));
            d[3] = 0.5 * (moment_at(s, 3, i, j + 1, t) - moment_at(s, 3, i, j - 1, t));
            double T = s->m[IDX(s, 3, i, j)];
            double nu = orc_property(s->nu_tab, s->ntab, s->T_lo, s->T_hi, T);
            double alpha = orc_property(s->al_tab, s->ntab, s->T_lo, s->T_hi, T);
            orc_collide_node(fl, gl, r, d, nu, alpha, s->p.Cs, s->p.Pr_t, s->p.axisym, fo, go, NULL);
            for (int k = 0; k < 9; ++k)
                s->f[IDX(s, k, i, j)] = fo[k];
            for (int k = 0; k < 4; ++k)
                s->g[IDX(s, k, i, j)] = go[k];
        }
    }
}

ORC_EXPORT void orc_step(orc_sim *s, int nsteps)
{
    for (int n = 0; n < nsteps; ++n) {
        stream_and_moments(s);
        collide_all(s);
        s->step += 1;
    }
}

/*
 * Macroscopic fields at the current time: the Eq. 2 moments of the
 * populations streamed from the stored state.  out = [rho, u_x, u_r, T],
 * each nr x nx row-major.
 */
ORC_EXPORT void orc_get_fields(orc_sim *s, double *out)
{
    stream_and_moments(s);
    size_t N = (size_t)s->p.nx * (size_t)s->p.nr;
    for (size_t n = 0; n < N; ++n) {
        double rho = s->m[n];
        out[n] = rho;
        out[N + n] = s->m[N + n] / rho;
        out[2 * N + n] = s->m[2 * N + n] / rho;
        out[3 * N + n] = s->m[3 * N + n];
    }
}

/* streamed populations of the current time (pass 1 only), for boundary checks */
ORC_EXPORT void orc_get_streamed(orc_sim *s, double *f, double *g)
{
    stream_and_moments(s);
    size_t N = (size_t)s->p.nx * (size_t)s->p.nr;
    memcpy(f, s->fs, 9 * N * sizeof(double));
    memcpy(g, s->gs, 4 * N * sizeof(double));
}
