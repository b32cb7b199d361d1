/*
 * lbm.h -- C ABI of the GB300 axisymmetric thermal lattice Boltzmann LES
 * library (liblbm).
 *
 * The library advances one lattice of the double-population model of
 * Djebali et al. (arXiv:1002.3028): D2Q9 populations f_k for density and
 * momentum and D2Q4 populations g_k for temperature, Eq. 1, with
 *   - the macroscopic moments of Eq. 2,
 *   - the Smagorinsky closed-form relaxation time of Eqs. 3-4 and the
 *     turbulent diffusivity of Eq. 5,
 *   - viscosity and diffusivity read from temperature-indexed tables
 *     (Section 2.3),
 *   - the axisymmetric source terms F1, F2i, S named under Eq. 1 (Zhou's
 *     axisymmetric model, the paper's ref. [4]),
 *   - the inlet profiles of Eq. 7 (Section 2.4) and axis, wall, open and
 *     outflow boundaries.
 * Every step is one pass of a fused pull-stream + collide kernel on the GPU;
 * the steps of one call run in one persistent launch.
 *
 * Conventions (all lattice units, dx = dt = 1):
 *   x is axial (index i, 0 <= i < nx); r is radial (index j, 0 <= j < nr);
 *   node j sits at radius r0 + j + 1/2.
 *   D2Q9 e_k: (0,0) (1,0) (0,1) (-1,0) (0,-1) (1,1) (-1,1) (-1,-1) (1,-1).
 *   D2Q4 e_k: (1,0) (0,1) (-1,0) (0,-1).
 *   Population arrays exchanged through this header are FP64, laid out
 *   [k][j][i] (k slowest, i fastest, no padding): 9 f planes, 4 g planes.
 *   Field arrays are [c][j][i] with c = rho, u_x, u_r, T.
 *
 * Threading and streams: a handle may be used from one host thread at a
 * time.  Every call that takes a stream enqueues its GPU work on that stream
 * (NULL = the legacy default stream) and returns without synchronising,
 * unless stated otherwise.  Host arrays passed in are copied before the call
 * returns; device arrays passed in must stay valid until the enqueued work
 * has completed.
 *
 * Errors: every int-returning call returns LBM_OK (0) or a negative
 * lbm_status; lbm_last_error() gives a message for the calling thread.
 * Outputs are left untouched on error.
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define LBM_API __attribute__((visibility("default")))
#else
#define LBM_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_lattice lbm_lattice; /* opaque handle */
typedef void *lbm_stream;               /* a cudaStream_t; NULL = default stream */

typedef enum {
    LBM_OK = 0,
    LBM_ERR_INVALID_ARG = -1, /* bad handle, size, boundary kind or table */
    LBM_ERR_OOM = -2,         /* device allocation failed or caller memory too small */
    LBM_ERR_CUDA = -3,        /* a CUDA runtime call or a kernel launch failed */
    LBM_ERR_DIVERGED = -4     /* non-finite or non-positive density / temperature found */
} lbm_status;

/* storage type of the populations on the device (the arithmetic is FP64
 * for LBM_F64 and FP32 for the others).
 *   LBM_F64, LBM_F32, LBM_F16, LBM_BF16  every population stored as its
 *       deviation from the rest state, f_k - w_k rho0 and g_k - T0/4
 *       (the reduced-precision format of the populations of Eq. 1 as
 *       deviations from the rest weights).
 *   LBM_F16S, LBM_BF16S  moment-split storage: per node the moments
 *       j = rho u and T - T0 in FP32, and each population as a 2-byte
 *       deviation from the part of its equilibrium linear in those moments,
 *       f_k - w_k rho0 - 3 w_k e_k.j and g_k - T/4 - T e_k.j / (2 rho0).  The
 *       2-byte rounding then scales with the non-equilibrium and quadratic
 *       parts, not with the velocity or the temperature excess: 76 bytes per
 *       lattice update instead of 52.  Two-buffer pattern only.  A checkpoint
 *       (lbm_save) holds the 13 population planes, then the (j_x, j_r)
 *       pairs of every node (FP32, interleaved), then T - T0 (FP32). */
typedef enum { LBM_F64 = 0, LBM_F32 = 1, LBM_F16 = 2, LBM_BF16 = 3, LBM_F16S = 4, LBM_BF16S = 5 } lbm_storage;

typedef enum { LBM_IN_INLET = 0, LBM_IN_PERIODIC = 1 } lbm_bc_in;
typedef enum { LBM_OUT_OUTFLOW = 0, LBM_OUT_WALL = 1, LBM_OUT_PERIODIC = 2 } lbm_bc_out;
typedef enum { LBM_TOP_WALL = 0, LBM_TOP_OPEN = 1 } lbm_bc_top;
typedef enum { LBM_BOTTOM_AXIS = 0, LBM_BOTTOM_WALL = 1 } lbm_bc_bottom;

/* Memory layout of the populations (lbm_desc.pattern).
 *   LBM_PATTERN_AB  two buffers: each step pulls from one and writes the
 *                   other (the default).
 *   LBM_PATTERN_AA  one buffer updated in place (the "AA" pattern of
 *                   Bailey et al., ICPP 2009), plus the moments at the warp
 *                   tiles' edges that neighbouring tiles exchange within a
 *                   step (the same-time neighbour moments of Eq. 1's
 *                   sources): 13 populations and about 1.5 moment values
 *                   per node instead of 26 populations (FP32: about 58
 *                   instead of 104 bytes per node; FP16/BF16 about 32
 *                   instead of 52; FP64 about 116 instead of 208).  Results
 *                   are bit for bit those of LBM_PATTERN_AB, except that
 *                   no previous state is kept (lbm_diagnostics reports no
 *                   residual).  Bands are at least 4 rows.  Batches hold
 *                   lattices of one pattern. */
typedef enum { LBM_PATTERN_AB = 0, LBM_PATTERN_AA = 1 } lbm_pattern;

/*
 * Lattice description (Section 2.4: a half-plane of nx x nr nodes whose
 * inlet edge carries the profiles of Eq. 7).
 *
 * Boundary rules, applied to every pulled source outside the lattice, the
 * radial rule before the axial one:
 *   bottom AXIS   specular mirror (requires r0 == 0);
 *   bottom/top WALL, outlet WALL
 *                 half-way bounce-back for f; anti-bounce-back for g holding
 *                 T_bottom / T_top / T_out;
 *   top OPEN, outlet OUTFLOW
 *                 zero-gradient copy of the last row / column, its density
 *                 shifted back to rho0 along the unit-density equilibrium;
 *   inlet INLET   equilibrium at the density of the first column, velocity
 *                 (u_in[j] + noise, 0), temperature T_in[j];
 *   PERIODIC      wrap (must be set on both axial ends).
 * noise: xi = noise_amp (2U - 1) on rows with u_in[j] != 0, U the top 53
 * bits of splitmix64(seed ^ splitmix64(step * 2^20 + j)) / 2^53.
 * axisym = 0 switches the axisymmetric sources off (the planar model).
 */
typedef struct {
    int32_t nx, nr;      /* 1 <= nx, nr < 2^20; 13 (nr + 2)(nx + 128) < 2^31 */
    int32_t storage;     /* lbm_storage */
    int32_t bc_in;       /* lbm_bc_in */
    int32_t bc_out;      /* lbm_bc_out */
    int32_t bc_top;      /* lbm_bc_top */
    int32_t bc_bottom;   /* lbm_bc_bottom */
    int32_t axisym;      /* 1: axisymmetric sources F1, F2i, S on */
    double r0;           /* radius of the bottom edge */
    double rho0, T0;     /* reference density and temperature (rest state) */
    double Cs;           /* Smagorinsky constant (Eq. 3); 0 = no model */
    double Pr_t;         /* turbulent Prandtl number (Eq. 5), > 0 */
    double T_top, T_bottom, T_out; /* wall temperatures */
    double noise_amp;    /* amplitude of the inlet velocity noise */
    uint64_t seed;       /* seed of the inlet noise */
    int32_t pattern;     /* lbm_pattern (0 = LBM_PATTERN_AB) */
} lbm_desc;

/* Message of the last failed call on this host thread ("" if none). */
LBM_API const char *lbm_last_error(void);

/* Bytes of device memory a lattice needs (two population buffers, or one
 * and the moment planes for LBM_PATTERN_AA, plus tables; 256-byte
 * aligned).  Returns LBM_ERR_INVALID_ARG for a bad desc. */
LBM_API int lbm_required_bytes(const lbm_desc *d, size_t *bytes);

/*
 * Create a lattice at rest (rho0, T0, u = 0), step counter 0, inlet
 * u_in = 0 and T_in = T0, properties nu = alpha = 0.1 on [T0, T0 + 1].
 *   dev_mem:  caller-owned device memory of at least lbm_required_bytes()
 *             bytes, 256-byte aligned, or NULL to let the library
 *             cudaMalloc (and later free) its own.  Caller memory must
 *             outlive the handle.
 *   out:      receives the handle; untouched on error.
 * The set-up (zeroing, tables, ghost cells; a stream-ordered allocation of
 * the library's own memory) is queued on the legacy default stream and the
 * host does not wait for it: every later call orders its stream after the
 * set-up's completion event.  Caller memory must be free of other work
 * queued on non-blocking streams when the call is made.
 * Errors: INVALID_ARG, OOM, CUDA.
 */
LBM_API int lbm_create(const lbm_desc *d, void *dev_mem, size_t bytes, lbm_lattice **out);

/* Release the handle.  The library's own memory is freed in stream order
 * after the last work queued through the handle, without waiting on the
 * host; caller memory may be reused once that work has run.  NULL is a
 * no-op. */
LBM_API void lbm_destroy(lbm_lattice *h);

/*
 * Inlet profiles of Eq. 7: host arrays of nr values, u_in = axial inlet
 * velocity and T_in = inlet temperature at each row (copied).
 */
LBM_API int lbm_set_inlet(lbm_lattice *h, const double *u_in, const double *T_in, int32_t nr,
                  lbm_stream stream);

/*
 * Temperature-dependent properties of Section 2.3: n >= 1 host values each
 * of the lattice viscosity nu and diffusivity alpha on a uniform grid over
 * [T_lo, T_hi] (n == 1: constants), linearly interpolated, T clamped to the
 * range.  tau_nu = 1/2 + 3 nu, tau_alpha = 1/2 + 2 alpha (Section 2.1).
 * Requires n <= 4096, T_hi > T_lo when n > 1, nu > 0 and alpha > 0.
 */
LBM_API int lbm_set_properties(lbm_lattice *h, const double *nu, const double *alpha, int32_t n,
                       double T_lo, double T_hi, lbm_stream stream);

/*
 * Advance nsteps >= 0 time steps (Eq. 1).  All the steps run in one
 * persistent launch of the fused kernel (more than one only when nsteps x
 * warp tiles exceeds 2^30): a warp tile of step t + 1 starts once the tiles
 * around it have finished step t.  The result is bit for bit that of nsteps
 * one-step calls.  Asynchronous; returns LBM_ERR_CUDA if a launch fails.  A
 * wait that runs out (it cannot in a correct launch; it is bounded all the
 * same) raises LBM_STATUS_TIMEOUT (see lbm_check) and ends the launch early.
 */
LBM_API int lbm_step(lbm_lattice *h, int32_t nsteps, lbm_stream stream);

/* Number of steps taken so far (the time index of the inlet noise). */
LBM_API int64_t lbm_get_step(const lbm_lattice *h);

/*
 * Global FP64 diagnostics of the current state (moments of Eq. 2 of the
 * streamed populations at every node): mass = Σ rho and heat = Σ T over the
 * nodes, mass_axi = Σ r rho and heat_axi = Σ r T (the axisymmetric
 * volume weight, 2 pi r dx dr up to the constant), max_speed = max |u|, the
 * steady-state residual between the current and the previous step
 * (residual_max = max |u(t) - u(t-1)| / max |u(t)|, residual_l2 =
 * sqrt(Σ |u(t) - u(t-1)|^2 / Σ |u(t)|^2); NaN unless the last change of the
 * state was a step, and always NaN for LBM_PATTERN_AA), and nonfinite = the number of nodes whose density is
 * not finite and positive or whose velocity or temperature is not finite.
 * Uses the lattice's own scratch area; synchronises the stream and writes
 * *out.  Returns LBM_ERR_DIVERGED (with *out filled) when nonfinite > 0.
 */
typedef struct {
    double mass, mass_axi, heat, heat_axi;
    double max_speed, residual_max, residual_l2;
    int64_t nonfinite;
} lbm_diag;
LBM_API int lbm_diagnostics(lbm_lattice *h, lbm_diag *out, lbm_stream stream);

/*
 * lbm_diagnostics_noalloc: the same diagnostics as lbm_diagnostics (same
 * quantities, equal up to FP64 summation order), for callers that cannot
 * allocate device memory: programs whose device memory is entirely handed
 * out by another allocator or budget, or that must keep a fixed device
 * footprint once set up.  It allocates nothing and does not use the
 * lattice's scratch area: its partial sums go to one fixed array compiled
 * into this library (1.2 MB, which every GPU that loads the library holds
 * until the process exits).  The paper has no counterpart; it is a service
 * of this library.
 *   - Lattices of at most 16384 rows (nr); larger ones are refused with
 *     LBM_ERR_INVALID_ARG (use lbm_diagnostics for them).
 *   - The lattice's device must be current.  A call looks up the array's
 *     device address (no allocation) unless its stream is capturing a
 *     graph, when it takes the address of the device's last lookup: make
 *     the first call on a device before any stream capture (a first call
 *     inside a capture is refused with LBM_ERR_INVALID_ARG).
 *   - Every call on a device shares the array and overwrites the slots it
 *     uses (nothing needs to start at zero); calls whose work overlaps on
 *     the GPU, from any thread or stream, race on it.
 *   - Synchronises the stream; returns LBM_ERR_DIVERGED as lbm_diagnostics.
 */
LBM_API int lbm_diagnostics_noalloc(lbm_lattice *h, lbm_diag *out, lbm_stream stream);

/* Error flags raised on the device since the last call, then cleared:
 * LBM_STATUS_TIMEOUT (1) = a bounded wait inside a kernel ran out (the
 * steps since the last check are invalid).  0 = no error.  Synchronises the
 * device. */
#define LBM_STATUS_TIMEOUT 1
LBM_API int lbm_check(lbm_lattice *h, int32_t *flags);

/*
 * Self-test of the bounded waits of the persistent step launch (either
 * pattern's; no counterpart in the paper).  Runs one launch on the default stream in
 * which every work item waits for neighbours of a step that never runs,
 * with a wait limit of a few tens of microseconds: each wait gives up,
 * raises LBM_STATUS_TIMEOUT and its warp stops; nothing is computed or
 * written, and the lattice's state and step count are unchanged.  Writes
 * the status read back (LBM_STATUS_TIMEOUT when the waits behaved) to
 * *flags and clears it.  For LBM_PATTERN_AA lattices of two or more work
 * items a second launch also tests the wait in the middle of an item: one
 * item forms and publishes its edge moments (scratch that the next step
 * recomputes) and waits for neighbours that never run; *flags is
 * LBM_STATUS_TIMEOUT only if both launches raised it.  Synchronises the
 * device.  Not for batch members.
 */
LBM_API int lbm_selftest_wait_timeout(lbm_lattice *h, int32_t *flags);

/*
 * Macroscopic fields at the current time: the Eq. 2 moments rho, u_x, u_r,
 * T of the populations streamed from the stored state.  dev_out is caller
 * device memory of 4 * nr * nx values of type out_type (LBM_F64 or LBM_F32),
 * layout [c][j][i].
 */
LBM_API int lbm_get_fields(lbm_lattice *h, void *dev_out, int32_t out_type, lbm_stream stream);

/*
 * Copy the stored post-collision populations out of / into the lattice as
 * absolute FP64 values: dev_f holds 9 * nr * nx values, dev_g 4 * nr * nx,
 * both caller device memory, layout [k][j][i].  set_state also sets the
 * step counter.  Values are rounded to the storage type on the way in.
 */
LBM_API int lbm_get_state(lbm_lattice *h, double *dev_f, double *dev_g, lbm_stream stream);
LBM_API int lbm_set_state(lbm_lattice *h, const double *dev_f, const double *dev_g, int64_t step,
                  lbm_stream stream);

/*
 * Checkpoint and resume, bit for bit.  The paper has no counterpart (its
 * runs are single uninterrupted integrations of Eq. 1); a checkpoint is the
 * stored state exactly as the step kernel keeps it, so a resumed lattice
 * continues exactly as an uninterrupted one would.
 *
 * lbm_checkpoint_bytes: size of a checkpoint, 13 * nr * nx values of the
 *   storage type (8, 4 or 2 bytes).
 * lbm_save: copy the stored post-collision populations, as deviations
 *   from rest (f_k - w_k rho0 and g_k - T0 / 4, in the storage type; the
 *   same values and layout for both patterns), into dev_out,
 *   caller device memory of lbm_checkpoint_bytes bytes, layout
 *   [q][j][i] with q = f0..f8, g0..g3.  The step counter is read with
 *   lbm_get_step.  Asynchronous on the stream.
 * lbm_restore: the reverse, into a lattice of the same size and storage
 *   (either pattern), and set its step counter to step (>= 0); the
 *   boundary ghosts are recomputed.  The next lbm_diagnostics residual has
 *   no previous state.  Returns LBM_ERR_INVALID_ARG for a NULL buffer or a
 *   negative step.
 */
LBM_API int lbm_checkpoint_bytes(const lbm_lattice *h, size_t *bytes);
LBM_API int lbm_save(lbm_lattice *h, void *dev_out, lbm_stream stream);
LBM_API int lbm_restore(lbm_lattice *h, const void *dev_in, int64_t step, lbm_stream stream);

/*
 * Launch shape of the step kernel: CTAs of warps_per_cta warps (1..8), one
 * warp per tile of a strip of columns (lbm_set_strip_width) x band_rows rows.
 * band_rows >= 1 fixes the band height; 0 lets the library choose it from
 * the number of warps the GPU holds at once (the default).
 * warps_per_cta == 0 keeps the current value (default 1).  Results do not
 * depend on the launch shape.
 */
LBM_API int lbm_set_launch(lbm_lattice *h, int32_t band_rows, int32_t warps_per_cta);

/* The launch shape lbm_step uses: band height, warps per CTA and CTAs per
 * launch (any pointer may be NULL). */
LBM_API int lbm_get_launch(const lbm_lattice *h, int32_t *band_rows, int32_t *warps_per_cta, int32_t *ctas);

/* Work-item size of lbm_step's persistent launch: a warp takes `group`
 * adjacent warp tiles of one band at a time and synchronises with its
 * neighbours once per item (1..64; 0 = automatic; LBM_PATTERN_AA lattices
 * widen items where the GPU holds too few warps for one band of items).
 * Results do not depend on it.  lbm_get_item_group returns the value in use (-1 for a bad handle). */
LBM_API int lbm_set_item_group(lbm_lattice *h, int32_t group);
LBM_API int32_t lbm_get_item_group(const lbm_lattice *h);

/*
 * Tile width of the two-buffer step kernel: each warp owns a strip of
 * `columns` lattice columns, one node per lane for 32, two per lane (with
 * paired FP32x2 arithmetic) for 64.  0 restores the default (64; 32 for
 * LBM_F64, which has no paired form).  A launch-shape parameter like the
 * band height: results are bit for bit the same at either width.  The AA
 * pattern keeps its default; a batch member uses its batch's width
 * (lbm_batch_set_strip_width; a batch of LBM_F16S or LBM_BF16S lattices
 * defaults to 32 columns, measured 13% faster on a ragged ensemble).  lbm_get_strip_width returns the width in use
 * (-1 for a bad handle).  The autotuner searches it with the band height and
 * the warps per CTA.  Returns LBM_ERR_INVALID_ARG for another width.
 */
LBM_API int lbm_set_strip_width(lbm_lattice *h, int32_t columns);
LBM_API int32_t lbm_get_strip_width(const lbm_lattice *h);

/*
 * Batches: independent lattices of any sizes (one storage type) stepped
 * together, all members' warp tiles in one persistent launch of many steps
 * (every member advances exactly as it would alone under Eq. 1).
 *   lbm_batch_create   empty batch for lattices of the given lbm_storage.
 *   lbm_batch_add / lbm_batch_remove
 *                      change the membership (takes effect at the next
 *                      lbm_batch_step; a lattice belongs to one batch at a
 *                      time; lbm_step on a member is an error; lbm_destroy
 *                      removes it; all members share one lbm_pattern).
 *                      Members keep their own state, inlet, tables and
 *                      step counter; lbm_get_fields and friends work on
 *                      members as usual.
 *   lbm_batch_step     nsteps steps of every member on the stream; with
 *                      use_graph != 0, whole chunks of 64 steps are replayed
 *                      from a captured CUDA graph of one launch (re-captured
 *                      when the membership or a member's parameters
 *                      change), the rest runs as one launch.
 *   lbm_batch_set_launch / lbm_batch_get_launch
 *                      launch shape shared by all members (as lbm_set_launch;
 *                      tiles = warp tiles per step).
 * The library allocates the batch's small device tables itself.  A batch
 * and its members may be used from one host thread at a time.
 */
typedef struct lbm_batch lbm_batch;
LBM_API int lbm_batch_create(int32_t storage, lbm_batch **out);
LBM_API void lbm_batch_destroy(lbm_batch *b);
LBM_API int lbm_batch_add(lbm_batch *b, lbm_lattice *h);
LBM_API int lbm_batch_remove(lbm_batch *b, lbm_lattice *h);
LBM_API int32_t lbm_batch_size(const lbm_batch *b);
LBM_API int lbm_batch_step(lbm_batch *b, int32_t nsteps, int32_t use_graph, lbm_stream stream);
LBM_API int lbm_batch_set_launch(lbm_batch *b, int32_t band_rows, int32_t warps_per_cta);
LBM_API int lbm_batch_get_launch(const lbm_batch *b, int32_t *band_rows, int32_t *warps_per_cta, int32_t *tiles);
LBM_API int lbm_batch_set_strip_width(lbm_batch *b, int32_t columns);
LBM_API int32_t lbm_batch_get_strip_width(const lbm_batch *b);

#ifdef __cplusplus
}
#endif

#endif /* LBM_H */
