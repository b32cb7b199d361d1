// C ABI of liblbm (declared in include/lbm.h): lattice handles, device
// memory layout (two population buffers, or one in the AA pattern), table
// uploads, the persistent multi-step launches of one lattice and of
// batches, state I/O, checkpoints and diagnostics.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "lbm.h"
#include "lbm_internal.h"

namespace {

thread_local char g_err[512] = "";

int fail(int code, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return code;
}

int cuda_fail(cudaError_t e, const char *what)
{
    return fail(LBM_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

// ---- host-to-device uploads without synchronisation ---------------------------
// Inlet profiles, property tables and batch tables are copied through pinned
// staging blocks (a ring per device), so cudaMemcpyAsync never has to stage
// pageable memory itself, which may synchronise the stream and so drain the
// work queued on it.  A block is reused once the copy that last read it has
// completed (its event).  An upload larger than a block takes the pageable
// path and synchronises its stream.
constexpr size_t kStageBytes = (size_t)1 << 20;
constexpr int kStageBlocks = 16;
constexpr int kMaxDevices = 64;

struct StageBlock {
    char *host = nullptr;
    cudaEvent_t done = nullptr;
};

std::mutex g_stage_mutex;
StageBlock g_stage[kMaxDevices][kStageBlocks];
int g_stage_next[kMaxDevices] = {};

struct Part {
    void *dst;
    const void *src;
    size_t n;
};

size_t round16(size_t n) { return (n + 15) / 16 * 16; }

// copies every part (host source, device destination) in the order of stream s
cudaError_t upload(const Part *parts, int nparts, cudaStream_t s)
{
    size_t total = 0;
    for (int k = 0; k < nparts; ++k)
        total += round16(parts[k].n);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return e;
    if (total > kStageBytes || dev < 0 || dev >= kMaxDevices) {
        for (int k = 0; k < nparts && e == cudaSuccess; ++k)
            if (parts[k].n > 0)
                e = cudaMemcpyAsync(parts[k].dst, parts[k].src, parts[k].n, cudaMemcpyHostToDevice, s);
        return e == cudaSuccess ? cudaStreamSynchronize(s) : e;
    }
    std::lock_guard<std::mutex> lock(g_stage_mutex);
    StageBlock &b = g_stage[dev][g_stage_next[dev]];
    g_stage_next[dev] = (g_stage_next[dev] + 1) % kStageBlocks;
    if (!b.host) {
        e = cudaHostAlloc(reinterpret_cast<void **>(&b.host), kStageBytes, cudaHostAllocPortable);
        if (e != cudaSuccess) {
            b.host = nullptr;
            return e;
        }
        e = cudaEventCreateWithFlags(&b.done, cudaEventDisableTiming);
        if (e != cudaSuccess) {
            cudaFreeHost(b.host);
            b.host = nullptr;
            b.done = nullptr;
            return e;
        }
    } else {
        e = cudaEventSynchronize(b.done);  // the copies that last read this block have run
        if (e != cudaSuccess)
            return e;
    }
    size_t off = 0;
    for (int k = 0; k < nparts && e == cudaSuccess; ++k) {
        if (parts[k].n == 0)
            continue;
        std::memcpy(b.host + off, parts[k].src, parts[k].n);
        e = cudaMemcpyAsync(parts[k].dst, b.host + off, parts[k].n, cudaMemcpyHostToDevice, s);
        off += round16(parts[k].n);
    }
    if (e == cudaSuccess)
        e = cudaEventRecord(b.done, s);
    return e;
}

constexpr int kMaxTable = 4096;
constexpr size_t kAlign = 256;

size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

// moment-split storage: FP32 moment planes beside the 2-byte population planes
bool is_split(int storage) { return storage == LBM_F16S || storage == LBM_BF16S; }


// lattice columns per warp strip of the step kernel: 32 nodes per lane-slot,
// two per lane in FP32 arithmetic
int strip_cols(int storage) { return storage == LBM_F64 ? 32 : 64; }

// nodes per lane of the two-buffer step kernels by default (strip width / 32)
int default_nv(int storage) { return storage == LBM_F64 ? 1 : 2; }

// ... and of a batch: moment-split batches default to 32-column strips (the ragged 256-jet
// ensemble in FP16 moment-split storage at band 64: 588 against 678 us per step at 64
// columns, whose 162-register tiles leave 12 warps per SM; the rest-deviation FP16 batch is
// faster at 64, 377 against 392 us)
int batch_default_nv(int storage) { return is_split(storage) ? 1 : default_nv(storage); }

size_t storage_bytes(int storage)
{
    switch (storage) {
    case LBM_F64: return 8;
    case LBM_F32: return 4;
    case LBM_F16: return 2;
    case LBM_F16S: return 2;
    case LBM_BF16S: return 2;
    case LBM_BF16: return 2;
    default: return 0;
    }
}

// Elements per padded row: PAD_COLS leading elements (the last of them is
// ghost column -1), then columns 0..nx (nx is the other ghost column)
// rounded up to a multiple of 64, then 32 more so a warp's staged window
// (its 32 or 64 columns and a 16-byte halo on each side) never leaves the
// row; every row and every warp strip starts on a 64-byte boundary.  For
// 4- and 8-byte values, then one 128-byte block more if the row would
// otherwise hold an even number of them: an odd number spreads the rows a
// warp tile stages over the memory channels (the 4096 x 1024 FP32 jet ran
// 78.9 instead of 79.4 us per step with rows of 133 blocks against 132; 134
// and 136 blocks ran 79.4 and 80.1).  The 2-byte kernels are bound by
// instruction issue, not by memory, and keep the shorter rows.
int row_pitch(int nx, int storage)
{
    const int es = (int)storage_bytes(storage);
    int row = lbm::PAD_COLS + (nx + 1 + 63) / 64 * 64 + 32;
    if (es >= 4 && (row * es / 128) % 2 == 0)
        row += 128 / es;
    return row;
}

struct Layout {
    int pitch;      // elements from one row of a population plane to the next (row stride)
    int64_t plane;  // elements from one population plane to the next (plane stride)
    size_t buf_bytes;                    // one population buffer (13 planes)
    size_t off_buf[2];                   // the same buffer twice for the AA pattern
    size_t off_edge;                     // AA pattern: edge moments of the warp tiles (lbm_aa.cuh)
    size_t off_uin_d, off_tin_d, off_uin_f, off_tin_f;
    size_t off_nu_d, off_al_d, off_nu_f, off_al_f;
    size_t off_status;
    size_t off_sync;  // multi-step launch: work counter, then one counter per warp tile
    size_t off_diag;  // diagnostics scratch: block partials, then the folded result
    size_t total;
};

int check_desc(const lbm_desc *d)
{
    if (!d)
        return fail(LBM_ERR_INVALID_ARG, "desc is NULL");
    if (d->nx < 1 || d->nr < 1)
        return fail(LBM_ERR_INVALID_ARG, "nx and nr must be >= 1 (got %d, %d)", d->nx, d->nr);
    if ((int64_t)d->nx * d->nr > INT32_MAX)
        return fail(LBM_ERR_INVALID_ARG, "nx * nr exceeds 2^31 - 1");
    if (d->nr >= (1 << 20))
        return fail(LBM_ERR_INVALID_ARG, "nr must be below 2^20 (inlet noise counter)");
    if (storage_bytes(d->storage) == 0)
        return fail(LBM_ERR_INVALID_ARG, "unknown storage type %d", d->storage);
    // the step kernel addresses a population buffer with 32-bit element offsets
    if (13 * (int64_t)row_pitch(d->nx, d->storage) * (d->nr + 2) >= INT32_MAX)
        return fail(LBM_ERR_INVALID_ARG, "lattice %d x %d exceeds 13 * (nr + 2) * pitch < 2^31 elements", d->nx, d->nr);
    if (d->pattern != LBM_PATTERN_AB && d->pattern != LBM_PATTERN_AA)
        return fail(LBM_ERR_INVALID_ARG, "unknown pattern %d", d->pattern);
    if (d->pattern == LBM_PATTERN_AA && is_split(d->storage))
        return fail(LBM_ERR_INVALID_ARG, "moment-split storage (LBM_F16S, LBM_BF16S) has the two-buffer pattern only");
    if (d->bc_in < 0 || d->bc_in > 1 || d->bc_out < 0 || d->bc_out > 2 || d->bc_top < 0 || d->bc_top > 1 ||
        d->bc_bottom < 0 || d->bc_bottom > 1)
        return fail(LBM_ERR_INVALID_ARG, "unknown boundary kind");
    if ((d->bc_in == LBM_IN_PERIODIC) != (d->bc_out == LBM_OUT_PERIODIC))
        return fail(LBM_ERR_INVALID_ARG, "periodic must be set on both axial ends");
    if (d->bc_bottom == LBM_BOTTOM_AXIS && d->r0 != 0.0)
        return fail(LBM_ERR_INVALID_ARG, "the axis requires r0 == 0");
    if (d->axisym && !(d->r0 >= 0.0))
        return fail(LBM_ERR_INVALID_ARG, "r0 must be >= 0 with the axisymmetric sources");
    if (!(d->rho0 > 0.0) || !std::isfinite(d->T0) || !(d->Pr_t > 0.0) || !(d->Cs >= 0.0))
        return fail(LBM_ERR_INVALID_ARG, "need rho0 > 0, finite T0, Pr_t > 0, Cs >= 0");
    return LBM_OK;
}

Layout make_layout(const lbm_desc *d)
{
    Layout L;
    L.pitch = row_pitch(d->nx, d->storage);
    L.plane = (int64_t)L.pitch * (d->nr + 2);  // ghost rows -1 and nr
    L.buf_bytes = is_split(d->storage)
                      ? align_up((size_t)lbm::split_moff(L.plane) + (size_t)lbm::SPLIT_MOMENTS * (size_t)L.plane * 4)
                      : align_up((size_t)13 * (size_t)L.plane * storage_bytes(d->storage));
    const bool aa = d->pattern == LBM_PATTERN_AA;
    size_t o = 0;
    L.off_buf[0] = o;
    o += L.buf_bytes;
    L.off_buf[1] = aa ? L.off_buf[0] : o;
    o += aa ? 0 : L.buf_bytes;
    L.off_edge = o;
    const int max_strips = (d->nx + strip_cols(d->storage) - 1) / strip_cols(d->storage);
    o += aa ? align_up((size_t)lbm::aa_edge_elems(d->nr, L.pitch, max_strips) * (d->storage == LBM_F64 ? 8 : 4)) : 0;
    const size_t nrd = align_up((size_t)d->nr * 8), nrf = align_up((size_t)d->nr * 4);
    L.off_uin_d = o; o += nrd;
    L.off_tin_d = o; o += nrd;
    L.off_uin_f = o; o += nrf;
    L.off_tin_f = o; o += nrf;
    const size_t td = align_up((size_t)kMaxTable * 8), tf = align_up((size_t)kMaxTable * 4);
    L.off_nu_d = o; o += td;
    L.off_al_d = o; o += td;
    L.off_nu_f = o; o += tf;
    L.off_al_f = o; o += tf;
    L.off_status = o; o += kAlign;
    // warp tiles are at least 32 columns by one row; the AA pattern counts both passes
    L.off_sync = o; o += align_up((size_t)4 * (1 + (aa ? 2 : 1) * (size_t)((d->nx + 31) / 32) * (size_t)d->nr));
    L.off_diag = o; o += align_up((size_t)(lbm::DIAG_MAX_BLOCKS + 1) * lbm::DIAG_SLOTS * sizeof(double));
    L.total = o;
    // Two-buffer lattices of the rest-deviation types interleave their 13
    // planes by row: a lattice row holds its 13 plane rows one after the
    // other, so the rows a warp tile stages lie together in memory (the
    // 4096 x 1024 FP32 jet: 80.0 -> 78.7 us per step; the arithmetic is
    // unchanged, and so are the results).  Every kernel addresses a cell as
    // q * plane + (j + 1) * pitch + i, so only the strides change (the AA
    // edge area keeps rows of one padded row, StepParams::epitch).  The
    // moment-split types keep whole planes (their moment area follows the
    // last plane).
    if (!is_split(d->storage)) {
        L.plane = L.pitch;
        L.pitch *= 13;
    }
    return L;
}

}  // namespace

struct lbm_batch;

struct lbm_lattice {
    lbm_desc d;
    lbm_batch *batch;  // the batch this lattice belongs to, if any
    Layout L;
    char *mem;
    bool own;
    int cur;  // buffer holding the current state
    int64_t step;
    int ntab;
    double T_lo, T_hi;
    bool prev_valid;       // the other buffer holds the state one step earlier
    int band, warps;       // launch shape; band 0 = chosen from the occupancy
    int band_eff, ctas;    // band and CTA count of a one-step lbm_step launch
    int ctas_max;          // CTAs resident on the device at once (persistent grid)
    int group;             // warp tiles per work item of lbm_step (0 = automatic)
    int device, sms;
    int nv;                // nodes per lane of the two-buffer kernels: warp strips of 32 nv columns
    bool aa;               // AA pattern: one buffer (cur stays 0) and the tiles' edge moments
    int phase;             // AA pattern: representation of the stored state (lbm_aa.cuh)
    cudaEvent_t ready;     // recorded after the set-up work lbm_create enqueued
    cudaEvent_t last;      // recorded after the last work enqueued on the lattice
    // counters of the two-buffer persistent launch, carried from launch to launch
    // (lbm::RunCtl): valid for sync_items work items; 0 = reset before the next launch
    int64_t sync_items;
    unsigned sync_cbase, sync_fbase;
    bool sync_captured;    // a launch was captured into a graph: reset before every launch

    void *buf(int b) const { return mem + L.off_buf[b]; }
    template <class T> T *at(size_t off) const { return reinterpret_cast<T *>(mem + off); }
};

struct lbm_batch {
    int storage;
    std::vector<lbm_lattice *> members;
    bool dirty;      // membership or a member's parameters changed since the tables were built
    int version;     // bumped on every rebuild (graph cache key)
    void *d_params;  // StepParams<C>[members]
    size_t cap_params;
    lbm::TileRef *d_tiles;
    size_t cap_tiles;
    unsigned *d_sync;  // multi-step launch: work counter, then one or (AA) two counters per table entry
    int ntiles;
    bool aa;           // members use the AA pattern (all members share one pattern)
    bool far;          // a periodic member has a one-column last strip (lbm::far_wrap)
    int aa_ctas_min;   // AA: CTAs that cover the widest member's edge-wait distance
    int band, warps, band_eff;
    int nv;        // nodes per lane: warp strips of 32 nv columns
    int sms;
    int ctas_max;  // CTAs resident on the device at once (persistent grid)
    cudaStream_t capture;  // private stream used to capture step graphs
    cudaGraphExec_t graph;
    int graph_version, graph_steps;
    cudaEvent_t last;  // recorded after the last batch launch
    bool launched;     // `last` has been recorded
};

namespace {

template <class C>
lbm::StepParams<C> make_params(const lbm_lattice *h, const C *u_in, const C *T_in, const C *nu, const C *al)
{
    const lbm_desc &d = h->d;
    lbm::StepParams<C> p;
    std::memset(&p, 0, sizeof(p));
    p.src = h->buf(h->cur);
    p.dst = h->buf(1 - h->cur);
    p.plane = h->L.plane;
    p.nx = d.nx;
    p.nr = d.nr;
    p.pitch = h->L.pitch;
    p.epitch = row_pitch(d.nx, d.storage);
    p.bc_in = d.bc_in;
    p.bc_out = d.bc_out;
    p.bc_top = d.bc_top;
    p.bc_bottom = d.bc_bottom;
    p.axisym = d.axisym ? 1 : 0;
    p.band = h->band_eff;
    p.nstrips = (d.nx + 32 * h->nv - 1) / (32 * h->nv);
    const int nbands = (d.nr + h->band_eff - 1) / h->band_eff;
    p.ntiles = p.nstrips * nbands;
    p.ntab = h->ntab;
    p.step = h->step;
    p.seed = d.seed;
    p.noise_amp = d.noise_amp;
    p.r0 = C(d.r0);
    p.rho0 = C(d.rho0);
    p.T0 = C(d.T0);
    p.cs2_18 = C(18.0 * d.Cs * d.Cs);
    p.inv_prt = C(1.0 / d.Pr_t);
    p.dT_top = C(d.T_top - d.T0);
    p.dT_bottom = C(d.T_bottom - d.T0);
    p.dT_out = C(d.T_out - d.T0);
    p.T_lo = C(h->T_lo);
    p.tab_scale = h->ntab > 1 ? C((double)(h->ntab - 1) / (h->T_hi - h->T_lo)) : C(0);
    p.hir0 = C(0.5 / d.rho0);
    p.u_in = u_in;
    p.T_in = T_in;
    p.nu_tab = nu;
    p.al_tab = al;
    p.status = h->at<int>(h->L.off_status);
    p.aa = h->aa ? 1 : 0;
    p.phase = h->aa ? h->phase : 0;
    p.edge = h->aa ? h->at<C>(h->L.off_edge) : nullptr;
    return p;
}

lbm::StepParams<double> params_d(const lbm_lattice *h)
{
    return make_params<double>(h, h->at<double>(h->L.off_uin_d), h->at<double>(h->L.off_tin_d),
                               h->at<double>(h->L.off_nu_d), h->at<double>(h->L.off_al_d));
}

lbm::StepParams<float> params_f(const lbm_lattice *h)
{
    return make_params<float>(h, h->at<float>(h->L.off_uin_f), h->at<float>(h->L.off_tin_f),
                              h->at<float>(h->L.off_nu_f), h->at<float>(h->L.off_al_f));
}

// warp tiles per work item of lbm_step: the set value, else 1
int item_group(const lbm_lattice *h) { return h->group > 0 ? h->group : 1; }

// Launch shape of the step kernel: a persistent grid of one-warp CTAs (by
// default) working through strip x band tiles.  A tile of step t + 1 waits
// for the tiles around it of step t, which precede it by one step's worth
// of tiles in the work order; the automatic band height keeps that distance
// at about 5.4 rounds of the resident warps (3.4 for 2-byte storage), which
// leaves the waits rare, with bands of 1..8 rows (each band stages two halo
// rows).  On the 4096 x 1024 jet this picks band 5 for FP32 and band 8 for
// FP16 storage.  FP32 at band 6 (4.5 rounds) ran either at 79 or at 87 us
// per step, one or the other for a whole launch, with three to four times
// as many blocked waits and 3% more DRAM reads in the slow launches; at
// band 5 every launch ran at 80 us (band 4: 83).  Lattices
// with fewer tiles than that are bound by the latency of one tile per step
// and get the shortest bands (1024 x 256: band 1, 2.3x faster than band 4).
// The grid holds at most one step's worth of tiles: warps beyond that could
// only wait.
int plan_launch(lbm_lattice *h)
{
    int per_sm = 0;
    cudaError_t e;
    switch (h->d.storage) {
    case LBM_F64: e = h->aa ? lbm::occupancy_aa_run_f64(h->warps, &per_sm) : lbm::occupancy_run_f64(h->warps, h->nv, &per_sm); break;
    case LBM_F32: e = h->aa ? lbm::occupancy_aa_run_f32(h->warps, &per_sm) : lbm::occupancy_run_f32(h->warps, h->nv, &per_sm); break;
    case LBM_F16: e = h->aa ? lbm::occupancy_aa_run_f16(h->warps, &per_sm) : lbm::occupancy_run_f16(h->warps, h->nv, &per_sm); break;
    case LBM_F16S: e = lbm::occupancy_run_f16s(h->warps, h->nv, &per_sm); break;
    case LBM_BF16S: e = lbm::occupancy_run_bf16s(h->warps, h->nv, &per_sm); break;
    default: e = h->aa ? lbm::occupancy_aa_run_bf16(h->warps, &per_sm) : lbm::occupancy_run_bf16(h->warps, h->nv, &per_sm); break;
    }
    if (e != cudaSuccess)
        return cuda_fail(e, "occupancy query");
    if (per_sm < 1)
        return fail(LBM_ERR_INVALID_ARG, "a CTA of %d warps does not fit on an SM", h->warps);
    const int resident_warps = per_sm * std::max(1, h->sms) * h->warps;
    const int nstrips = (h->d.nx + 32 * h->nv - 1) / (32 * h->nv);
    if (h->band > 0) {
        h->band_eff = h->band;
    } else {
        // tenths of a round between dependent items (AA: 3.4 for every storage type).  On
        // the 4096 x 1024 jet, of bands 4..16: FP32 band 5 (5.4 rounds; band 6 runs a launch
        // at either 79 or 87 us per step); 2-byte storage 4.0 rounds: rest-deviation FP16
        // band 7 (65.1 us per step against 66.5 at band 6 and 69.0 at band 8), moment-split
        // band 9 of its 12 warps per SM (89.8 us every launch; band 10 ran 88.8 with some
        // launches at 90-95, band 8 91.3 and band 11 108)
        const bool split = is_split(h->d.storage) && !h->aa;
        const int64_t rounds10 = h->aa ? 34 : (storage_bytes(h->d.storage) == 2 ? 40 : 54);
        const int64_t want_tiles = std::max<int64_t>(1, rounds10 * resident_warps / 10);
        const int64_t band = ((int64_t)h->d.nr * nstrips + want_tiles - 1) / want_tiles;
        h->band_eff = (int)std::min<int64_t>(split ? 10 : 8, std::max<int64_t>(1, band));
    }
    if (h->aa)  // the edge area holds the edge rows of bands of at least AA_BAND_MIN rows
        h->band_eff = std::max(h->band_eff, std::min(lbm::AA_BAND_MIN, h->d.nr));
    const int64_t ntiles = (int64_t)nstrips * ((h->d.nr + h->band_eff - 1) / h->band_eff);
    h->ctas_max = per_sm * std::max(1, h->sms);
    h->ctas = (int)std::min<int64_t>(h->ctas_max, (ntiles + h->warps - 1) / h->warps);
    return LBM_OK;
}

// Schedule of an AA-pattern launch (lbm_aa.cuh): an item waits in the
// middle of its work for the edges of items up to D = one band of items
// plus one further on, so at least D + 2 warps must be resident; items are
// widened (more strips per item) until they are.
struct AAPlan {
    int group;
    int64_t items, per_launch;
    int ctas;
};

AAPlan aa_plan(const lbm_lattice *h)
{
    const lbm_desc &d = h->d;
    const int nstrips = (d.nx + 32 * h->nv - 1) / (32 * h->nv);
    const int64_t nbands = (d.nr + h->band_eff - 1) / h->band_eff;
    const int64_t resident = (int64_t)h->ctas_max * h->warps;
    AAPlan a;
    for (a.group = std::max(1, item_group(h));; ++a.group) {
        const int64_t cols = lbm::item_cols(nstrips, a.group);
        a.items = cols * nbands;
        const int64_t D = std::min<int64_t>(a.items - 1, cols + 1);
        if (resident >= D + 2 || a.group >= nstrips)
            break;
    }
    const int64_t cols = lbm::item_cols(nstrips, a.group);
    const int64_t D = std::min<int64_t>(a.items - 1, cols + 1);
    a.ctas = (int)std::min<int64_t>(h->ctas_max, (std::max<int64_t>(a.items, D + 2) + h->warps - 1) / h->warps);
    // the work counter stays below 2^31
    a.per_launch = std::max<int64_t>(1, ((int64_t)1 << 31) / std::max<int64_t>(1, 2 * a.items));
    return a;
}

cudaError_t aa_launch(lbm_lattice *h, const lbm::RunCtl &ctl, int ctas, cudaStream_t s)
{
    switch (h->d.storage) {
    case LBM_F64: return lbm::launch_aa_run_f64(params_d(h), ctl, h->warps, ctas, s);
    case LBM_F32: return lbm::launch_aa_run_f32(params_f(h), ctl, h->warps, ctas, s);
    case LBM_F16: return lbm::launch_aa_run_f16(params_f(h), ctl, h->warps, ctas, s);
    default: return lbm::launch_aa_run_bf16(params_f(h), ctl, h->warps, ctas, s);
    }
}

// recompute the boundary ghosts of the current state (after it or the inlet changed)
int fill_ghosts(lbm_lattice *h, cudaStream_t s)
{
    cudaError_t e;
    if (h->aa) {
        switch (h->d.storage) {
        case LBM_F64: e = lbm::launch_aa_fill_f64(params_d(h), s); break;
        case LBM_F32: e = lbm::launch_aa_fill_f32(params_f(h), s); break;
        case LBM_F16: e = lbm::launch_aa_fill_f16(params_f(h), s); break;
        default: e = lbm::launch_aa_fill_bf16(params_f(h), s); break;
        }
        return e == cudaSuccess ? LBM_OK : cuda_fail(e, "ghost fill kernel launch");
    }
    switch (h->d.storage) {
    case LBM_F64: {
        auto p = params_d(h);
        p.dst = h->buf(h->cur);
        e = lbm::launch_fill_f64(p, s);
        break;
    }
    case LBM_F32: {
        auto p = params_f(h);
        p.dst = h->buf(h->cur);
        e = lbm::launch_fill_f32(p, s);
        break;
    }
    case LBM_F16: {
        auto p = params_f(h);
        p.dst = h->buf(h->cur);
        e = lbm::launch_fill_f16(p, s);
        break;
    }
    case LBM_F16S: {
        auto p = params_f(h);
        p.dst = h->buf(h->cur);
        e = lbm::launch_fill_f16s(p, s);
        break;
    }
    case LBM_BF16S: {
        auto p = params_f(h);
        p.dst = h->buf(h->cur);
        e = lbm::launch_fill_bf16s(p, s);
        break;
    }
    default: {
        auto p = params_f(h);
        p.dst = h->buf(h->cur);
        e = lbm::launch_fill_bf16(p, s);
        break;
    }
    }
    return e == cudaSuccess ? LBM_OK : cuda_fail(e, "ghost fill kernel launch");
}

int upload_pair(lbm_lattice *h, size_t off_d, size_t off_f, const double *src, int n, cudaStream_t s,
                const char *what)
{
    std::vector<float> tmp((size_t)n);
    for (int k = 0; k < n; ++k)
        tmp[(size_t)k] = (float)src[k];
    const Part parts[2] = {{h->mem + off_d, src, (size_t)n * 8}, {h->mem + off_f, tmp.data(), (size_t)n * 4}};
    cudaError_t e = upload(parts, 2, s);
    if (e != cudaSuccess)
        return cuda_fail(e, what);
    return LBM_OK;
}

bool valid(const lbm_lattice *h) { return h != nullptr && h->mem != nullptr; }

// Work that a call enqueues on stream s comes after the lattice's set-up
// (enter) and is remembered as the lattice's last use (leave), after which
// lbm_destroy releases memory the library allocated.
int enter(const lbm_lattice *h, cudaStream_t s)
{
    cudaError_t e = cudaStreamWaitEvent(s, h->ready, 0);
    return e == cudaSuccess ? LBM_OK : cuda_fail(e, "ordering the stream after the lattice's set-up");
}

int leave(lbm_lattice *h, cudaStream_t s, int rc)
{
    if (rc == LBM_OK) {
        cudaError_t e = cudaEventRecord(h->last, s);
        if (e != cudaSuccess)
            return cuda_fail(e, "recording the lattice's last use");
    }
    return rc;
}

}  // namespace


// ---- batches ------------------------------------------------------------------------
namespace {

constexpr int kGraphSteps = 64;  // steps of the one launch a captured batch graph holds

size_t params_size(int storage)
{
    return storage == LBM_F64 ? sizeof(lbm::StepParams<double>) : sizeof(lbm::StepParams<float>);
}

int batch_occupancy(lbm_batch *b, int warps, int *per_sm)
{
    cudaError_t e;
    switch (b->storage) {
    case LBM_F64: e = b->aa ? lbm::occupancy_aa_batch_f64(warps, per_sm) : lbm::occupancy_batch_f64(warps, b->nv, per_sm); break;
    case LBM_F32: e = b->aa ? lbm::occupancy_aa_batch_f32(warps, per_sm) : lbm::occupancy_batch_f32(warps, b->nv, per_sm); break;
    case LBM_F16: e = b->aa ? lbm::occupancy_aa_batch_f16(warps, per_sm) : lbm::occupancy_batch_f16(warps, b->nv, per_sm); break;
    case LBM_F16S: e = lbm::occupancy_batch_f16s(warps, b->nv, per_sm); break;
    case LBM_BF16S: e = lbm::occupancy_batch_bf16s(warps, b->nv, per_sm); break;
    default: e = b->aa ? lbm::occupancy_aa_batch_bf16(warps, per_sm) : lbm::occupancy_batch_bf16(warps, b->nv, per_sm); break;
    }
    return e == cudaSuccess ? LBM_OK : cuda_fail(e, "batch occupancy query");
}

void drop_graph(lbm_batch *b)
{
    if (b->graph) {
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
    }
}

// build the parameter and tile tables of the current members
int batch_rebuild(lbm_batch *b, cudaStream_t s)
{
    const int n = (int)b->members.size();
    b->aa = n > 0 && b->members[0]->aa;
    int per_sm = 0;
    int rc = batch_occupancy(b, b->warps, &per_sm);
    if (rc)
        return rc;
    if (per_sm < 1)
        return fail(LBM_ERR_INVALID_ARG, "a CTA of %d warps does not fit on an SM", b->warps);
    const int cols = 32 * b->nv;
    int64_t area = 0;  // strips x rows over all members
    for (lbm_lattice *h : b->members)
        area += (int64_t)((h->d.nx + cols - 1) / cols) * h->d.nr;
    if (b->band > 0) {
        b->band_eff = b->band;
    } else {
        // as for one lattice (plan_launch), up to a cap by storage type: a batch's tiles of
        // one step are spread over many lattices, and longer bands cut the halo cost of small
        // ones.  The ragged 256-jet ensemble, us per step: FP32 438.8 at band 16 (441.6 at
        // 12, 445.9 at 24); rest-deviation FP16 369.3 at 32 (376.9 at 16, 385.5 at 64);
        // moment-split FP16 585.9 at 64 (648.0 at 16, 603.6 at 96, 667.2 at 128)
        const int64_t rounds10 = storage_bytes(b->storage) == 2 ? 34 : 45;
        const int64_t want_tiles = std::max<int64_t>(1, rounds10 * (int64_t)per_sm * std::max(1, b->sms) * b->warps / 10);
        const int64_t band = (area + want_tiles - 1) / want_tiles;
        const int64_t cap = b->aa ? 16 : (is_split(b->storage) ? 64 : (storage_bytes(b->storage) == 2 ? 32 : 16));
        b->band_eff = (int)std::min<int64_t>(cap, std::max<int64_t>(1, band));
    }
    if (b->aa)  // the members' edge areas hold bands of at least AA_BAND_MIN rows
        b->band_eff = std::max(b->band_eff, lbm::AA_BAND_MIN);
    // AA: an item waits on the edges of items up to one band of its lattice's tiles plus one
    // away, so the launch needs that many warps plus two for the widest member
    int max_strips = 1;
    b->far = false;
    for (lbm_lattice *h : b->members) {
        const int ns = (h->d.nx + cols - 1) / cols;
        max_strips = std::max(max_strips, ns);
        b->far = b->far || lbm::far_wrap(h->d.bc_in, h->d.nx, ns, cols);
    }
    b->aa_ctas_min = (max_strips + 3 + b->warps - 1) / b->warps;
    if (b->aa && b->aa_ctas_min > per_sm * std::max(1, b->sms))
        return fail(LBM_ERR_INVALID_ARG, "an AA batch member of %d strips is too wide for the resident warps",
                    max_strips);
    std::vector<lbm::TileRef> tiles;
    std::vector<unsigned char> params(params_size(b->storage) * (size_t)std::max(1, n));
    for (int m = 0; m < n; ++m) {
        lbm_lattice *h = b->members[(size_t)m];
        const int saved = h->band_eff, saved_nv = h->nv;
        h->band_eff = b->band_eff;
        h->nv = b->nv;
        if (b->storage == LBM_F64) {
            const auto p = params_d(h);
            std::memcpy(params.data() + (size_t)m * sizeof(p), &p, sizeof(p));
            for (int t = 0; t < p.ntiles; ++t)
                tiles.push_back({m, t});
        } else {
            const auto p = params_f(h);
            std::memcpy(params.data() + (size_t)m * sizeof(p), &p, sizeof(p));
            for (int t = 0; t < p.ntiles; ++t)
                tiles.push_back({m, t});
        }
        h->band_eff = saved;
        h->nv = saved_nv;
    }
    if (tiles.size() > (size_t)INT32_MAX)
        return fail(LBM_ERR_INVALID_ARG, "too many tiles in the batch");
    cudaError_t e = cudaSuccess;
    if (params.size() > b->cap_params || tiles.size() > b->cap_tiles) {
        // the old tables may still be read by queued steps: they are released in stream order
        if (params.size() > b->cap_params) {
            if (b->d_params)
                cudaFreeAsync(b->d_params, s);
            b->d_params = nullptr;
            e = cudaMallocAsync(&b->d_params, params.size() * 2, s);
            b->cap_params = e == cudaSuccess ? params.size() * 2 : 0;
        }
        if (e == cudaSuccess && tiles.size() > b->cap_tiles) {
            if (b->d_tiles)
                cudaFreeAsync(b->d_tiles, s);
            if (b->d_sync)
                cudaFreeAsync(b->d_sync, s);
            b->d_tiles = nullptr;
            b->d_sync = nullptr;
            const size_t cap = std::max<size_t>(1, tiles.size() * 2);
            e = cudaMallocAsync(&b->d_tiles, cap * sizeof(lbm::TileRef), s);
            if (e == cudaSuccess)
                e = cudaMallocAsync(&b->d_sync, (2 * cap + 1) * sizeof(unsigned), s);
            b->cap_tiles = e == cudaSuccess ? cap : 0;
        }
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(LBM_ERR_OOM, "batch table allocation: %s", cudaGetErrorString(e));
        }
    }
    const Part parts[2] = {{b->d_params, params.data(), params_size(b->storage) * (size_t)n},
                           {b->d_tiles, tiles.data(), tiles.size() * sizeof(lbm::TileRef)}};
    e = upload(parts, 2, s);
    if (e != cudaSuccess)
        return cuda_fail(e, "batch table upload");
    // the new members' set-up comes first
    for (lbm_lattice *h : b->members) {
        int rc2 = enter(h, s);
        if (rc2)
            return rc2;
    }
    b->ntiles = (int)tiles.size();
    b->ctas_max = per_sm * std::max(1, b->sms);
    b->dirty = false;
    b->version += 1;
    return LBM_OK;
}

// nsteps steps of every member in one persistent launch (counters zeroed first)
cudaError_t batch_launch(lbm_batch *b, int nsteps, cudaStream_t s)
{
    const int n = (int)b->members.size();
    cudaError_t e = cudaMemsetAsync(b->d_sync, 0, (2 * b->cap_tiles + 1) * sizeof(unsigned), s);
    if (e != cudaSuccess)
        return e;
    lbm::RunCtl ctl;
    ctl.counter = b->d_sync;
    ctl.flags = b->d_sync + 1;
    ctl.nsteps = nsteps;
    ctl.radius = b->band_eff >= 2 ? 1 : 2;
    ctl.wrap = 0;  // read from each lattice's parameters
    ctl.spin_limit = lbm::RUN_SPIN_LIMIT;
    ctl.group = 1;
    int ctas = (int)std::min<int64_t>(b->ctas_max, ((int64_t)b->ntiles + b->warps - 1) / b->warps);
    if (b->aa) {
        ctas = std::min(b->ctas_max, std::max(ctas, b->aa_ctas_min));
        ctl.radius = 1;
        switch (b->storage) {
        case LBM_F64:
            return lbm::launch_aa_batch_f64(b->d_tiles, b->ntiles, static_cast<lbm::StepParams<double> *>(b->d_params),
                                            n, ctl, b->warps, ctas, s);
        case LBM_F32:
            return lbm::launch_aa_batch_f32(b->d_tiles, b->ntiles, static_cast<lbm::StepParams<float> *>(b->d_params),
                                            n, ctl, b->warps, ctas, s);
        case LBM_F16:
            return lbm::launch_aa_batch_f16(b->d_tiles, b->ntiles, static_cast<lbm::StepParams<float> *>(b->d_params),
                                            n, ctl, b->warps, ctas, s);
        default:
            return lbm::launch_aa_batch_bf16(b->d_tiles, b->ntiles, static_cast<lbm::StepParams<float> *>(b->d_params),
                                             n, ctl, b->warps, ctas, s);
        }
    }
    switch (b->storage) {
    case LBM_F64:
        return lbm::launch_batch_f64(b->d_tiles, b->ntiles, static_cast<lbm::StepParams<double> *>(b->d_params), n,
                                     ctl, b->warps, ctas, b->far ? 1 : 0, b->nv, s);
    case LBM_F32:
        return lbm::launch_batch_f32(b->d_tiles, b->ntiles, static_cast<lbm::StepParams<float> *>(b->d_params), n,
                                     ctl, b->warps, ctas, b->far ? 1 : 0, b->nv, s);
    case LBM_F16:
        return lbm::launch_batch_f16(b->d_tiles, b->ntiles, static_cast<lbm::StepParams<float> *>(b->d_params), n,
                                     ctl, b->warps, ctas, b->far ? 1 : 0, b->nv, s);
    case LBM_F16S:
        return lbm::launch_batch_f16s(b->d_tiles, b->ntiles, static_cast<lbm::StepParams<float> *>(b->d_params), n,
                                      ctl, b->warps, ctas, b->far ? 1 : 0, b->nv, s);
    case LBM_BF16S:
        return lbm::launch_batch_bf16s(b->d_tiles, b->ntiles, static_cast<lbm::StepParams<float> *>(b->d_params), n,
                                       ctl, b->warps, ctas, b->far ? 1 : 0, b->nv, s);
    default:
        return lbm::launch_batch_bf16(b->d_tiles, b->ntiles, static_cast<lbm::StepParams<float> *>(b->d_params), n,
                                      ctl, b->warps, ctas, b->far ? 1 : 0, b->nv, s);
    }
}

// steps per batch launch: the work counter stays below 2^31
int64_t batch_steps_per_launch(const lbm_batch *b)
{
    return std::max<int64_t>(1, ((int64_t)1 << 31) / std::max<int64_t>(1, 2 * (int64_t)b->ntiles));
}

// a graph of one launch of kGraphSteps steps, captured once per table
// version; the executable graph is updated in place (launches already queued
// keep their parameters), or re-instantiated once the batch's queued work
// has run if the update is refused
int batch_graph(lbm_batch *b)
{
    if (b->graph && b->graph_version == b->version)
        return LBM_OK;
    cudaGraph_t g = nullptr;
    const int steps = (int)std::min<int64_t>(kGraphSteps, batch_steps_per_launch(b));
    cudaError_t e = cudaStreamBeginCapture(b->capture, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess)
        e = batch_launch(b, steps, b->capture);
    cudaError_t e2 = cudaStreamEndCapture(b->capture, &g);
    if (e == cudaSuccess)
        e = e2;
    bool updated = false;
    if (e == cudaSuccess && b->graph) {
        cudaGraphExecUpdateResultInfo info;
        updated = cudaGraphExecUpdate(b->graph, g, &info) == cudaSuccess;
        if (!updated) {
            cudaGetLastError();
            if (b->launched)
                cudaEventSynchronize(b->last);
            drop_graph(b);
        }
    }
    if (e == cudaSuccess && !updated)
        e = cudaGraphInstantiate(&b->graph, g, 0);
    if (g)
        cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        b->graph = nullptr;
        cudaGetLastError();
        return cuda_fail(e, "capturing the batch step graph");
    }
    b->graph_version = b->version;
    b->graph_steps = steps;
    return LBM_OK;
}

void batch_advance_host(lbm_batch *b, int nsteps)
{
    for (lbm_lattice *h : b->members) {
        h->step += nsteps;
        if (h->aa)
            h->phase ^= nsteps & 1;
        else if (nsteps & 1)
            h->cur = 1 - h->cur;
        if (nsteps > 0)
            h->prev_valid = true;
    }
}

// fill an lbm_diag from the folded FP64 slots of the diagnostics reduction
int finish_diag(const double *v, int have_prev, lbm_diag *out)
{
    out->mass = v[0];
    out->mass_axi = v[1];
    out->heat = v[2];
    out->heat_axi = v[3];
    out->max_speed = v[6];
    const double nan = std::nan("");
    out->residual_l2 = (have_prev && v[8] > 0.0) ? std::sqrt(v[4] / v[8]) : nan;
    out->residual_max = (have_prev && v[6] > 0.0) ? v[5] / v[6] : nan;
    out->nonfinite = (int64_t)v[7];
    if (out->nonfinite > 0)
        return fail(LBM_ERR_DIVERGED, "%lld nodes with non-finite or non-positive density or temperature",
                    (long long)out->nonfinite);
    return LBM_OK;
}

}  // namespace

namespace lbm {

int lattice_view(const lbm_lattice *h, LatticeView *out)
{
    if (!valid(h) || !out)
        return fail(LBM_ERR_INVALID_ARG, "bad handle or NULL output");
    out->storage = h->d.storage;
    out->device = h->device;
    out->prev_valid = h->prev_valid && !h->aa ? 1 : 0;
    out->nx = h->d.nx;
    out->nr = h->d.nr;
    if (h->d.storage == LBM_F64)
        out->pd = params_d(h);
    else
        out->pf = params_f(h);
    return LBM_OK;
}

int api_fail(int code, const char *msg) { return fail(code, "%s", msg); }

int lattice_enter(const lbm_lattice *h, cudaStream_t s) { return enter(h, s); }

int lattice_leave(lbm_lattice *h, cudaStream_t s, int rc) { return leave(h, s, rc); }

int diag_finish(const double *v, int have_prev, lbm_diag *out) { return finish_diag(v, have_prev, out); }

}  // namespace lbm

extern "C" {

const char *lbm_last_error(void) { return g_err; }

int lbm_required_bytes(const lbm_desc *d, size_t *bytes)
{
    int rc = check_desc(d);
    if (rc)
        return rc;
    if (!bytes)
        return fail(LBM_ERR_INVALID_ARG, "bytes is NULL");
    *bytes = make_layout(d).total;
    return LBM_OK;
}

int lbm_create(const lbm_desc *d, void *dev_mem, size_t bytes, lbm_lattice **out)
{
    g_err[0] = 0;
    int rc = check_desc(d);
    if (rc)
        return rc;
    if (!out)
        return fail(LBM_ERR_INVALID_ARG, "out is NULL");
    Layout L = make_layout(d);
    if (dev_mem && bytes < L.total)
        return fail(LBM_ERR_OOM, "caller memory holds %zu bytes, the lattice needs %zu", bytes, L.total);
    if (dev_mem && (reinterpret_cast<uintptr_t>(dev_mem) % kAlign) != 0)
        return fail(LBM_ERR_INVALID_ARG, "caller memory must be 256-byte aligned");
    lbm_lattice *h = new (std::nothrow) lbm_lattice();
    if (!h)
        return fail(LBM_ERR_OOM, "host allocation failed");
    h->d = *d;
    h->L = L;
    h->batch = nullptr;
    h->prev_valid = false;
    h->own = dev_mem == nullptr;
    h->cur = 0;
    h->step = 0;
    h->band = 0;
    h->warps = 1;
    h->group = 0;
    h->aa = d->pattern == LBM_PATTERN_AA;
    h->phase = 0;
    h->nv = default_nv(d->storage);
    h->sync_items = 0;
    h->sync_cbase = h->sync_fbase = 0;
    h->sync_captured = false;
    cudaGetDevice(&h->device);
    h->sms = 1;
    cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, h->device);
    // Set-up is enqueued on the legacy default stream with no host
    // synchronisation: work of other streams is ordered after it through the
    // `ready` event (enter), so creating a lattice never drains the device.
    cudaStream_t s0 = nullptr;
    h->ready = h->last = nullptr;
    cudaError_t e = cudaEventCreateWithFlags(&h->ready, cudaEventDisableTiming);
    if (e == cudaSuccess)
        e = cudaEventCreateWithFlags(&h->last, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        if (h->ready)
            cudaEventDestroy(h->ready);
        delete h;
        cudaGetLastError();
        return cuda_fail(e, "creating the lattice's events");
    }
    auto undo = [&]() {
        if (h->own)
            cudaFreeAsync(h->mem, s0);
        cudaEventDestroy(h->ready);
        cudaEventDestroy(h->last);
        delete h;
    };
    if (h->own) {
        void *p = nullptr;
        e = cudaMallocAsync(&p, L.total, s0);
        if (e != cudaSuccess) {
            h->own = false;
            undo();
            cudaGetLastError();
            return fail(LBM_ERR_OOM, "cudaMallocAsync of %zu bytes: %s", L.total, cudaGetErrorString(e));
        }
        h->mem = static_cast<char *>(p);
    } else {
        h->mem = static_cast<char *>(dev_mem);
    }
    // rest state: every stored deviation is zero
    e = cudaMemsetAsync(h->mem, 0, L.total, s0);
    if (e != cudaSuccess) {
        undo();
        return cuda_fail(e, "initialising lattice memory");
    }
    // defaults: no inflow, T_in = T0, nu = alpha = 0.1 on [T0, T0 + 1]
    std::vector<double> zeros((size_t)d->nr, 0.0), tin((size_t)d->nr, d->T0);
    const double one = 0.1;
    h->ntab = 1;
    h->T_lo = d->T0;
    h->T_hi = d->T0 + 1.0;
    rc = upload_pair(h, L.off_uin_d, L.off_uin_f, zeros.data(), d->nr, s0, "inlet upload");
    if (!rc) rc = upload_pair(h, L.off_tin_d, L.off_tin_f, tin.data(), d->nr, s0, "inlet upload");
    if (!rc) rc = upload_pair(h, L.off_nu_d, L.off_nu_f, &one, 1, s0, "table upload");
    if (!rc) rc = upload_pair(h, L.off_al_d, L.off_al_f, &one, 1, s0, "table upload");
    if (!rc)
        rc = plan_launch(h);
    if (!rc)
        rc = fill_ghosts(h, s0);
    if (!rc) {
        e = cudaEventRecord(h->ready, s0);
        if (e == cudaSuccess)
            e = cudaEventRecord(h->last, s0);
        if (e != cudaSuccess)
            rc = cuda_fail(e, "recording the end of the set-up");
    }
    if (rc) {
        undo();
        return rc;
    }
    *out = h;
    return LBM_OK;
}

void lbm_destroy(lbm_lattice *h)
{
    if (!h)
        return;
    if (h->batch)
        lbm_batch_remove(h->batch, h);
    if (h->own && h->mem) {
        // released in stream order after the lattice's last use: no host synchronisation
        cudaStreamWaitEvent(nullptr, h->last, 0);
        cudaFreeAsync(h->mem, nullptr);
    }
    h->mem = nullptr;
    cudaEventDestroy(h->ready);
    cudaEventDestroy(h->last);
    delete h;
}

static int set_inlet_impl(lbm_lattice *h, const double *u_in, const double *T_in, int32_t nr, lbm_stream stream)
{
    if (!valid(h) || !u_in || !T_in)
        return fail(LBM_ERR_INVALID_ARG, "bad handle or NULL profile");
    if (nr != h->d.nr)
        return fail(LBM_ERR_INVALID_ARG, "profile length %d != nr %d", nr, h->d.nr);
    for (int j = 0; j < nr; ++j)
        if (!std::isfinite(u_in[j]) || !std::isfinite(T_in[j]))
            return fail(LBM_ERR_INVALID_ARG, "non-finite inlet value at row %d", j);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int rc = upload_pair(h, h->L.off_uin_d, h->L.off_uin_f, u_in, nr, s, "inlet upload");
    if (!rc)
        rc = upload_pair(h, h->L.off_tin_d, h->L.off_tin_f, T_in, nr, s, "inlet upload");
    if (!rc)
        rc = fill_ghosts(h, s);  // the inlet ghosts carry the profile
    if (h->batch)
        h->batch->dirty = true;
    return rc;
}

static int set_properties_impl(lbm_lattice *h, const double *nu, const double *alpha, int32_t n, double T_lo, double T_hi,
                       lbm_stream stream)
{
    if (!valid(h) || !nu || !alpha)
        return fail(LBM_ERR_INVALID_ARG, "bad handle or NULL table");
    if (n < 1 || n > kMaxTable)
        return fail(LBM_ERR_INVALID_ARG, "table length %d outside [1, %d]", n, kMaxTable);
    if (n > 1 && !(T_hi > T_lo))
        return fail(LBM_ERR_INVALID_ARG, "need T_hi > T_lo");
    for (int k = 0; k < n; ++k)
        if (!(nu[k] > 0.0) || !(alpha[k] > 0.0) || !std::isfinite(nu[k]) || !std::isfinite(alpha[k]))
            return fail(LBM_ERR_INVALID_ARG, "table entry %d must be finite and > 0 (tau > 1/2)", k);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int rc = upload_pair(h, h->L.off_nu_d, h->L.off_nu_f, nu, n, s, "table upload");
    if (!rc)
        rc = upload_pair(h, h->L.off_al_d, h->L.off_al_f, alpha, n, s, "table upload");
    if (rc)
        return rc;
    h->ntab = n;
    h->T_lo = T_lo;
    h->T_hi = n > 1 ? T_hi : T_lo + 1.0;
    if (h->batch)
        h->batch->dirty = true;
    return LBM_OK;
}

static int step_impl(lbm_lattice *h, int32_t nsteps, lbm_stream stream)
{
    if (!valid(h) || nsteps < 0)
        return fail(LBM_ERR_INVALID_ARG, "bad handle or negative step count");
    if (h->batch)
        return fail(LBM_ERR_INVALID_ARG, "the lattice belongs to a batch: step the batch");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const lbm_desc &d = h->d;
    lbm::RunCtl ctl;
    ctl.group = item_group(h);
    if (h->aa) {
        const AAPlan a = aa_plan(h);
        unsigned *sync = h->at<unsigned>(h->L.off_sync);
        ctl.group = a.group;
        ctl.counter = sync;
        ctl.flags = sync + 1;
        ctl.radius = 1;
        ctl.wrap = d.bc_in == LBM_IN_PERIODIC ? 1 : 0;
        ctl.spin_limit = lbm::RUN_SPIN_LIMIT;
        for (int64_t done = 0; done < nsteps;) {
            const int m = (int)std::min<int64_t>(a.per_launch, nsteps - done);
            cudaError_t e = cudaMemsetAsync(sync, 0, (size_t)4 * (size_t)(1 + 2 * a.items), s);
            if (e != cudaSuccess)
                return cuda_fail(e, "work counter reset");
            ctl.nsteps = m;
            e = aa_launch(h, ctl, a.ctas, s);
            if (e != cudaSuccess)
                return cuda_fail(e, "step kernel launch");
            h->phase ^= (m & 1);
            h->step += m;
            h->prev_valid = true;
            done += m;
        }
        return LBM_OK;
    }
    const int nstrips = (d.nx + 32 * h->nv - 1) / (32 * h->nv);
    const int64_t items = (int64_t)lbm::item_cols(nstrips, ctl.group) * ((d.nr + h->band_eff - 1) / h->band_eff);
    // steps per launch: the work indices of one launch stay below 2^31
    const int64_t per_launch = std::max<int64_t>(1, ((int64_t)1 << 31) / std::max<int64_t>(1, 2 * items));
    unsigned *sync = h->at<unsigned>(h->L.off_sync);
    ctl.counter = sync;
    ctl.flags = sync + 1;
    ctl.radius = h->band_eff >= 2 ? 1 : 2;
    ctl.wrap = d.bc_in == LBM_IN_PERIODIC ? 1 : 0;
    ctl.spin_limit = lbm::RUN_SPIN_LIMIT;
    // The counters carry on from the previous launch (RunCtl) unless the item
    // count changed, a wait ran out (lbm_check) or the launch goes into a graph,
    // whose replays must each start from a reset.
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cap) != cudaSuccess)
        return cuda_fail(cudaGetLastError(), "querying the stream");
    if (cap != cudaStreamCaptureStatusNone)
        h->sync_captured = true;
    for (int64_t done = 0; done < nsteps;) {
        const int m = (int)std::min<int64_t>(per_launch, nsteps - done);
        cudaError_t e = cudaSuccess;
        if (h->sync_items != items || h->sync_captured) {
            e = cudaMemsetAsync(sync, 0, (size_t)4 * (size_t)(1 + items), s);
            if (e != cudaSuccess) {
                h->sync_items = 0;
                return cuda_fail(e, "work counter reset");
            }
            h->sync_items = items;
            h->sync_cbase = h->sync_fbase = 0;
        }
        ctl.nsteps = m;
        ctl.cbase = h->sync_cbase;
        ctl.fbase = h->sync_fbase;
        ctl.first = 0;
        const int ctas = (int)std::min<int64_t>(h->ctas_max, (items + h->warps - 1) / h->warps);
        switch (d.storage) {
        case LBM_F64: e = lbm::launch_run_f64(params_d(h), ctl, h->warps, ctas, h->nv, s); break;
        case LBM_F32: e = lbm::launch_run_f32(params_f(h), ctl, h->warps, ctas, h->nv, s); break;
        case LBM_F16: e = lbm::launch_run_f16(params_f(h), ctl, h->warps, ctas, h->nv, s); break;
        case LBM_F16S: e = lbm::launch_run_f16s(params_f(h), ctl, h->warps, ctas, h->nv, s); break;
        case LBM_BF16S: e = lbm::launch_run_bf16s(params_f(h), ctl, h->warps, ctas, h->nv, s); break;
        default: e = lbm::launch_run_bf16(params_f(h), ctl, h->warps, ctas, h->nv, s); break;
        }
        if (e != cudaSuccess) {
            h->sync_items = 0;
            return cuda_fail(e, "step kernel launch");
        }
        h->sync_cbase += (unsigned)m * (unsigned)items + (unsigned)ctas * (unsigned)h->warps;
        h->sync_fbase += 32u * (unsigned)(m - 1);
        h->cur ^= (m & 1);
        h->step += m;
        h->prev_valid = true;
        done += m;
    }
    return LBM_OK;
}

int lbm_selftest_wait_timeout(lbm_lattice *h, int32_t *flags)
{
    if (!valid(h) || !flags)
        return fail(LBM_ERR_INVALID_ARG, "bad handle or NULL output");
    if (h->batch)
        return fail(LBM_ERR_INVALID_ARG, "the lattice belongs to a batch");
    cudaStream_t s = nullptr;
    int rc = lbm_check(h, flags);  // start from a clear status
    if (rc)
        return rc;
    const lbm_desc &d = h->d;
    lbm::RunCtl ctl;
    ctl.group = item_group(h);
    const int nstrips = (d.nx + 32 * h->nv - 1) / (32 * h->nv);
    const unsigned items = (unsigned)lbm::item_cols(nstrips, ctl.group) * (unsigned)((d.nr + h->band_eff - 1) / h->band_eff);
    unsigned *sync = h->at<unsigned>(h->L.off_sync);
    ctl.counter = sync;
    ctl.flags = sync + 1;
    ctl.radius = h->band_eff >= 2 ? 1 : 2;
    ctl.wrap = d.bc_in == LBM_IN_PERIODIC ? 1 : 0;
    ctl.spin_limit = 64;  // a few tens of microseconds
    ctl.nsteps = 2;
    if (h->aa) {
        // every counter at zero and the work counter past sub-step 0: each
        // item taken belongs to sub-step 1 and waits for a sub-step that never runs
        const AAPlan a = aa_plan(h);
        ctl.group = a.group;
        ctl.radius = 1;
        const unsigned start = (unsigned)a.items;
        cudaError_t e = cudaMemsetAsync(sync, 0, (size_t)4 * (size_t)(1 + 2 * a.items), s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(sync, &start, sizeof(unsigned), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess)
            e = aa_launch(h, ctl, a.ctas, s);
        if (e != cudaSuccess)
            return cuda_fail(e, "self-test launch");
        int32_t first = 0;
        rc = lbm_check(h, &first);
        if (rc)
            return rc;
        if (a.items < 2) {  // one item has no neighbour whose edges it could wait for
            *flags = first;
            return LBM_OK;
        }
        // the mid-item wait: only the last item of one step runs; it publishes its
        // edges and waits for those of neighbours that never run (the populations are
        // not written; the edges it wrote are recomputed by the next step)
        ctl.nsteps = 1;
        const unsigned last = (unsigned)(a.items - 1);
        e = cudaMemsetAsync(sync, 0, (size_t)4 * (size_t)(1 + 2 * a.items), s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(sync, &last, sizeof(unsigned), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess)
            e = aa_launch(h, ctl, a.ctas, s);
        if (e != cudaSuccess)
            return cuda_fail(e, "self-test launch");
        int32_t second = 0;
        rc = lbm_check(h, &second);
        if (rc)
            return rc;
        *flags = first & second;  // LBM_STATUS_TIMEOUT only if both waits gave up
        return LBM_OK;
    }
    // every counter at zero and the first item past sub-step 0: each item
    // taken belongs to sub-step 1 and waits for a sub-step that never runs
    h->sync_items = 0;  // the next lbm_step starts from a reset
    ctl.first = items;
    cudaError_t e = cudaMemsetAsync(sync, 0, (size_t)4 * (size_t)(1 + items), s);
    if (e == cudaSuccess) {
        const int ctas = (int)std::min<int64_t>(h->ctas_max, ((int64_t)items + h->warps - 1) / h->warps);
        switch (d.storage) {
        case LBM_F64: e = lbm::launch_run_f64(params_d(h), ctl, h->warps, ctas, h->nv, s); break;
        case LBM_F32: e = lbm::launch_run_f32(params_f(h), ctl, h->warps, ctas, h->nv, s); break;
        case LBM_F16: e = lbm::launch_run_f16(params_f(h), ctl, h->warps, ctas, h->nv, s); break;
        case LBM_F16S: e = lbm::launch_run_f16s(params_f(h), ctl, h->warps, ctas, h->nv, s); break;
        case LBM_BF16S: e = lbm::launch_run_bf16s(params_f(h), ctl, h->warps, ctas, h->nv, s); break;
        default: e = lbm::launch_run_bf16(params_f(h), ctl, h->warps, ctas, h->nv, s); break;
        }
    }
    if (e != cudaSuccess)
        return cuda_fail(e, "self-test launch");
    return lbm_check(h, flags);  // synchronises, reads and clears the status
}

int lbm_set_item_group(lbm_lattice *h, int32_t group)
{
    if (!valid(h) || group < 0 || group > 64)
        return fail(LBM_ERR_INVALID_ARG, "bad handle or group (0..64)");
    h->group = group;
    return LBM_OK;
}

int32_t lbm_get_item_group(const lbm_lattice *h) { return valid(h) ? item_group(h) : -1; }

int64_t lbm_get_step(const lbm_lattice *h) { return valid(h) ? h->step : -1; }

static int diagnostics_impl(lbm_lattice *h, lbm_diag *out, lbm_stream stream)
{
    if (!valid(h) || !out)
        return fail(LBM_ERR_INVALID_ARG, "bad handle or NULL output");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int64_t N = (int64_t)h->d.nx * h->d.nr;
    const int nblocks = (int)std::min<int64_t>(
        {(int64_t)lbm::DIAG_MAX_BLOCKS, (N + lbm::DIAG_THREADS - 1) / lbm::DIAG_THREADS, 4 * (int64_t)h->sms});
    double *partials = h->at<double>(h->L.off_diag);
    double *res = partials + (size_t)lbm::DIAG_MAX_BLOCKS * lbm::DIAG_SLOTS;
    const int prev = h->prev_valid && !h->aa ? 1 : 0;  // an AA lattice keeps no previous state
    cudaError_t e;
    switch (h->d.storage) {
    case LBM_F64: e = lbm::launch_diag_f64(params_d(h), prev, partials, nblocks, res, s); break;
    case LBM_F32: e = lbm::launch_diag_f32(params_f(h), prev, partials, nblocks, res, s); break;
    case LBM_F16: e = lbm::launch_diag_f16(params_f(h), prev, partials, nblocks, res, s); break;
    case LBM_F16S: e = lbm::launch_diag_f16s(params_f(h), prev, partials, nblocks, res, s); break;
    case LBM_BF16S: e = lbm::launch_diag_bf16s(params_f(h), prev, partials, nblocks, res, s); break;
    default: e = lbm::launch_diag_bf16(params_f(h), prev, partials, nblocks, res, s); break;
    }
    double v[lbm::DIAG_SLOTS];
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(v, res, sizeof(v), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(s);
    if (e != cudaSuccess)
        return cuda_fail(e, "diagnostics");
    return finish_diag(v, prev, out);
}

int lbm_check(lbm_lattice *h, int32_t *flags)
{
    if (!valid(h) || !flags)
        return fail(LBM_ERR_INVALID_ARG, "bad handle or NULL flags");
    int v = 0;
    cudaError_t e = cudaMemcpy(&v, h->mem + h->L.off_status, sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess)
        e = cudaMemset(h->mem + h->L.off_status, 0, sizeof(int));
    if (e != cudaSuccess)
        return cuda_fail(e, "reading the status word");
    if (v & lbm::STATUS_TIMEOUT)
        h->sync_items = 0;  // a launch stopped early: its counters are not where the host expects
    *flags = v;
    return LBM_OK;
}

static int get_fields_impl(lbm_lattice *h, void *dev_out, int32_t out_type, lbm_stream stream)
{
    if (!valid(h) || !dev_out)
        return fail(LBM_ERR_INVALID_ARG, "bad handle or NULL output");
    if (out_type != LBM_F64 && out_type != LBM_F32)
        return fail(LBM_ERR_INVALID_ARG, "out_type must be LBM_F64 or LBM_F32");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int f64 = out_type == LBM_F64;
    cudaError_t e;
    switch (h->d.storage) {
    case LBM_F64: e = lbm::launch_fields_f64(params_d(h), dev_out, f64, s); break;
    case LBM_F32: e = lbm::launch_fields_f32(params_f(h), dev_out, f64, s); break;
    case LBM_F16: e = lbm::launch_fields_f16(params_f(h), dev_out, f64, s); break;
    case LBM_F16S: e = lbm::launch_fields_f16s(params_f(h), dev_out, f64, s); break;
    case LBM_BF16S: e = lbm::launch_fields_bf16s(params_f(h), dev_out, f64, s); break;
    default: e = lbm::launch_fields_bf16(params_f(h), dev_out, f64, s); break;
    }
    return e == cudaSuccess ? LBM_OK : cuda_fail(e, "fields kernel launch");
}

static int get_state_impl(lbm_lattice *h, double *dev_f, double *dev_g, lbm_stream stream)
{
    if (!valid(h) || !dev_f || !dev_g)
        return fail(LBM_ERR_INVALID_ARG, "bad handle or NULL output");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const lbm_desc &d = h->d;
    const void *b = h->buf(h->cur);
    cudaError_t e;
    if (h->aa) {
        switch (d.storage) {
        case LBM_F64: e = lbm::launch_aa_state_out_f64(b, h->phase, dev_f, dev_g, d.nx, d.nr, h->L.pitch, h->L.plane, d.rho0, d.T0, s); break;
        case LBM_F32: e = lbm::launch_aa_state_out_f32(b, h->phase, dev_f, dev_g, d.nx, d.nr, h->L.pitch, h->L.plane, d.rho0, d.T0, s); break;
        case LBM_F16: e = lbm::launch_aa_state_out_f16(b, h->phase, dev_f, dev_g, d.nx, d.nr, h->L.pitch, h->L.plane, d.rho0, d.T0, s); break;
        default: e = lbm::launch_aa_state_out_bf16(b, h->phase, dev_f, dev_g, d.nx, d.nr, h->L.pitch, h->L.plane, d.rho0, d.T0, s); break;
        }
        return e == cudaSuccess ? LBM_OK : cuda_fail(e, "state read kernel launch");
    }
    switch (d.storage) {
    case LBM_F64: e = lbm::launch_state_out_f64(b, dev_f, dev_g, d.nx, d.nr, h->L.pitch, h->L.plane, d.rho0, d.T0, s); break;
    case LBM_F32: e = lbm::launch_state_out_f32(b, dev_f, dev_g, d.nx, d.nr, h->L.pitch, h->L.plane, d.rho0, d.T0, s); break;
    case LBM_F16: e = lbm::launch_state_out_f16(b, dev_f, dev_g, d.nx, d.nr, h->L.pitch, h->L.plane, d.rho0, d.T0, s); break;
    case LBM_F16S: e = lbm::launch_state_out_f16s(b, dev_f, dev_g, d.nx, d.nr, h->L.pitch, h->L.plane, d.rho0, d.T0, s); break;
    case LBM_BF16S: e = lbm::launch_state_out_bf16s(b, dev_f, dev_g, d.nx, d.nr, h->L.pitch, h->L.plane, d.rho0, d.T0, s); break;
    default: e = lbm::launch_state_out_bf16(b, dev_f, dev_g, d.nx, d.nr, h->L.pitch, h->L.plane, d.rho0, d.T0, s); break;
    }
    return e == cudaSuccess ? LBM_OK : cuda_fail(e, "state read kernel launch");
}

static int set_state_impl(lbm_lattice *h, const double *dev_f, const double *dev_g, int64_t step, lbm_stream stream)
{
    if (!valid(h) || !dev_f || !dev_g || step < 0)
        return fail(LBM_ERR_INVALID_ARG, "bad handle, NULL input or negative step");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const lbm_desc &d = h->d;
    void *b = h->buf(h->cur);
    cudaError_t e;
    if (h->aa) {  // written in representation 0
        switch (d.storage) {
        case LBM_F64: e = lbm::launch_aa_state_in_f64(b, dev_f, dev_g, d.nx, d.nr, h->L.pitch, h->L.plane, d.rho0, d.T0, s); break;
        case LBM_F32: e = lbm::launch_aa_state_in_f32(b, dev_f, dev_g, d.nx, d.nr, h->L.pitch, h->L.plane, d.rho0, d.T0, s); break;
        case LBM_F16: e = lbm::launch_aa_state_in_f16(b, dev_f, dev_g, d.nx, d.nr, h->L.pitch, h->L.plane, d.rho0, d.T0, s); break;
        default: e = lbm::launch_aa_state_in_bf16(b, dev_f, dev_g, d.nx, d.nr, h->L.pitch, h->L.plane, d.rho0, d.T0, s); break;
        }
        h->phase = 0;
    } else {
        switch (d.storage) {
        case LBM_F64: e = lbm::launch_state_in_f64(b, dev_f, dev_g, d.nx, d.nr, h->L.pitch, h->L.plane, d.rho0, d.T0, s); break;
        case LBM_F32: e = lbm::launch_state_in_f32(b, dev_f, dev_g, d.nx, d.nr, h->L.pitch, h->L.plane, d.rho0, d.T0, s); break;
        case LBM_F16: e = lbm::launch_state_in_f16(b, dev_f, dev_g, d.nx, d.nr, h->L.pitch, h->L.plane, d.rho0, d.T0, s); break;
        case LBM_F16S: e = lbm::launch_state_in_f16s(b, dev_f, dev_g, d.nx, d.nr, h->L.pitch, h->L.plane, d.rho0, d.T0, s); break;
        case LBM_BF16S: e = lbm::launch_state_in_bf16s(b, dev_f, dev_g, d.nx, d.nr, h->L.pitch, h->L.plane, d.rho0, d.T0, s); break;
        default: e = lbm::launch_state_in_bf16(b, dev_f, dev_g, d.nx, d.nr, h->L.pitch, h->L.plane, d.rho0, d.T0, s); break;
        }
    }
    if (e != cudaSuccess)
        return cuda_fail(e, "state write kernel launch");
    h->step = step;
    h->prev_valid = false;
    if (h->batch)
        h->batch->dirty = true;
    return fill_ghosts(h, s);
}

int lbm_checkpoint_bytes(const lbm_lattice *h, size_t *bytes)
{
    if (!valid(h) || !bytes)
        return fail(LBM_ERR_INVALID_ARG, "bad handle or NULL output");
    *bytes = (size_t)13 * (size_t)h->d.nr * (size_t)h->d.nx * storage_bytes(h->d.storage);
    if (is_split(h->d.storage))  // then the FP32 moment planes
        *bytes += (size_t)lbm::SPLIT_MOMENTS * (size_t)h->d.nr * (size_t)h->d.nx * 4;
    return LBM_OK;
}

// one strided copy per plane between the padded buffer and a dense [q][j][i]
// array of post-collision values: plane q at its nodes (two buffers), or
// in the AA pattern the window of the representation's plane that holds
// population q of every node (lbm::aa_post_cell; restores write
// representation 0)
static int copy_planes(lbm_lattice *h, void *dense, bool out, cudaStream_t s)
{
    const size_t es = storage_bytes(h->d.storage);
    const size_t row = (size_t)h->d.nx * es;
    const size_t pitch = (size_t)h->L.pitch * es;
    char *buf = static_cast<char *>(h->buf(h->cur));
    const int phase = h->aa && out ? h->phase : 0;
    for (int q = 0; q < 13; ++q) {
        const int64_t first = h->aa ? lbm::aa_post_cell(phase, q, 0, 0, h->L.pitch, h->L.plane)
                                    : (int64_t)q * h->L.plane + h->L.pitch + lbm::PAD_COLS;
        char *padded = buf + (size_t)first * es;
        char *flat = static_cast<char *>(dense) + (size_t)q * (size_t)h->d.nr * row;
        cudaError_t e = out ? cudaMemcpy2DAsync(flat, row, padded, pitch, row, h->d.nr, cudaMemcpyDeviceToDevice, s)
                            : cudaMemcpy2DAsync(padded, pitch, flat, row, row, h->d.nr, cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess)
            return cuda_fail(e, "checkpoint plane copy");
    }
    if (is_split(h->d.storage)) {  // then the (j_x, j_r) pairs, then T - T0, without ghosts or padding
        char *mbase = buf + lbm::split_moff(h->L.plane);
        char *mflat = static_cast<char *>(dense) + (size_t)13 * (size_t)h->d.nr * row;
        for (int m = 0; m < 2; ++m) {  // m = 0: pairs (8 bytes a node), m = 1: T - T0 (4 bytes)
            const size_t es_m = m == 0 ? 8 : 4;
            const size_t mrow = (size_t)h->d.nx * es_m, mpitch = (size_t)h->L.pitch * es_m;
            char *padded = mbase + (m == 0 ? 0 : (size_t)h->L.plane * 8) +
                           ((size_t)h->L.pitch + lbm::PAD_COLS) * es_m;
            char *flat = mflat + (m == 0 ? 0 : (size_t)h->d.nr * (size_t)h->d.nx * 8);
            cudaError_t e = out ? cudaMemcpy2DAsync(flat, mrow, padded, mpitch, mrow, h->d.nr, cudaMemcpyDeviceToDevice, s)
                                : cudaMemcpy2DAsync(padded, mpitch, flat, mrow, mrow, h->d.nr, cudaMemcpyDeviceToDevice, s);
            if (e != cudaSuccess)
                return cuda_fail(e, "checkpoint moment plane copy");
        }
    }
    return LBM_OK;
}

static int save_impl(lbm_lattice *h, void *dev_out, lbm_stream stream)
{
    if (!valid(h) || !dev_out)
        return fail(LBM_ERR_INVALID_ARG, "bad handle or NULL output");
    return copy_planes(h, dev_out, true, static_cast<cudaStream_t>(stream));
}

static int restore_impl(lbm_lattice *h, const void *dev_in, int64_t step, lbm_stream stream)
{
    if (!valid(h) || !dev_in || step < 0)
        return fail(LBM_ERR_INVALID_ARG, "bad handle, NULL input or negative step");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int rc = copy_planes(h, const_cast<void *>(dev_in), false, s);
    if (rc != LBM_OK)
        return rc;
    h->phase = 0;
    h->step = step;
    h->prev_valid = false;
    if (h->batch)
        h->batch->dirty = true;
    return fill_ghosts(h, s);
}

int lbm_set_launch(lbm_lattice *h, int32_t band_rows, int32_t warps_per_cta)
{
    if (!valid(h) || band_rows < 0 || warps_per_cta < 0 || warps_per_cta > 8)
        return fail(LBM_ERR_INVALID_ARG, "bad handle or launch shape (warps per CTA 1..8)");
    h->band = band_rows;
    if (warps_per_cta > 0)
        h->warps = warps_per_cta;
    return plan_launch(h);
}

// the strip width a lattice or batch of this storage type accepts: 0 (the default), or 32
// columns (one node per lane) and, for FP32 arithmetic, 64 (two per lane); the AA pattern
// keeps its default
static int strip_nv(int storage, bool aa, int32_t cols, int *nv)
{
    if (cols == 0) {
        *nv = default_nv(storage);
        return LBM_OK;
    }
    if (aa && cols != 32 * default_nv(storage))
        return fail(LBM_ERR_INVALID_ARG, "the AA pattern keeps strips of %d columns", 32 * default_nv(storage));
    if (cols == 32 || (cols == 64 && storage != LBM_F64)) {
        *nv = cols / 32;
        return LBM_OK;
    }
    return fail(LBM_ERR_INVALID_ARG, "strip width %d: 0, 32%s", cols, storage == LBM_F64 ? "" : " or 64");
}

int lbm_set_strip_width(lbm_lattice *h, int32_t columns)
{
    if (!valid(h))
        return fail(LBM_ERR_INVALID_ARG, "bad handle");
    if (h->batch)
        return fail(LBM_ERR_INVALID_ARG, "the lattice belongs to a batch: set the batch's strip width");
    int nv = 0;
    int rc = strip_nv(h->d.storage, h->aa, columns, &nv);
    if (rc)
        return rc;
    const int old = h->nv;
    h->nv = nv;
    rc = plan_launch(h);
    if (rc)
        h->nv = old;
    return rc;
}

int32_t lbm_get_strip_width(const lbm_lattice *h) { return valid(h) ? 32 * h->nv : -1; }

int lbm_get_launch(const lbm_lattice *h, int32_t *band_rows, int32_t *warps_per_cta, int32_t *ctas)
{
    if (!valid(h))
        return fail(LBM_ERR_INVALID_ARG, "bad handle");
    if (band_rows)
        *band_rows = h->band_eff;
    if (warps_per_cta)
        *warps_per_cta = h->warps;
    if (ctas)
        *ctas = h->ctas;
    return LBM_OK;
}


int lbm_batch_create(int32_t storage, lbm_batch **out)
{
    if (!out || storage_bytes(storage) == 0)
        return fail(LBM_ERR_INVALID_ARG, "bad storage type or NULL out");
    lbm_batch *b = new (std::nothrow) lbm_batch();
    if (!b)
        return fail(LBM_ERR_OOM, "host allocation failed");
    b->storage = storage;
    b->dirty = true;
    b->warps = 1;
    b->nv = batch_default_nv(storage);
    int dev = 0;
    cudaGetDevice(&dev);
    b->sms = 1;
    cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev);
    cudaError_t e = cudaStreamCreateWithFlags(&b->capture, cudaStreamNonBlocking);
    if (e == cudaSuccess) {
        e = cudaEventCreateWithFlags(&b->last, cudaEventDisableTiming);
        if (e != cudaSuccess)
            cudaStreamDestroy(b->capture);
    }
    if (e != cudaSuccess) {
        delete b;
        return cuda_fail(e, "creating the capture stream");
    }
    b->launched = false;
    *out = b;
    return LBM_OK;
}

void lbm_batch_destroy(lbm_batch *b)
{
    if (!b)
        return;
    if (b->launched)
        cudaEventSynchronize(b->last);  // the batch's own queued launches, not the whole device
    for (lbm_lattice *h : b->members)
        h->batch = nullptr;
    drop_graph(b);
    for (void *p : {b->d_params, static_cast<void *>(b->d_tiles), static_cast<void *>(b->d_sync)})
        if (p)
            cudaFreeAsync(p, nullptr);
    cudaStreamDestroy(b->capture);
    cudaEventDestroy(b->last);
    delete b;
}

int lbm_batch_add(lbm_batch *b, lbm_lattice *h)
{
    if (!b || !valid(h))
        return fail(LBM_ERR_INVALID_ARG, "bad batch or lattice handle");
    if (h->batch)
        return fail(LBM_ERR_INVALID_ARG, "the lattice already belongs to a batch");
    if (h->d.storage != b->storage)
        return fail(LBM_ERR_INVALID_ARG, "storage type %d differs from the batch's %d", h->d.storage, b->storage);
    if (!b->members.empty() && b->members[0]->aa != h->aa)
        return fail(LBM_ERR_INVALID_ARG, "the members of a batch share one pattern");
    if (h->aa && b->nv != default_nv(b->storage))
        return fail(LBM_ERR_INVALID_ARG, "AA lattices join batches of the default strip width");
    b->members.push_back(h);
    h->batch = b;
    b->dirty = true;
    return LBM_OK;
}

int lbm_batch_remove(lbm_batch *b, lbm_lattice *h)
{
    if (!b || !h || h->batch != b)
        return fail(LBM_ERR_INVALID_ARG, "the lattice is not in this batch");
    for (size_t m = 0; m < b->members.size(); ++m)
        if (b->members[m] == h) {
            b->members.erase(b->members.begin() + (long)m);
            break;
        }
    h->batch = nullptr;
    b->dirty = true;
    if (b->launched) {  // the lattice's last use is the batch's last launch
        cudaError_t e = cudaStreamWaitEvent(nullptr, b->last, 0);
        if (e == cudaSuccess)
            e = cudaEventRecord(h->last, nullptr);
        if (e != cudaSuccess)
            return cuda_fail(e, "recording the lattice's last use");
    }
    return LBM_OK;
}

int32_t lbm_batch_size(const lbm_batch *b) { return b ? (int32_t)b->members.size() : -1; }

int lbm_batch_set_launch(lbm_batch *b, int32_t band_rows, int32_t warps_per_cta)
{
    if (!b || band_rows < 0 || warps_per_cta < 0 || warps_per_cta > 8)
        return fail(LBM_ERR_INVALID_ARG, "bad batch or launch shape (warps per CTA 1..8)");
    b->band = band_rows;
    if (warps_per_cta > 0)
        b->warps = warps_per_cta;
    b->dirty = true;
    return LBM_OK;
}

int lbm_batch_set_strip_width(lbm_batch *b, int32_t columns)
{
    if (!b)
        return fail(LBM_ERR_INVALID_ARG, "bad batch handle");
    int nv = 0;
    const bool aa = !b->members.empty() && b->members[0]->aa;
    int rc = strip_nv(b->storage, aa, columns, &nv);
    if (rc)
        return rc;
    b->nv = columns == 0 ? batch_default_nv(b->storage) : nv;
    b->dirty = true;
    return LBM_OK;
}

int32_t lbm_batch_get_strip_width(const lbm_batch *b) { return b ? 32 * b->nv : -1; }

int lbm_batch_get_launch(const lbm_batch *b, int32_t *band_rows, int32_t *warps_per_cta, int32_t *tiles)
{
    if (!b)
        return fail(LBM_ERR_INVALID_ARG, "bad batch handle");
    if (band_rows)
        *band_rows = b->band_eff;
    if (warps_per_cta)
        *warps_per_cta = b->warps;
    if (tiles)
        *tiles = b->ntiles;
    return LBM_OK;
}

int lbm_batch_step(lbm_batch *b, int32_t nsteps, int32_t use_graph, lbm_stream stream)
{
    if (!b || nsteps < 0)
        return fail(LBM_ERR_INVALID_ARG, "bad batch handle or negative step count");
    if (b->members.empty() || nsteps == 0)
        return LBM_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (b->dirty) {
        int rc = batch_rebuild(b, s);
        if (rc)
            return rc;
    }
    int done = 0;
    if (use_graph) {
        int rc = batch_graph(b);
        if (rc)
            return rc;
        for (; done + b->graph_steps <= nsteps; done += b->graph_steps) {
            cudaError_t e = cudaGraphLaunch(b->graph, s);
            if (e != cudaSuccess) {
                batch_advance_host(b, done);
                return cuda_fail(e, "batch graph launch");
            }
        }
    }
    while (done < nsteps) {
        const int m = (int)std::min<int64_t>(batch_steps_per_launch(b), nsteps - done);
        cudaError_t e = batch_launch(b, m, s);
        if (e != cudaSuccess) {
            batch_advance_host(b, done);
            return cuda_fail(e, "batch step launch");
        }
        done += m;
    }
    batch_advance_host(b, nsteps);
    cudaError_t e = cudaEventRecord(b->last, s);
    if (e != cudaSuccess)
        return cuda_fail(e, "recording the batch's last launch");
    b->launched = true;
    return LBM_OK;
}


// The entry points that enqueue work on a caller's stream: the stream is
// first ordered after the lattice's set-up, and the call's work is then
// recorded as the lattice's last use.

int lbm_set_inlet(lbm_lattice *h, const double *u_in, const double *T_in, int32_t nr, lbm_stream stream)
{
    if (!valid(h))
        return fail(LBM_ERR_INVALID_ARG, "bad lattice handle");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int rc = enter(h, s);
    return rc ? rc : leave(h, s, set_inlet_impl(h, u_in, T_in, nr, stream));
}

int lbm_set_properties(lbm_lattice *h, const double *nu, const double *alpha, int32_t n, double T_lo, double T_hi,
                       lbm_stream stream)
{
    if (!valid(h))
        return fail(LBM_ERR_INVALID_ARG, "bad lattice handle");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int rc = enter(h, s);
    return rc ? rc : leave(h, s, set_properties_impl(h, nu, alpha, n, T_lo, T_hi, stream));
}

int lbm_step(lbm_lattice *h, int32_t nsteps, lbm_stream stream)
{
    if (!valid(h))
        return fail(LBM_ERR_INVALID_ARG, "bad lattice handle");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int rc = enter(h, s);
    return rc ? rc : leave(h, s, step_impl(h, nsteps, stream));
}

int lbm_get_fields(lbm_lattice *h, void *dev_out, int32_t out_type, lbm_stream stream)
{
    if (!valid(h))
        return fail(LBM_ERR_INVALID_ARG, "bad lattice handle");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int rc = enter(h, s);
    return rc ? rc : leave(h, s, get_fields_impl(h, dev_out, out_type, stream));
}

int lbm_get_state(lbm_lattice *h, double *dev_f, double *dev_g, lbm_stream stream)
{
    if (!valid(h))
        return fail(LBM_ERR_INVALID_ARG, "bad lattice handle");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int rc = enter(h, s);
    return rc ? rc : leave(h, s, get_state_impl(h, dev_f, dev_g, stream));
}

int lbm_set_state(lbm_lattice *h, const double *dev_f, const double *dev_g, int64_t step, lbm_stream stream)
{
    if (!valid(h))
        return fail(LBM_ERR_INVALID_ARG, "bad lattice handle");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int rc = enter(h, s);
    return rc ? rc : leave(h, s, set_state_impl(h, dev_f, dev_g, step, stream));
}

int lbm_save(lbm_lattice *h, void *dev_out, lbm_stream stream)
{
    if (!valid(h))
        return fail(LBM_ERR_INVALID_ARG, "bad lattice handle");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int rc = enter(h, s);
    return rc ? rc : leave(h, s, save_impl(h, dev_out, stream));
}

int lbm_restore(lbm_lattice *h, const void *dev_in, int64_t step, lbm_stream stream)
{
    if (!valid(h))
        return fail(LBM_ERR_INVALID_ARG, "bad lattice handle");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int rc = enter(h, s);
    return rc ? rc : leave(h, s, restore_impl(h, dev_in, step, stream));
}

int lbm_diagnostics(lbm_lattice *h, lbm_diag *out, lbm_stream stream)
{
    if (!valid(h))
        return fail(LBM_ERR_INVALID_ARG, "bad lattice handle");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int rc = enter(h, s);
    return rc ? rc : leave(h, s, diagnostics_impl(h, out, stream));
}

}  // extern "C"
