// C-ABI of libwcsim: argument checks, the plane object and stream-ordered launches.
// Every entry point returns a wcsim_status; nothing here aborts or synchronizes the host
// except the calls whose contract says so (create, plane_check, stage_times).
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <cmath>
#include <new>
#include <vector>

#include "async_copy.cuh"
#include "wcsim_internal.cuh"

using namespace wcsim;

namespace {

thread_local char g_err[512] = "";

wcsim_status fail(wcsim_status s, const char* fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return s;
}

wcsim_status cuda_fail(cudaError_t e, const char* what)
{
    if (e == cudaErrorMemoryAllocation)
        return fail(WCSIM_ENOMEM, "%s: %s", what, cudaGetErrorString(e));
    return fail(WCSIM_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

// Make the plane's device current for the duration of a call and restore the caller's.
struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) { ok = false; return; }
        if (prev != dev && cudaSetDevice(dev) != cudaSuccess) ok = false;
    }
    ~DeviceGuard()
    {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

bool finite_pos(double x) { return isfinite(x) && x > 0.0; }

}  // namespace

constexpr int kStages = 5;       // forward: prep (zero grid or bin depos), rasterize,
                                 // rows_r2c (with the rasterization when fused), wire_pass,
                                 // rows_c2r
constexpr int kMarks = 32;       // forward timeline events
constexpr int kBwdStages = 7;    // backward: zero, rasterize, r2c(S), r2c(G), wire adjoint,
                                 // c2r of dL/dS, depo adjoint

struct wcsim_plane {
    wcsim_geometry g;
    wcsim_drift_params prm;
    ConvDims dims;
    FftPlan pt, pw;
    float2* tw_t = nullptr;
    float2* tw_w = nullptr;
    float2* tw_warp = nullptr;  // twiddles of the one-warp-per-column wire pass (or NULL)
    float2* H = nullptr;        // Hermitian part of R / (n_fw n_ft), [n_imp][4 nkb][n_fw]
    float* grid = nullptr;      // [n_rows][n_ticks]
    float2* shat = nullptr;     // time-axis spectra, blocked [n_imp][nkb][n_wires][4]
    float2* mt = nullptr;       // wire-summed spectra, blocked [nkb][n_wires][4]
    float2* g2d = nullptr;      // adjoint: 2D spectrum of G, blocked [nkb][n_fw][4]
    float* noise_amp = nullptr; // Eq. 1's noise: A(k) / n_ft, k < nh (null: no noise)
    uint64_t noise_seed = 0;
    float adc_gain = 0.0f, adc_pedestal = 0.0f;   // digitizer (adc_max 0: none set)
    int32_t adc_max = 0;
    int* flags = nullptr;       // device flag word
    int* queue = nullptr;       // work-queue counter of batched rasterizations
    // scratch of batched runs: bcap events' grids, time-axis and wire-summed spectra
    float* bgrid = nullptr;
    float2* bshat = nullptr;
    float2* bmt = nullptr;
    int32_t bcap = 0;
    int32_t bclean = 0;         // leading batch grid slots known to be all zero
    int device = 0;
    bool grid_clean = false;    // the plane's grid is all zero (consume-and-clear state)
    // wcsim_plane_set_reuse_forward: shat holds the mean-path spectra of the last run on
    // (fwd_depos, fwd_prm) while fwd_valid
    bool reuse_fwd = false;
    bool fwd_valid = false;
    // mode 2 (one-warp wire pass only): the forward's wire pass also writes the 2D spectra of
    // S to s2d (time-frequency major [n_imp][4 nkb][n_fw]); keep_s2d is set for the duration of such a
    // forward, s2d_valid says the last one wrote them (read together with fwd_valid)
    float2* s2d = nullptr;
    bool keep_s2d = false;
    bool s2d_valid = false;
    wcsim_depos fwd_depos = {};
    wcsim_drift_params fwd_prm = {};
    bool wire_block = false;    // autotuned: use the block-level wire pass even if the warp one fits
    bool adj_block = false;     // use the block-level wire adjoint even if the warp one fits
    int32_t kd = 32;            // rasterization tile: depos per CTA and lanes per depo (the
    int32_t kg = 8;             // autotuner may change them)
    // forward with rasterization fused into the time-axis transform: depo binning scratch,
    // and the impact positions per wire-pass launch (the time-axis spectra of that many
    // impact positions are alive at a time)
    bool fused = false;
    bool fused_fits = false;    // the fused transform fits shared memory for the time plan
    FusedScratch fs;
    bool timing = false;
    // forward stage timeline: events, and spans (kind, begin event, end event) between them
    cudaEvent_t ev[kMarks] = {};
    int32_t tl_n = 0;           // events recorded
    int32_t tl_last = -1;       // last event of the sequential marks on the caller's stream
    int32_t sp_kind[kMarks] = {}, sp_b[kMarks] = {}, sp_e[kMarks] = {};
    int32_t sp_n = 0;
    cudaEvent_t evb[kBwdStages + 1] = {};
    bool ev_valid = false;
    bool bwd_recorded = false;
};

namespace {

wcsim_status check_geometry(const wcsim_geometry* g)
{
    if (!g) return fail(WCSIM_EINVAL, "geometry is NULL");
    if (g->n_wires < 1 || g->n_imp < 1 || g->n_ticks < 1)
        return fail(WCSIM_ESHAPE, "n_wires, n_imp, n_ticks must be >= 1 (got %d, %d, %d)",
                    g->n_wires, g->n_imp, g->n_ticks);
    if (g->reserved != 0) return fail(WCSIM_EINVAL, "geometry.reserved must be 0");
    if (!finite_pos(g->pitch_mm) || !finite_pos(g->tick_us))
        return fail(WCSIM_EINVAL, "pitch_mm and tick_us must be finite and > 0");
    if (!isfinite(g->p0_mm) || !isfinite(g->t0_us))
        return fail(WCSIM_EINVAL, "p0_mm and t0_us must be finite");
    if ((int64_t)g->n_wires * g->n_imp > (int64_t)1 << 30)
        return fail(WCSIM_ESHAPE, "n_wires * n_imp too large");
    return WCSIM_OK;
}

wcsim_status check_params(const wcsim_drift_params* p)
{
    if (!p) return fail(WCSIM_EINVAL, "params is NULL");
    if (!finite_pos(p->v_mm_per_us)) return fail(WCSIM_EINVAL, "v_mm_per_us must be finite and > 0");
    if (!(isfinite(p->DL_cm2_s) && p->DL_cm2_s >= 0.0) ||
        !(isfinite(p->DT_cm2_s) && p->DT_cm2_s >= 0.0))
        return fail(WCSIM_EINVAL, "DL_cm2_s and DT_cm2_s must be finite and >= 0");
    if (!(p->lifetime_us > 0.0)) return fail(WCSIM_EINVAL, "lifetime_us must be > 0");
    if (!finite_pos(p->nsigma)) return fail(WCSIM_EINVAL, "nsigma must be finite and > 0");
    if (p->fluctuate < 0 || p->fluctuate > 2)
        return fail(WCSIM_EINVAL, "fluctuate must be 0, 1 or 2");
    if (p->renormalize != 0 && p->renormalize != 1)
        return fail(WCSIM_EINVAL, "renormalize must be 0 or 1");
    if (p->reserved != 0) return fail(WCSIM_EINVAL, "reserved must be 0");
    return WCSIM_OK;
}

wcsim_status check_depos(const wcsim_depos* d)
{
    if (!d) return fail(WCSIM_EINVAL, "depos is NULL");
    if (d->n < 0) return fail(WCSIM_ESHAPE, "depos.n must be >= 0");
    if (d->n > ((int64_t)1 << 32)) return fail(WCSIM_ESHAPE, "depos.n too large (max 2^32)");
    if (d->n > 0 && (!d->p_mm || !d->t_us || !d->tdrift_us || !d->q || !d->id))
        return fail(WCSIM_EINVAL, "depo array pointer is NULL");
    return WCSIM_OK;
}

// The per-call constants of the bin decision, in the same operation order the oracle
// documents: d = pitch / n_imp, 1/d, 1/tick in FP64; 2 D [mm^2/us] = 2 (D 1e-4) rounded to
// FP32; 1/v, n_sigma, 1/bin rounded to FP32.
RasterConsts make_consts(const wcsim_plane* pl)
{
    RasterConsts c;
    const wcsim_geometry& g = pl->g;
    const wcsim_drift_params& p = pl->prm;
    const double dp = g.pitch_mm / (double)g.n_imp;
    c.p0 = g.p0_mm;
    c.t0 = g.t0_us;
    c.inv_dp = 1.0 / dp;
    c.inv_dt = 1.0 / g.tick_us;
    c.two_dt = (float)(2.0 * (p.DT_cm2_s * 1e-4));
    c.two_dl = (float)(2.0 * (p.DL_cm2_s * 1e-4));
    c.inv_v = (float)(1.0 / p.v_mm_per_us);
    c.nsig = (float)p.nsigma;
    c.inv_dp_f = (float)c.inv_dp;
    c.inv_dt_f = (float)c.inv_dt;
    c.dp_f = (float)dp;
    c.dt_f = (float)g.tick_us;
    c.inv_tau = (float)(1.0 / p.lifetime_us);
    c.n_rows = (int64_t)g.n_wires * g.n_imp;
    c.n_ticks = g.n_ticks;
    c.fluctuate = p.fluctuate;
    c.renorm = p.renormalize;
    c.key0 = (uint32_t)p.seed;
    c.key1 = (uint32_t)(p.seed >> 32);
    c.plane_id = p.plane_id;
    c.depos_per_block = pl->kd;
    c.lanes_per_depo = pl->kg;
    c.DL = p.DL_cm2_s;
    c.DT = p.DT_cm2_s;
    c.v = p.v_mm_per_us;
    c.tau = p.lifetime_us;
    // Stirling's remainder for the exact binomial's small counts, from log-gamma in FP64
    c.stirl[0] = 0.0f;
    for (int m = 1; m < 16; ++m)
        c.stirl[m] = (float)(std::lgamma(m + 1.0) -
                             ((m + 0.5) * std::log((double)m) - m + 0.5 * std::log(6.283185307179586477)));
    return c;
}

DepoArrays depo_arrays(const wcsim_depos* d)
{
    DepoArrays a;
    a.p = d->p_mm;
    a.t = d->t_us;
    a.td = d->tdrift_us;
    a.q = d->q;
    a.id = d->id;
    a.n = d->n;
    return a;
}

void plane_free(wcsim_plane* pl)
{
    if (!pl) return;
    cudaFree(pl->tw_t);
    cudaFree(pl->tw_w);
    cudaFree(pl->tw_warp);
    cudaFree(pl->H);
    cudaFree(pl->grid);
    cudaFree(pl->shat);
    cudaFree(pl->mt);
    cudaFree(pl->g2d);
    cudaFree(pl->s2d);
    cudaFree(pl->noise_amp);
    cudaFree(pl->flags);
    cudaFree(pl->queue);
    cudaFree(pl->bgrid);
    cudaFree(pl->bshat);
    cudaFree(pl->bmt);
    cudaFree(pl->fs.dec);
    cudaFree(pl->fs.pos);
    cudaFree(pl->fs.cnt);
    cudaFree(pl->fs.off);
    cudaFree(pl->fs.sorted);
    cudaFree(pl->fs.wts);
    if (pl->ev_valid) {
        for (auto& e : pl->ev) cudaEventDestroy(e);
        for (auto& e : pl->evb) cudaEventDestroy(e);
    }
    delete pl;
}

// Forward timeline.  tl_record records an event on s (index, or -1 when timing is off or
// the events are used up); tl_span adds a span of stage kind k between two events.
// Stage kinds: 0 prep, 1 rasterize, 2 rows_r2c, 3 wire_pass, 4 rows_c2r; spans of one kind
// are summed by wcsim_plane_stage_times.
inline int tl_record(wcsim_plane* pl, cudaStream_t s)
{
    if (!pl->timing || pl->tl_n >= kMarks) return -1;
    cudaEventRecord(pl->ev[pl->tl_n], s);
    return pl->tl_n++;
}

inline void tl_span(wcsim_plane* pl, int kind, int b, int e)
{
    if (b < 0 || e < 0 || pl->sp_n >= kMarks) return;
    pl->sp_kind[pl->sp_n] = kind;
    pl->sp_b[pl->sp_n] = b;
    pl->sp_e[pl->sp_n] = e;
    ++pl->sp_n;
}

// Sequential marks on one stream: mark(pl, 0) starts a forward's timeline, mark(pl, i > 0)
// closes a span of stage kind i - 1 since the previous mark.
inline void mark(wcsim_plane* pl, int i, cudaStream_t s)
{
    if (!pl->timing) return;
    if (i == 0) {
        pl->tl_n = 0;
        pl->sp_n = 0;
        pl->tl_last = tl_record(pl, s);
        return;
    }
    const int e = tl_record(pl, s);
    tl_span(pl, i - 1, pl->tl_last, e);
    pl->tl_last = e;
}

inline void markb(wcsim_plane* pl, int i, cudaStream_t s)
{
    if (pl->timing) {
        cudaEventRecord(pl->evb[i], s);
        pl->bwd_recorded = true;
    }
}

// Eq. 2 after the rasterization: the time-axis transform of every grid row (r2c(s)), the
// wire pass and the inverse time FFT, one launch each on s, with timeline spans around them.
template <class R2C>
wcsim_status convolve_stages(wcsim_plane* pl, R2C r2c, float* wave, cudaStream_t s)
{
    const ConvDims& d = pl->dims;
    cudaError_t e;
    int b = tl_record(pl, s);
    if ((e = r2c(s))) return cuda_fail(e, "rows_r2c launch");
    int t = tl_record(pl, s);
    tl_span(pl, 2, b, t);
    if (pl->tw_warp && !pl->wire_block)
        e = launch_wire_warp(d, pl->tw_warp, pl->shat, pl->H, pl->mt, pl->flags, s, 1,
                             pl->keep_s2d ? pl->s2d : nullptr);
    else
        e = launch_wire_pass(d, pl->pw, pl->shat, pl->H, pl->mt, pl->flags, s);
    if (e) return cuda_fail(e, "wire_pass launch");
    b = t;
    t = tl_record(pl, s);
    tl_span(pl, 3, b, t);
    if ((e = launch_rows_c2r(d, pl->pt, pl->mt, wave, s))) return cuda_fail(e, "rows_c2r launch");
    tl_span(pl, 4, t, tl_record(pl, s));
    return WCSIM_OK;
}

// A forward that will keep the 2D spectra of S for the backward (set_reuse_forward mode 2):
// mean path, one-warp wire pass, buffer allocated.
bool keeps_s2d(const wcsim_plane* pl)
{
    return pl->s2d && pl->reuse_fwd && pl->prm.fluctuate == 0 && pl->tw_warp && !pl->wire_block;
}

wcsim_status do_convolve(wcsim_plane* pl, const float* grid, float* wave, cudaStream_t s)
{
    pl->fwd_valid = false;              // the spectra are about to be those of `grid`
    const ConvDims d = pl->dims;
    const FftPlan pt = pl->pt;
    int* flags = pl->flags;
    float2* shat = pl->shat;
    auto r2c = [&](cudaStream_t strm) {
        return launch_rows_r2c(d, pt, grid, shat, flags, strm);
    };
    return convolve_stages(pl, r2c, wave, s);
}

// Binning scratch for n depos (grown, never shrunk; allocates only when n exceeds it).
wcsim_status fused_reserve(wcsim_plane* pl, int64_t n)
{
    FusedScratch& f = pl->fs;
    if (n <= f.cap) return WCSIM_OK;
    cudaFree(f.dec);
    cudaFree(f.pos);
    cudaFree(f.sorted);
    cudaFree(f.wts);
    f.dec = f.sorted = nullptr;
    f.pos = nullptr;
    f.wts = nullptr;
    f.cap = 0;
    const int64_t cap = (n + 4095) & ~(int64_t)4095;
    cudaError_t e = cudaMalloc(&f.dec, (size_t)cap * kDecisionBytes);
    if (!e) e = cudaMalloc(&f.sorted, (size_t)cap * kDecisionBytes);
    if (!e) e = cudaMalloc(&f.pos, (size_t)cap * sizeof(int32_t));
    if (!e) e = cudaMalloc(&f.wts, (size_t)cap * kFusedSlots * sizeof(float));
    if (e) return cuda_fail(e, "depo binning scratch allocation");
    f.cap = cap;
    return WCSIM_OK;
}

// The fused forward applies: not the exact binomial (its draws stay in the plain
// rasterizer), depo counts that fit the binning's 32-bit slots.
bool fused_applies(const wcsim_plane* pl, const wcsim_depos* depos)
{
    return pl->fused && pl->fused_fits && pl->prm.fluctuate != 2 &&
           depos->n < ((int64_t)1 << 31);
}

// wcsim_run's forward with the rasterization inside the time-axis transform (the grid is
// never written): depo binning, then convolve_stages with the fused transform.
wcsim_status fused_forward(wcsim_plane* pl, const wcsim_depos* depos, void* out, cudaStream_t s)
{
    wcsim_status st = fused_reserve(pl, depos->n);
    if (st) return st;
    const ConvDims& d = pl->dims;
    RasterConsts c = make_consts(pl);
    cudaError_t e = launch_bin_depos(c, depo_arrays(depos), d.n_imp, d.n_w, pl->fs, pl->flags, s);
    if (e) return cuda_fail(e, "depo binning launch");
    mark(pl, 1, s);
    const FftPlan pt = pl->pt;
    const FusedScratch fs = pl->fs;
    float2* shat = pl->shat;
    auto r2c = [&](cudaStream_t strm) {
        return launch_rows_r2c_fused(d, pt, c, fs, shat, strm);
    };
    pl->keep_s2d = keeps_s2d(pl);
    st = convolve_stages(pl, r2c, static_cast<float*>(out), s);
    const bool kept = pl->keep_s2d;
    pl->keep_s2d = false;
    if (st) return st;
    pl->fwd_valid = false;
    if (pl->reuse_fwd && pl->prm.fluctuate == 0) {
        pl->fwd_valid = true;           // shat: the mean-path spectra of these depos
        pl->s2d_valid = kept;
        pl->fwd_depos = *depos;
        pl->fwd_prm = pl->prm;
    }
    return WCSIM_OK;
}

}  // namespace

namespace {

size_t ev_grid_elems(const ConvDims& d) { return (size_t)d.n_w * d.n_imp * d.n_t; }
size_t ev_shat_elems(const ConvDims& d) { return (size_t)d.n_w * d.n_imp * d.nkb * kBlockCols; }
size_t ev_mt_elems(const ConvDims& d) { return (size_t)d.n_w * d.nkb * kBlockCols; }

wcsim_status reserve_batch(wcsim_plane* pl, int32_t n)
{
    if (n <= pl->bcap) return WCSIM_OK;
    cudaFree(pl->bgrid);
    cudaFree(pl->bshat);
    cudaFree(pl->bmt);
    pl->bgrid = nullptr;
    pl->bshat = nullptr;
    pl->bmt = nullptr;
    pl->bcap = 0;
    const ConvDims& d = pl->dims;
    cudaError_t e = cudaMalloc(&pl->bgrid, (size_t)n * ev_grid_elems(d) * sizeof(float));
    if (!e) e = cudaMalloc(&pl->bshat, (size_t)n * ev_shat_elems(d) * sizeof(float2));
    if (!e) e = cudaMalloc(&pl->bmt, (size_t)n * ev_mt_elems(d) * sizeof(float2));
    if (e) return cuda_fail(e, "batch scratch allocation");
    pl->bcap = n;
    pl->bclean = 0;
    return WCSIM_OK;
}

// Events ev[0..k) of one plane (global batch indices idx[] for the seeds), k <= kMaxBatch.
// The inverse time FFT of a run adds the plane's noise, when it has one (Eq. 1).
void with_noise(const wcsim_plane* pl, ConvDims& d)
{
    d.noise_amp = pl->noise_amp;
    d.noise_seed = pl->noise_seed;
    d.plane_id = pl->prm.plane_id;
}

// Batch scratch of plane pl for its k events (global batch indices idx[]), with their grid
// slots reset where they are not known to be clean.  On success the grids are ready for
// rasterization and pl->bclean holds the slots that will be clean after the run.
wcsim_status prepare_group(wcsim_plane* pl, int k, int32_t* clean_after, cudaStream_t s)
{
    wcsim_status st = reserve_batch(pl, k);
    if (st) return st;
    const ConvDims& d0 = pl->dims;
    // the time-axis transform clears each grid as it reads it (consume and clear), so a grid
    // slot needs a reset only before its first use after an allocation or a failed run
    if (pl->bclean < k) {
        cudaError_t e = cudaMemsetAsync(pl->bgrid, 0, (size_t)k * ev_grid_elems(d0) * sizeof(float), s);
        if (e) return cuda_fail(e, "batch grid reset");
    }
    *clean_after = pl->bclean > k ? pl->bclean : k;
    pl->bclean = 0;                     // until the run has been enqueued in full
    return WCSIM_OK;
}

// The per-plane rasterization of events idx[0..k) (when the batch's queue launch does not
// apply) into their grid slots.
wcsim_status rasterize_group(wcsim_plane* pl, int k, const int32_t* idx, const wcsim_depos* depos,
                             cudaStream_t s)
{
    const ConvDims& d0 = pl->dims;
    RasterConsts c = make_consts(pl);
    BatchEvents ev;
    ev.n = k;
    ev.block_start[0] = 0;
    for (int i = 0; i < k; ++i) {
        const wcsim_depos* dp = &depos[idx[i]];
        ev.d[i] = depo_arrays(dp);
        ev.grid[i] = pl->bgrid + (size_t)i * ev_grid_elems(d0);
        const uint64_t seed = pl->prm.seed + (uint64_t)idx[i];     // per-event stream
        ev.key0[i] = (uint32_t)seed;
        ev.key1[i] = (uint32_t)(seed >> 32);
        ev.block_start[i + 1] = ev.block_start[i] + rasterize_blocks(dp->n, c.depos_per_block);
    }
    cudaError_t e = launch_rasterize_batch(c, ev, pl->flags, s);
    return e ? cuda_fail(e, "batch rasterize launch") : WCSIM_OK;
}

// Eq. 2 for the k events of plane pl whose grids are rasterized: one launch per stage over
// the k events.
wcsim_status convolve_group(wcsim_plane* pl, int k, const int32_t* idx, float* const* waves,
                            int32_t clean_after, cudaStream_t s)
{
    const ConvDims& d0 = pl->dims;
    ConvDims d = d0;
    d.ev_grid = (int64_t)ev_grid_elems(d0);
    d.ev_shat = (int64_t)ev_shat_elems(d0);
    d.ev_mt = (int64_t)ev_mt_elems(d0);
    d.clear_input = 1;
    cudaError_t e;
    if ((e = launch_rows_r2c_batch(d, pl->pt, pl->bgrid, pl->bshat, k, s)))
        return cuda_fail(e, "batch rows_r2c launch");
    d.clear_input = 0;
    if (pl->tw_warp && !pl->wire_block) {
        if ((e = launch_wire_warp(d, pl->tw_warp, pl->bshat, pl->H, pl->bmt, pl->flags, s, k)))
            return cuda_fail(e, "batch wire launch");
    } else {
        for (int i = 0; i < k; ++i)
            if ((e = launch_wire_pass(d0, pl->pw, pl->bshat + i * d.ev_shat, pl->H, pl->bmt + i * d.ev_mt,
                                      pl->flags, s)))
                return cuda_fail(e, "batch wire launch");
    }
    WavePtrs w;
    for (int i = 0; i < k; ++i) {
        w.p[i] = waves[idx[i]];
        w.ev[i] = idx[i];
    }
    with_noise(pl, d);
    if ((e = launch_rows_c2r_batch(d, pl->pt, pl->bmt, w, k, s))) return cuda_fail(e, "batch rows_c2r launch");
    pl->bclean = clean_after;
    return WCSIM_OK;
}

}  // namespace

wcsim_status wcsim::report_error(wcsim_status s, const char* msg) { return fail(s, "%s", msg); }

extern "C" {

const char* wcsim_last_error(void) { return g_err; }

const char* wcsim_version(void) { return "wcsim 0.1 (sm_103a)"; }

wcsim_status wcsim_plane_create(const wcsim_geometry* geom, const void* resp_c64, int32_t n_fw,
                                int32_t n_ft, const wcsim_drift_params* params, void* stream,
                                wcsim_plane** out)
{
    if (!out) return fail(WCSIM_EINVAL, "out is NULL");
    *out = nullptr;
    wcsim_status st;
    if ((st = check_geometry(geom))) return st;
    if ((st = check_params(params))) return st;
    if (!resp_c64) return fail(WCSIM_EINVAL, "response pointer is NULL");
    if (n_fw == 0) n_fw = geom->n_wires;
    if (n_ft == 0) n_ft = geom->n_ticks;
    if (n_fw < geom->n_wires || n_ft < geom->n_ticks)
        return fail(WCSIM_ESHAPE, "spectrum (%d x %d) smaller than the frame (%d x %d)", n_fw,
                    n_ft, geom->n_wires, geom->n_ticks);
    if (n_ft > kMaxFftN || n_fw > kMaxWireN)
        return fail(WCSIM_ESHAPE, "FFT size %d x %d above the supported %d x %d", n_fw, n_ft,
                    kMaxWireN, kMaxFftN);
    int32_t rad[kMaxPasses], np;
    if (!fft_factor(n_fw, rad, &np) || !fft_factor(n_ft, rad, &np))
        return fail(WCSIM_ESHAPE, "FFT sizes must factor into 2, 3, 5, 7 (got %d x %d)", n_fw, n_ft);

    wcsim_plane* pl = new (std::nothrow) wcsim_plane();
    if (!pl) return fail(WCSIM_ENOMEM, "host allocation failed");
    pl->g = *geom;
    pl->prm = *params;
    cudaError_t e = cudaGetDevice(&pl->device);
    if (e) { plane_free(pl); return cuda_fail(e, "cudaGetDevice"); }
    ConvDims& d = pl->dims;
    d.n_w = geom->n_wires;
    d.n_imp = geom->n_imp;
    d.n_t = geom->n_ticks;
    d.n_fw = n_fw;
    d.n_ft = n_ft;
    d.nh = n_ft / 2 + 1;
    d.nkb = (d.nh + kBlockCols - 1) / kBlockCols;
    // Kernel variant of the time-axis forward FFT; WCSIM_ROWS_KERNEL=staged|direct overrides.
    d.rows_variant = 0;
    if (const char* v = getenv("WCSIM_ROWS_KERNEL")) d.rows_variant = (strcmp(v, "staged") == 0) ? 1 : 0;
    // The time-axis kernels move blocked half spectra by TMA box copies; WCSIM_SPECTRA_TMA=0
    // selects per-thread loads and stores.
    if (const char* v = getenv("WCSIM_SPECTRA_TMA")) d.spectra_tma = strcmp(v, "0") != 0;
    // Impact groups of the one-warp wire adjoint (CTAs per frequency block); WCSIM_ADJ_SPLIT.
    if (const char* v = getenv("WCSIM_ADJ_SPLIT")) d.adj_split = atoi(v);
    cudaStream_t s = (cudaStream_t)stream;
    const size_t n_rows = (size_t)d.n_w * d.n_imp;
#define WC_TRY(call, what)                                  \
    do {                                                    \
        cudaError_t _e = (call);                            \
        if (_e != cudaSuccess) {                            \
            plane_free(pl);                                 \
            return cuda_fail(_e, what);                     \
        }                                                   \
    } while (0)
    WC_TRY(fft_plan_create(n_ft, &pl->pt, &pl->tw_t), "time-axis FFT plan");
    WC_TRY(fft_plan_create(n_fw, &pl->pw, &pl->tw_w), "wire-axis FFT plan");
    // Wire-axis kernel; WCSIM_WIRE_KERNEL=block forces the block-level engine.
    {
        const char* v = getenv("WCSIM_WIRE_KERNEL");
        const bool block = v && strcmp(v, "block") == 0;
        if (!block && wire_warp_supported(n_fw) && geom->n_wires <= n_fw) {
            WC_TRY(wire_warp_twiddles(n_fw, &pl->tw_warp), "wire-axis twiddles");
            const size_t g2d = (size_t)((n_ft / 2 + 1 + kBlockCols - 1) / kBlockCols) * kBlockCols * n_fw;
            WC_TRY(cudaMalloc(&pl->g2d, g2d * sizeof(float2)), "adjoint scratch allocation");
        }
    }
    const size_t cols = (size_t)d.nkb * kBlockCols;
    WC_TRY(cudaMalloc(&pl->H, (size_t)d.n_imp * d.n_fw * cols * sizeof(float2)), "response allocation");
    WC_TRY(cudaMalloc(&pl->grid, n_rows * d.n_t * sizeof(float)), "grid allocation");
    WC_TRY(cudaMalloc(&pl->shat, n_rows * cols * sizeof(float2)), "spectrum allocation");
    WC_TRY(cudaMalloc(&pl->mt, (size_t)d.n_w * cols * sizeof(float2)), "spectrum allocation");
    WC_TRY(cudaMalloc(&pl->flags, sizeof(int)), "flag allocation");
    WC_TRY(cudaMalloc(&pl->queue, sizeof(int)), "queue counter allocation");
    WC_TRY(cudaMalloc(&pl->fs.cnt, (size_t)(d.n_w + 1) * sizeof(int32_t)), "bin count allocation");
    WC_TRY(cudaMalloc(&pl->fs.off, (size_t)(d.n_w + 2) * sizeof(int32_t)), "bin offset allocation");
    WC_TRY(cudaMemsetAsync(pl->fs.cnt, 0, (size_t)(d.n_w + 1) * sizeof(int32_t), s), "bin count reset");
    pl->fused_fits = fused_supported(pl->pt);
    // forward variant; WCSIM_FORWARD=fused|plain overrides the default (plain)
    if (const char* v = getenv("WCSIM_FORWARD")) pl->fused = strcmp(v, "fused") == 0;
    // wire adjoint; WCSIM_ADJOINT_KERNEL=block forces the block-level engine
    if (const char* v = getenv("WCSIM_ADJOINT_KERNEL")) pl->adj_block = strcmp(v, "block") == 0;
    WC_TRY(cudaMemsetAsync(pl->flags, 0, sizeof(int), s), "flag reset");
    WC_TRY(launch_make_hermitian(d, (const float2*)resp_c64, pl->H,
                                 (float)(1.0 / ((double)n_fw * (double)n_ft)), s),
           "response preparation");
    WC_TRY(cudaStreamSynchronize(s), "response preparation");
    for (auto& ev : pl->ev) WC_TRY(cudaEventCreate(&ev), "event creation");
    for (auto& ev : pl->evb) WC_TRY(cudaEventCreate(&ev), "event creation");
    pl->ev_valid = true;
#undef WC_TRY
    *out = pl;
    return WCSIM_OK;
}

wcsim_status wcsim_plane_set_params(wcsim_plane* pl, const wcsim_drift_params* params)
{
    if (!pl) return fail(WCSIM_EINVAL, "plane is NULL");
    wcsim_status st = check_params(params);
    if (st) return st;
    pl->prm = *params;
    return WCSIM_OK;
}

wcsim_status wcsim_plane_set_response(wcsim_plane* pl, const void* resp_c64, void* stream)
{
    if (!pl) return fail(WCSIM_EINVAL, "plane is NULL");
    if (!resp_c64) return fail(WCSIM_EINVAL, "response pointer is NULL");
    DeviceGuard dg(pl->device);
    if (!dg.ok) return fail(WCSIM_ECUDA, "cannot select the plane's device");
    const ConvDims& d = pl->dims;
    cudaError_t e = launch_make_hermitian(d, (const float2*)resp_c64, pl->H,
                                          (float)(1.0 / ((double)d.n_fw * (double)d.n_ft)),
                                          (cudaStream_t)stream);
    return e ? cuda_fail(e, "response preparation") : WCSIM_OK;
}

wcsim_status wcsim_rasterize(wcsim_plane* pl, const wcsim_depos* depos, float* grid, void* stream)
{
    if (!pl) return fail(WCSIM_EINVAL, "plane is NULL");
    wcsim_status st = check_depos(depos);
    if (st) return st;
    if (!grid) return fail(WCSIM_EINVAL, "grid is NULL");
    DeviceGuard dg(pl->device);
    if (!dg.ok) return fail(WCSIM_ECUDA, "cannot select the plane's device");
    cudaStream_t s = (cudaStream_t)stream;
    mark(pl, 0, s);
    pl->fwd_valid = false;
    cudaError_t e = launch_rasterize(make_consts(pl), depo_arrays(depos), grid, pl->flags, s);
    if (e) return cuda_fail(e, "rasterize launch");
    mark(pl, 2, s);
    return WCSIM_OK;
}

wcsim_status wcsim_convolve(wcsim_plane* pl, const float* grid, float* wave, void* stream)
{
    if (!pl) return fail(WCSIM_EINVAL, "plane is NULL");
    if (!grid || !wave) return fail(WCSIM_EINVAL, "grid or wave is NULL");
    DeviceGuard dg(pl->device);
    if (!dg.ok) return fail(WCSIM_ECUDA, "cannot select the plane's device");
    cudaStream_t s = (cudaStream_t)stream;
    mark(pl, 0, s);
    return do_convolve(pl, grid, wave, s);
}

// wcsim_run and wcsim_run_adc: rasterize into the plane's grid, then convolve (with the
// plane's noise); adc: the inverse time FFT writes the plane's ADC codes to out.
// target (not with adc): out receives M - target, and loss (if not null) 1/2 sum of squares.
static wcsim_status run_frame(wcsim_plane* pl, const wcsim_depos* depos, void* out, bool adc,
                              void* stream, const float* target = nullptr,
                              double* loss = nullptr)
{
    if (!pl) return fail(WCSIM_EINVAL, "plane is NULL");
    wcsim_status st = check_depos(depos);
    if (st) return st;
    if (!out) return fail(WCSIM_EINVAL, "output is NULL");
    if (adc && pl->adc_max <= 0) return fail(WCSIM_EINVAL, "no digitizer set (wcsim_plane_set_digitizer)");
    DeviceGuard dg(pl->device);
    if (!dg.ok) return fail(WCSIM_ECUDA, "cannot select the plane's device");
    cudaStream_t s = (cudaStream_t)stream;
    const ConvDims& d = pl->dims;
    cudaError_t e = cudaSuccess;
    if (loss && (e = cudaMemsetAsync(loss, 0, sizeof(double), s))) return cuda_fail(e, "loss reset");
    mark(pl, 0, s);
    pl->dims.target = target;
    pl->dims.loss = target ? loss : nullptr;
    if (fused_applies(pl, depos)) {
        with_noise(pl, pl->dims);
        if (adc) {
            pl->dims.adc_gain = pl->adc_gain;
            pl->dims.adc_pedestal = pl->adc_pedestal;
            pl->dims.adc_max = pl->adc_max;
        }
        st = fused_forward(pl, depos, out, s);
        pl->dims.noise_amp = nullptr;
        pl->dims.adc_max = 0;
        pl->dims.target = nullptr;
        pl->dims.loss = nullptr;
        return st;
    }
    if (!pl->grid_clean) {
        e = cudaMemsetAsync(pl->grid, 0, (size_t)d.n_w * d.n_imp * d.n_t * sizeof(float), s);
        if (e) {
            pl->dims.target = nullptr;
            pl->dims.loss = nullptr;
            return cuda_fail(e, "grid reset");
        }
    }
    pl->grid_clean = false;
    mark(pl, 1, s);
    e = launch_rasterize(make_consts(pl), depo_arrays(depos), pl->grid, pl->flags, s);
    if (e) {
        pl->dims.target = nullptr;
        pl->dims.loss = nullptr;
        return cuda_fail(e, "rasterize launch");
    }
    mark(pl, 2, s);
    // the time-axis transform reads the plane's own grid once: it clears it as it goes
    // (the direct kernel; the staged one reads through bulk copies and leaves it as is)
    pl->dims.clear_input = (pl->dims.rows_variant == 0);
    with_noise(pl, pl->dims);
    if (adc) {
        pl->dims.adc_gain = pl->adc_gain;
        pl->dims.adc_pedestal = pl->adc_pedestal;
        pl->dims.adc_max = pl->adc_max;
    }
    pl->keep_s2d = keeps_s2d(pl);
    st = do_convolve(pl, pl->grid, static_cast<float*>(out), s);
    const bool kept = pl->keep_s2d;
    pl->keep_s2d = false;
    pl->dims.clear_input = 0;
    pl->dims.noise_amp = nullptr;
    pl->dims.adc_max = 0;
    pl->dims.target = nullptr;
    pl->dims.loss = nullptr;
    if (st == WCSIM_OK && pl->dims.rows_variant == 0) pl->grid_clean = true;
    if (st == WCSIM_OK && pl->reuse_fwd && pl->prm.fluctuate == 0) {
        pl->fwd_valid = true;           // shat: the mean-path spectra of these depos
        pl->s2d_valid = kept;
        pl->fwd_depos = *depos;
        pl->fwd_prm = pl->prm;
    }
    return st;
}

wcsim_status wcsim_run(wcsim_plane* pl, const wcsim_depos* depos, float* wave, void* stream)
{
    return run_frame(pl, depos, wave, false, stream);
}

wcsim_status wcsim_run_adc(wcsim_plane* pl, const wcsim_depos* depos, uint16_t* adc, void* stream)
{
    return run_frame(pl, depos, adc, true, stream);
}

wcsim_status wcsim_run_residual(wcsim_plane* pl, const wcsim_depos* depos, const float* target,
                                float* residual, double* loss, void* stream)
{
    if (!target) return fail(WCSIM_EINVAL, "target is NULL");
    return run_frame(pl, depos, residual, false, stream, target, loss);
}

wcsim_status wcsim_plane_set_digitizer(wcsim_plane* pl, float gain, float pedestal, int32_t bits)
{
    if (!pl) return fail(WCSIM_EINVAL, "plane is NULL");
    if (bits < 1 || bits > 16) return fail(WCSIM_EINVAL, "ADC bits must be in 1..16 (got %d)", bits);
    if (!isfinite(gain) || !isfinite(pedestal))
        return fail(WCSIM_EINVAL, "ADC gain and pedestal must be finite");
    pl->adc_gain = gain;
    pl->adc_pedestal = pedestal;
    pl->adc_max = (1 << bits) - 1;
    return WCSIM_OK;
}

// have_shat: the plane's spectra already hold the time-axis FFT of `grid` (a forward on the
// same grid just computed them), so that transform is skipped
// have_s2d: the forward also kept the 2D spectra of S (reuse mode 2): dL/dR streams from them
// (part A only transforms G) and the spectra of the grid are not needed at all
static wcsim_status convolve_adjoint(wcsim_plane* pl, const float* grad_wave, const float* grid,
                                     float* dgrid, void* grad_resp_c64, void* stream,
                                     bool have_shat, bool have_s2d = false)
{
    if (!pl) return fail(WCSIM_EINVAL, "plane is NULL");
    if (!grad_wave || !grid || !dgrid) return fail(WCSIM_EINVAL, "grad_wave, grid or dgrid is NULL");
    DeviceGuard dg(pl->device);
    if (!dg.ok) return fail(WCSIM_ECUDA, "cannot select the plane's device");
    cudaStream_t s = (cudaStream_t)stream;
    const ConvDims& d = pl->dims;
    ConvDims dG = d;                    // G's rows: one "impact position" per wire
    dG.n_imp = 1;
    cudaError_t e;
    pl->fwd_valid = false;              // the adjoint overwrites the spectra
    if (!have_shat && (e = launch_rows_r2c(d, pl->pt, grid, pl->shat, pl->flags, s)))
        return cuda_fail(e, "rows_r2c launch");
    markb(pl, 3, s);
    if ((e = launch_rows_r2c(dG, pl->pt, grad_wave, pl->mt, pl->flags, s))) return cuda_fail(e, "rows_r2c launch");
    markb(pl, 4, s);
    const float inv_n = (float)(1.0 / ((double)d.n_fw * (double)d.n_ft));
    const bool warp = pl->tw_warp && !pl->adj_block;
    if (warp && have_s2d && grad_resp_c64) {
        if (!(e = launch_wire_adjoint_warp(d, pl->tw_warp, pl->mt, pl->shat, pl->H, pl->g2d,
                                           nullptr, inv_n, s)))
            e = launch_dr_rows(d, pl->s2d, pl->g2d, (float2*)grad_resp_c64, inv_n, s);
    } else if (warp)
        e = launch_wire_adjoint_warp(d, pl->tw_warp, pl->mt, pl->shat, pl->H, pl->g2d,
                                     (float2*)grad_resp_c64, inv_n, s);
    else
        e = launch_wire_adjoint_block(d, pl->pw, pl->mt, pl->shat, pl->H, (float2*)grad_resp_c64,
                                      inv_n, s);
    if (e) return cuda_fail(e, "wire adjoint launch");
    markb(pl, 5, s);
    if ((e = launch_rows_c2r_grid(d, pl->pt, pl->shat, dgrid, s))) return cuda_fail(e, "rows_c2r_grid launch");
    markb(pl, 6, s);
    return WCSIM_OK;
}

wcsim_status wcsim_convolve_adjoint(wcsim_plane* pl, const float* grad_wave, const float* grid,
                                    float* dgrid, void* grad_resp_c64, void* stream)
{
    return convolve_adjoint(pl, grad_wave, grid, dgrid, grad_resp_c64, stream, false);
}

wcsim_status wcsim_rasterize_adjoint(wcsim_plane* pl, const wcsim_depos* depos, const float* dgrid,
                                     wcsim_depo_grads* grads, void* stream)
{
    if (!pl) return fail(WCSIM_EINVAL, "plane is NULL");
    wcsim_status st = check_depos(depos);
    if (st) return st;
    if (!dgrid || !grads) return fail(WCSIM_EINVAL, "dgrid or grads is NULL");
    DeviceGuard dg(pl->device);
    if (!dg.ok) return fail(WCSIM_ECUDA, "cannot select the plane's device");
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e;
    pl->fwd_valid = false;
    if (grads->dglobal && (e = cudaMemsetAsync(grads->dglobal, 0, 3 * sizeof(double), s)))
        return cuda_fail(e, "gradient reset");
    DepoGrads g{grads->dq, grads->dp, grads->dt, grads->dsigma_L, grads->dsigma_T, grads->dglobal};
    if ((e = launch_depo_adjoint(make_consts(pl), depo_arrays(depos), dgrid, g, pl->flags, s)))
        return cuda_fail(e, "depo adjoint launch");
    markb(pl, 7, s);
    return WCSIM_OK;
}

wcsim_status wcsim_run_backward(wcsim_plane* pl, const wcsim_depos* depos, const float* grad_wave,
                                wcsim_depo_grads* grads, void* grad_resp_c64, void* stream)
{
    if (!pl) return fail(WCSIM_EINVAL, "plane is NULL");
    wcsim_status st = check_depos(depos);
    if (st) return st;
    if (!grad_wave || !grads) return fail(WCSIM_EINVAL, "grad_wave or grads is NULL");
    DeviceGuard dg(pl->device);
    if (!dg.ok) return fail(WCSIM_ECUDA, "cannot select the plane's device");
    cudaStream_t s = (cudaStream_t)stream;
    const ConvDims& d = pl->dims;
    cudaError_t e = cudaSuccess;
    // the spectra of the mean-path grid are still in place after a forward on the same depos
    // and parameters (wcsim_plane_set_reuse_forward): no need to recompute them
    const bool reuse = pl->reuse_fwd && pl->fwd_valid &&
                       memcmp(&pl->fwd_depos, depos, sizeof(wcsim_depos)) == 0 &&
                       memcmp(&pl->fwd_prm, &pl->prm, sizeof(wcsim_drift_params)) == 0;
    pl->fwd_valid = false;
    markb(pl, 0, s);
    if (!reuse && !pl->grid_clean) {
        e = cudaMemsetAsync(pl->grid, 0, (size_t)d.n_w * d.n_imp * d.n_t * sizeof(float), s);
        if (e) return cuda_fail(e, "grid reset");
    }
    pl->grid_clean = false;             // the grid ends up holding dL/dS
    markb(pl, 1, s);
    if (!reuse) {
        RasterConsts c = make_consts(pl);
        c.fluctuate = 0;                // the gradient is that of the mean waveform
        if ((e = launch_rasterize(c, depo_arrays(depos), pl->grid, pl->flags, s)))
            return cuda_fail(e, "rasterize launch");
    }
    markb(pl, 2, s);
    if ((st = convolve_adjoint(pl, grad_wave, pl->grid, pl->grid, grad_resp_c64, stream, reuse,
                               reuse && pl->s2d_valid)))
        return st;
    return wcsim_rasterize_adjoint(pl, depos, pl->grid, grads, stream);
}

wcsim_status wcsim_plane_reserve_batch(wcsim_plane* pl, int32_t n_events)
{
    if (!pl) return fail(WCSIM_EINVAL, "plane is NULL");
    if (n_events < 0 || n_events > kMaxBatch)
        return fail(WCSIM_ESHAPE, "n_events must be in [0, %d]", kMaxBatch);
    DeviceGuard dg(pl->device);
    if (!dg.ok) return fail(WCSIM_ECUDA, "cannot select the plane's device");
    return reserve_batch(pl, n_events);
}

wcsim_status wcsim_batch_run(int32_t n_events, wcsim_plane* const* planes,
                                        const wcsim_depos* depos, float* const* waves, void* stream)
{
    if (n_events < 0 || n_events > kMaxBatch)
        return fail(WCSIM_ESHAPE, "n_events must be in [0, %d]", kMaxBatch);
    if (n_events == 0) return WCSIM_OK;
    if (!planes || !depos || !waves) return fail(WCSIM_EINVAL, "planes, depos or waves is NULL");
    for (int i = 0; i < n_events; ++i) {
        if (!planes[i] || !waves[i]) return fail(WCSIM_EINVAL, "event %d: plane or wave is NULL", i);
        wcsim_status st = check_depos(&depos[i]);
        if (st) return st;
        if (planes[i]->device != planes[0]->device)
            return fail(WCSIM_EINVAL, "all planes of a batch must live on one device");
    }
    for (int i = 0; i < n_events; ++i) planes[i]->fwd_valid = false;
    DeviceGuard dg(planes[0]->device);
    if (!dg.ok) return fail(WCSIM_ECUDA, "cannot select the plane's device");
    cudaStream_t s = (cudaStream_t)stream;
    // group events by plane, in order of first appearance; slot[e]: event e's grid slot in
    // its plane's batch scratch
    int32_t slot[kMaxBatch], first[kMaxBatch], count[kMaxBatch];
    int32_t members[kMaxBatch][kMaxBatch], clean_after[kMaxBatch];
    int n_groups = 0;
    for (int i = 0; i < n_events; ++i) {
        int g = 0;
        while (g < n_groups && planes[first[g]] != planes[i]) ++g;
        if (g == n_groups) {
            first[g] = i;
            count[g] = 0;
            ++n_groups;
        }
        slot[i] = count[g];
        members[g][count[g]++] = i;
    }
    for (int g = 0; g < n_groups; ++g) {
        wcsim_status st = prepare_group(planes[first[g]], count[g], &clean_after[g], s);
        if (st) return st;
    }
    // one persistent rasterization over every event of the batch (a work queue of (event,
    // depo block) items) when the planes share the rasterization tile and the kind of
    // fluctuation draw; otherwise one launch per plane
    bool queue = true;
    const RasterConsts c0 = make_consts(planes[0]);
    for (int i = 1; i < n_events && queue; ++i) {
        const wcsim_plane* p = planes[i];
        queue = p->kd == planes[0]->kd && p->kg == planes[0]->kg &&
                (p->prm.fluctuate == 2) == (c0.fluctuate == 2);
    }
    if (queue) {
        QueueEvents q;
        q.n = n_events;
        q.block_start[0] = 0;
        for (int i = 0; i < n_events; ++i) {
            wcsim_plane* p = planes[i];
            q.c[i] = make_consts(p);
            const uint64_t seed = p->prm.seed + (uint64_t)i;         // per-event stream
            q.c[i].key0 = (uint32_t)seed;
            q.c[i].key1 = (uint32_t)(seed >> 32);
            q.d[i] = depo_arrays(&depos[i]);
            q.grid[i] = p->bgrid + (size_t)slot[i] * ev_grid_elems(p->dims);
            q.flags[i] = p->flags;
            q.block_start[i + 1] = q.block_start[i] + rasterize_blocks(depos[i].n, c0.depos_per_block);
        }
        cudaError_t e = launch_rasterize_queue(q, planes[0]->queue, s);
        if (e) return cuda_fail(e, "batch rasterize launch");
    } else {
        for (int g = 0; g < n_groups; ++g) {
            wcsim_status st = rasterize_group(planes[first[g]], count[g], members[g], depos, s);
            if (st) return st;
        }
    }
    for (int g = 0; g < n_groups; ++g) {
        wcsim_status st = convolve_group(planes[first[g]], count[g], members[g], waves,
                                         clean_after[g], s);
        if (st) return st;
    }
    return WCSIM_OK;
}

wcsim_status wcsim_plane_autotune(wcsim_plane* pl, const wcsim_depos* depos, void* stream,
                                  wcsim_tune_report* report)
{
    if (!pl) return fail(WCSIM_EINVAL, "plane is NULL");
    pl->fwd_valid = false;
    wcsim_status st = check_depos(depos);
    if (st) return st;
    DeviceGuard dg(pl->device);
    if (!dg.ok) return fail(WCSIM_ECUDA, "cannot select the plane's device");
    cudaStream_t s = (cudaStream_t)stream;
    ConvDims& d = pl->dims;
    const size_t grid_bytes = (size_t)d.n_w * d.n_imp * d.n_t * sizeof(float);
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) || cudaEventCreate(&e1)) return fail(WCSIM_ECUDA, "event creation failed");
    cudaError_t err = cudaSuccess;
    int timed = 0;
    // best of 5 after 2 warm-ups, in ms; sets err on a launch failure
    auto time_it = [&](auto fn) -> float {
        for (int i = 0; i < 2 && !err; ++i) err = fn();
        float best = 1e30f;
        for (int i = 0; i < 5 && !err; ++i) {
            cudaEventRecord(e0, s);
            err = fn();
            cudaEventRecord(e1, s);
            if (!err) err = cudaEventSynchronize(e1);
            float ms = 0.f;
            if (!err) err = cudaEventElapsedTime(&ms, e0, e1);
            if (ms < best) best = ms;
        }
        ++timed;
        return best;
    };
    wcsim_tune_report rep{};
    // 1. rasterization tile: depos per CTA, lanes per depo
    {
        const int tiles[][2] = {{32, 8}, {64, 8}, {128, 8}, {256, 8}, {64, 16}, {128, 16},
                                {256, 16}, {64, 32}, {128, 32}, {256, 32}};
        float best = 1e30f;
        for (const auto& t : tiles) {
            pl->kd = t[0];
            pl->kg = t[1];
            RasterConsts c = make_consts(pl);
            const float ms = time_it([&] { return launch_rasterize(c, depo_arrays(depos), pl->grid, pl->flags, s); });
            if (ms < best) { best = ms; rep.depos_per_block = t[0]; rep.lanes_per_depo = t[1]; }
        }
        pl->kd = rep.depos_per_block;
        pl->kg = rep.lanes_per_depo;
        rep.ms_rasterize = best;
        // a representative grid for the FFT stages
        if (!err) err = cudaMemsetAsync(pl->grid, 0, grid_bytes, s);
        if (!err) err = launch_rasterize(make_consts(pl), depo_arrays(depos), pl->grid, pl->flags, s);
    }
    // 2. time-axis plan: forward over the grid + inverse (into the grid's first rows)
    int32_t cand[8][kMaxPasses], cnp[8];
    const int nc = err ? 0 : fft_plan_candidates(d.n_ft, cand, cnp, 8);
    {
        float best = 1e30f;
        int bi = -1;
        FftPlan bp{};
        float2* btw = nullptr;
        const int keep_variant = d.rows_variant;
        d.rows_variant = 0;
        for (int ci = 0; ci < nc && !err; ++ci) {
            FftPlan p;
            float2* tw = nullptr;
            if ((err = fft_plan_create_radices(d.n_ft, cand[ci], cnp[ci], &p, &tw))) break;
            const float ms = time_it([&] { return launch_rows_r2c(d, p, pl->grid, pl->shat, pl->flags, s); }) +
                             time_it([&] { return launch_rows_c2r(d, p, pl->mt, pl->grid, s); });
            if (!err && ms < best) {
                best = ms;
                bi = ci;
                cudaFree(btw);
                bp = p;
                btw = tw;
            } else {
                cudaFree(tw);
            }
        }
        d.rows_variant = keep_variant;
        if (bi >= 0 && !err) {
            cudaFree(pl->tw_t);
            pl->pt = bp;
            pl->fused_fits = fused_supported(pl->pt);
            pl->tw_t = btw;
        } else {
            cudaFree(btw);
        }
        for (int i = 0; i < pl->pt.npass && i < 8; ++i) rep.time_radix[i] = pl->pt.radix[i];
        rep.ms_rows = best;
    }
    // 3. time-axis forward kernel: direct (clears its input) vs staged (+ a grid reset)
    if (!err) {
        if (!err) err = cudaMemsetAsync(pl->grid, 0, grid_bytes, s);
        if (!err) err = launch_rasterize(make_consts(pl), depo_arrays(depos), pl->grid, pl->flags, s);
        const int keep = d.rows_variant;
        d.rows_variant = 0;
        const float direct = time_it([&] { return launch_rows_r2c(d, pl->pt, pl->grid, pl->shat, pl->flags, s); });
        d.rows_variant = 1;
        const float staged = time_it([&] {
            cudaError_t x = cudaMemsetAsync(pl->grid, 0, grid_bytes, s);
            return x ? x : launch_rows_r2c(d, pl->pt, pl->grid, pl->shat, pl->flags, s);
        });
        d.rows_variant = (staged < direct) ? 1 : 0;
        (void)keep;
        rep.rows_variant = d.rows_variant;
    }
    // 4. wire pass: warp-per-column vs block-level
    if (!err) {
        float warp = 1e30f, block;
        if (pl->tw_warp)
            warp = time_it([&] { return launch_wire_warp(d, pl->tw_warp, pl->shat, pl->H, pl->mt, pl->flags, s); });
        block = time_it([&] { return launch_wire_pass(d, pl->pw, pl->shat, pl->H, pl->mt, pl->flags, s); });
        pl->wire_block = !(warp <= block);
        rep.wire_variant = pl->wire_block ? 1 : 0;
        rep.ms_wire = pl->wire_block ? block : warp;
    }
    // 5. forward variant: the whole wcsim_run, plain and fused (into a temporary frame)
    rep.forward_fused = pl->fused ? 1 : 0;
    if (!err && pl->fused_fits && pl->prm.fluctuate != 2 && depos->n < ((int64_t)1 << 31)) {
        float* wave = nullptr;
        err = cudaMalloc(&wave, (size_t)d.n_w * d.n_t * sizeof(float));
        if (!err) {
            const bool keep_timing = pl->timing;
            pl->timing = false;
            wcsim_status st2 = WCSIM_OK;
            auto fwd = [&](bool fused) {
                pl->fused = fused;
                return [&, fused]() -> cudaError_t {
                    pl->fused = fused;
                    st2 = wcsim_run(pl, depos, wave, stream);
                    return st2 == WCSIM_OK ? cudaSuccess : cudaErrorLaunchFailure;
                };
            };
            rep.ms_forward_plain = time_it(fwd(false));
            if (!err) rep.ms_forward_fused = time_it(fwd(true));
            pl->fused = !err && rep.ms_forward_fused < rep.ms_forward_plain;
            rep.forward_fused = pl->fused ? 1 : 0;
            pl->timing = keep_timing;
            cudaFree(wave);
            if (st2 != WCSIM_OK) {
                cudaEventDestroy(e0);
                cudaEventDestroy(e1);
                return st2;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    pl->grid_clean = false;
    if (err) return cuda_fail(err, "autotune");
    rep.candidates_timed = timed;
    if (report) *report = rep;
    return WCSIM_OK;
}

wcsim_status wcsim_windows(wcsim_plane* pl, const wcsim_depos* depos, int32_t* out, void* stream)
{
    if (!pl) return fail(WCSIM_EINVAL, "plane is NULL");
    wcsim_status st = check_depos(depos);
    if (st) return st;
    if (!out && depos->n > 0) return fail(WCSIM_EINVAL, "out is NULL");
    if (((uintptr_t)out & 15) != 0) return fail(WCSIM_EINVAL, "out must be 16-byte aligned");
    pl->fwd_valid = false;
    DeviceGuard dg(pl->device);
    if (!dg.ok) return fail(WCSIM_ECUDA, "cannot select the plane's device");
    cudaError_t e = launch_windows(make_consts(pl), depo_arrays(depos), out, pl->flags,
                                   (cudaStream_t)stream);
    return e ? cuda_fail(e, "windows launch") : WCSIM_OK;
}

wcsim_status wcsim_plane_check(wcsim_plane* pl, void* stream, int32_t* flags)
{
    if (!pl) return fail(WCSIM_EINVAL, "plane is NULL");
    DeviceGuard dg(pl->device);
    if (!dg.ok) return fail(WCSIM_ECUDA, "cannot select the plane's device");
    cudaStream_t s = (cudaStream_t)stream;
    int h = 0;
    cudaError_t e = cudaMemcpyAsync(&h, pl->flags, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (!e) e = cudaMemsetAsync(pl->flags, 0, sizeof(int), s);
    if (!e) e = cudaStreamSynchronize(s);
    if (e) return cuda_fail(e, "flag read");
    if (flags) *flags = h;
    if (h & kErrTimeout)
        return fail(WCSIM_ETIMEOUT, "a device-side wait for an asynchronous copy gave up (flags 0x%x)", h);
    if (h) return fail(WCSIM_EDEVICE_CHECK, "device flagged invalid depo values (flags 0x%x)", h);
    return WCSIM_OK;
}

wcsim_status wcsim_plane_set_noise(wcsim_plane* pl, const float* amp, int32_t n_amp,
                                   uint64_t seed, void* stream)
{
    if (!pl) return fail(WCSIM_EINVAL, "plane is NULL");
    if (!amp || n_amp == 0) {
        cudaFree(pl->noise_amp);
        pl->noise_amp = nullptr;
        return WCSIM_OK;
    }
    if (n_amp != pl->dims.nh)
        return fail(WCSIM_ESHAPE, "the noise amplitude spectrum needs n_ft / 2 + 1 = %d values (got %d)",
                    pl->dims.nh, n_amp);
    DeviceGuard dg(pl->device);
    if (!dg.ok) return fail(WCSIM_ECUDA, "cannot select the plane's device");
    std::vector<float> a((size_t)n_amp);
    for (int k = 0; k < n_amp; ++k) {
        if (!(amp[k] >= 0.0f) || !isfinite(amp[k]))
            return fail(WCSIM_EINVAL, "noise amplitude %d is negative or not finite", k);
        a[(size_t)k] = (float)((double)amp[k] / (double)pl->dims.n_ft);
    }
    cudaError_t e = cudaSuccess;
    if (!pl->noise_amp) e = cudaMalloc(&pl->noise_amp, (size_t)n_amp * sizeof(float));
    cudaStream_t s = (cudaStream_t)stream;
    if (!e) e = cudaMemcpyAsync(pl->noise_amp, a.data(), (size_t)n_amp * sizeof(float),
                                cudaMemcpyHostToDevice, s);
    if (!e) e = cudaStreamSynchronize(s);
    if (e) return cuda_fail(e, "noise spectrum upload");
    pl->noise_seed = seed;
    return WCSIM_OK;
}

wcsim_status wcsim_plane_set_raster_tile(wcsim_plane* pl, int32_t depos_per_block,
                                         int32_t lanes_per_depo)
{
    if (!pl) return fail(WCSIM_EINVAL, "plane is NULL");
    if (!raster_tile_supported(depos_per_block, lanes_per_depo))
        return fail(WCSIM_EINVAL, "no rasterization tile of %d depos per CTA and %d lanes per depo",
                    depos_per_block, lanes_per_depo);
    pl->kd = depos_per_block;
    pl->kg = lanes_per_depo;
    return WCSIM_OK;
}

wcsim_status wcsim_plane_set_forward(wcsim_plane* pl, int32_t fused)
{
    if (!pl) return fail(WCSIM_EINVAL, "plane is NULL");
    if (fused != 0 && fused != 1) return fail(WCSIM_EINVAL, "fused must be 0 or 1 (got %d)", fused);
    pl->fused = fused != 0;
    pl->fwd_valid = false;
    return WCSIM_OK;
}

wcsim_status wcsim_plane_set_reuse_forward(wcsim_plane* pl, int32_t enable)
{
    if (!pl) return fail(WCSIM_EINVAL, "plane is NULL");
    if (enable < 0 || enable > 2) return fail(WCSIM_EINVAL, "enable must be 0, 1 or 2 (got %d)", enable);
    pl->fwd_valid = false;
    pl->s2d_valid = false;
    if (enable == 2 && pl->tw_warp && !pl->s2d) {
        DeviceGuard dg(pl->device);
        if (!dg.ok) return fail(WCSIM_ECUDA, "cannot select the plane's device");
        const ConvDims& d = pl->dims;
        const size_t n = (size_t)d.n_imp * d.n_fw * kBlockCols * d.nkb;
        cudaError_t e = cudaMalloc(&pl->s2d, n * sizeof(float2));
        if (e) {
            pl->s2d = nullptr;
            return cuda_fail(e, "2D spectra allocation");
        }
    } else if (enable != 2 && pl->s2d) {
        DeviceGuard dg(pl->device);
        cudaFree(pl->s2d);              // synchronising: no work of the plane is in flight after
        pl->s2d = nullptr;
    }
    pl->reuse_fwd = enable != 0;
    return WCSIM_OK;
}

wcsim_status wcsim_plane_set_wait_limit(wcsim_plane* pl, uint64_t ns)
{
    if (!pl) return fail(WCSIM_EINVAL, "plane is NULL");
    pl->dims.wait_ns = ns;
    return WCSIM_OK;
}

wcsim_status wcsim_plane_set_timing(wcsim_plane* pl, int32_t enable)
{
    if (!pl) return fail(WCSIM_EINVAL, "plane is NULL");
    pl->timing = enable != 0;
    return WCSIM_OK;
}

wcsim_status wcsim_plane_stage_times(wcsim_plane* pl, float* ms, int32_t n)
{
    if (!pl || (!ms && n > 0)) return fail(WCSIM_EINVAL, "plane or ms is NULL");
    if (!pl->timing) return fail(WCSIM_EINVAL, "timing is not enabled on this plane");
    DeviceGuard dg(pl->device);
    if (!dg.ok) return fail(WCSIM_ECUDA, "cannot select the plane's device");
    cudaError_t e = cudaSuccess;
    float sum[kStages] = {};
    for (int i = 0; i < pl->tl_n; ++i)
        if ((e = cudaEventSynchronize(pl->ev[i]))) return cuda_fail(e, "event synchronize");
    for (int i = 0; i < pl->sp_n; ++i) {
        float t = 0.f;
        if ((e = cudaEventElapsedTime(&t, pl->ev[pl->sp_b[i]], pl->ev[pl->sp_e[i]])))
            return cuda_fail(e, "event elapsed time");
        const int k = pl->sp_kind[i];
        if (k >= 0 && k < kStages) sum[k] += t;
    }
    for (int i = 0; i < n && i < kStages; ++i) ms[i] = sum[i];
    for (int i = 0; i < kBwdStages && kStages + i < n; ++i) {
        float t = 0.f;
        if (pl->bwd_recorded) {
            if (i == 0 && (e = cudaEventSynchronize(pl->evb[kBwdStages]))) return cuda_fail(e, "event synchronize");
            if ((e = cudaEventElapsedTime(&t, pl->evb[i], pl->evb[i + 1]))) return cuda_fail(e, "event elapsed time");
        }
        ms[kStages + i] = t;
    }
    return WCSIM_OK;
}

wcsim_status wcsim_plane_destroy(wcsim_plane* pl)
{
    if (!pl) return WCSIM_OK;
    DeviceGuard dg(pl->device);
    plane_free(pl);
    return WCSIM_OK;
}

}  // extern "C"
