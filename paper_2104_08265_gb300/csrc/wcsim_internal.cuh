// Internal declarations shared by the CUDA translation units of libwcsim.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/wcsim.h"

struct CUtensorMap_st;     // the driver's tensor map (cuda.h), by pointer only here

namespace wcsim {

// ------------------------------------------------------------------ depo rasterization
// Per-call constants of the drift + bin decision.  The FP64 fields place a depo on the
// grid (positions reach metres, bins are a fraction of a mm); the FP32 fields give the
// half-width n*sigma/bin.  Both are formed on the host once per call.
struct RasterConsts {
    double p0, t0, inv_dp, inv_dt;          // FP64: origins, 1/bin
    float two_dt, two_dl, inv_v, nsig;      // FP32: 2 D_T, 2 D_L [mm^2/us], 1/v, n_sigma
    float inv_dp_f, inv_dt_f;               // FP32 copies of 1/bin
    float dp_f, dt_f;                       // FP32 bin sizes [mm], [us]
    float inv_tau;                          // FP32 1/lifetime
    int64_t n_rows;                         // n_wires * n_imp
    int32_t n_ticks;
    int32_t fluctuate;
    int32_t renorm;                         // 1: each axis' weights divided by their window sum
    uint32_t key0, key1, plane_id;
    double DL, DT, v, tau;                  // FP64 parameters for the global gradients
    int32_t depos_per_block;                // rasterization tile: depos per CTA and lanes
    int32_t lanes_per_depo;                 // per depo (raster_tile_supported)
    float stirl[16];                        // Stirling's remainder log m! - [(m + 1/2) log m
                                            // - m + 1/2 log 2 pi], m = 0..15 (exact binomial)
};

struct DepoGrads {
    float *dq, *dp, *dt, *dsl, *dst;        // per depo, each may be null
    double* dglobal;                        // [3]: dL/dD_L, dL/dD_T, dL/dtau (accumulated)
};

struct DepoArrays {
    const double* p;
    const double* t;
    const double* td;
    const float* q;
    const uint32_t* id;
    int64_t n;
};

constexpr int kMaxBatch = 64;          // events per batched launch

// Per-event inputs of a batched rasterization, passed by value.
struct BatchEvents {
    int32_t n;
    int32_t block_start[kMaxBatch + 1];  // first CTA of each event (prefix sum)
    DepoArrays d[kMaxBatch];
    float* grid[kMaxBatch];
    uint32_t key0[kMaxBatch], key1[kMaxBatch];
};

// Every event of a batch, whatever its plane, for one persistent rasterization over a work
// queue of (event, depo block) items; passed by value.
struct QueueEvents {
    int32_t n;
    int32_t block_start[kMaxBatch + 1];  // first item of each event (prefix sum)
    RasterConsts c[kMaxBatch];           // the event's plane constants and fluctuation key
    DepoArrays d[kMaxBatch];
    float* grid[kMaxBatch];
    int* flags[kMaxBatch];               // the event's plane's flag word
};

struct WavePtrs {
    float* p[kMaxBatch];
    int32_t ev[kMaxBatch];     // event index within the caller's batch (noise key offset)
};

cudaError_t launch_rasterize(const RasterConsts& c, const DepoArrays& d, float* grid,
                             int* flags, cudaStream_t s);
cudaError_t launch_windows(const RasterConsts& c, const DepoArrays& d, int32_t* out,
                           int* flags, cudaStream_t s);
// Rasterize several events of one plane in one launch (c.key0/key1 ignored: per event).
cudaError_t launch_rasterize_batch(const RasterConsts& c, const BatchEvents& ev, int* flags,
                                   cudaStream_t s);
int rasterize_blocks(int64_t n_depos, int depos_per_block);
// Rasterize every event of q in one persistent launch: CTAs pop (event, block) items from
// *queue (zeroed here on the stream first) until all q.block_start[q.n] are done.  All events
// use the tile (depos_per_block, lanes_per_depo) and fluctuation mode of q.c[0].
cudaError_t launch_rasterize_queue(const QueueEvents& q, int* queue, cudaStream_t s);
// Whether the rasterizers have an instance for this tile (depos per CTA, lanes per depo).
bool raster_tile_supported(int depos_per_block, int lanes_per_depo);
// Adjoint of drift + rasterization (mean path, windows fixed): dgrid -> per-depo and global
// gradients (dglobal must be zeroed by the caller).
cudaError_t launch_depo_adjoint(const RasterConsts& c, const DepoArrays& d, const float* dgrid,
                                const DepoGrads& g, int* flags, cudaStream_t s);

// ------------------------------------------------------------------ FFT
constexpr int kMaxPasses = 16;
constexpr int kMaxFftN = 13500;       // time axis: two padded N-point buffers per CTA
constexpr int kMaxWireN = 8192;

// Mixed-radix Stockham plan for one length N = prod(radix[p]).  Pass p combines groups
// of ns[p] already-transformed points; tw_off[p] indexes its (radix-1) * ns twiddles in
// the plan's table (entry (r - 1) ns + k = exp(-2 pi i r k / (ns radix)));
// ns_magic[p] = ceil(2^32 / ns[p]) turns j / ns into a multiply-high.
struct FftPlan {
    int32_t n;
    int32_t npass;
    int32_t radix[kMaxPasses];
    int32_t ns[kMaxPasses];
    int32_t tw_off[kMaxPasses];
    uint32_t ns_magic[kMaxPasses];
    const float2* tw;                 // device table, forward sign (exp(-i ...))
};

// Factor n into register-DFT radices (<= 25, primes 2, 3, 5, 7) with the fewest passes;
// false if impossible.
bool fft_factor(int n, int32_t* radix, int32_t* npass);
// Build the plan and upload its twiddle table (FP64 host values rounded to FP32).
cudaError_t fft_plan_create(int n, FftPlan* plan, float2** dev_tw);
// Alternative plans for autotuning: the default first, then other radix sets with the
// same pass count (decreasing order, and radix 16 first where present).  Returns the count.
int fft_plan_candidates(int n, int32_t (*radix)[kMaxPasses], int32_t* npass, int max_out);
// A plan with the given radices (in pass order) and its uploaded twiddle table.
cudaError_t fft_plan_create_radices(int n, const int32_t* radices, int npass, FftPlan* plan,
                                    float2** dev_tw);
// The plan without its table (plan->tw left NULL); returns the table length in entries,
// or -1 if n does not factor.  Allocates nothing.
int fft_plan_describe(int n, FftPlan* plan);
// Record a failure message for wcsim_last_error() and return s.
wcsim_status report_error(wcsim_status s, const char* msg);

// Spectra over (time frequency kt < nh, wire or wire frequency) are stored in blocks of
// kBlockCols adjacent time frequencies: element (kt, w) of an [n][nh] spectrum lives at
// ((kt / 4) * n + w) * 4 + kt % 4.  One block is a contiguous 32 n-byte tile: the wire
// pass fetches it with a single bulk copy.  Columns nh .. 4 nkb - 1 are zero.
constexpr int kBlockCols = 4;

struct ConvDims {
    int32_t n_w, n_imp, n_t;   // frame
    int32_t n_fw, n_ft;        // FFT sizes
    int32_t nh;                // n_ft / 2 + 1
    int32_t nkb;               // ceil(nh / kBlockCols)
    int32_t rows_variant;      // time-axis forward kernel: 0 direct loads, 1 bulk-staged
    int32_t clear_input;       // time-axis forward: write zeros over the rows it has read
    int32_t spectra_tma = 1;   // time-axis kernels: blocked half spectra by TMA box copies
    int32_t adj_split = 0;     // one-warp wire adjoint: CTAs per frequency block (0: chosen
                               // from the wave fill, adjoint_split)
    // Batched runs: event e's grid, time-axis spectra and wire-summed spectra start
    // e * ev_grid, e * ev_shat and e * ev_mt elements after the first event's.
    int64_t ev_grid, ev_shat, ev_mt;
    // limit of each device-side wait for a bulk asynchronous copy (ns of %globaltimer);
    // a wait that runs out raises the timeout flag and its CTA leaves
    uint64_t wait_ns = 2000000000ull;
    // Eq. 1's noise, added to the wire-summed time spectra as the inverse time FFT stages
    // them (null: none): A(k) / n_ft for k < nh (device), Philox key = noise_seed + event
    // index, counter word 3 = plane_id
    const float* noise_amp = nullptr;
    uint64_t noise_seed = 0;
    uint32_t plane_id = 0;
    // adc_max > 0: the inverse time FFT writes ADC codes (uint16) instead of floats:
    // clamp(floor(fl(fl(adc_gain M) + adc_pedestal) + 1/2), 0, adc_max)
    float adc_gain = 0.0f, adc_pedestal = 0.0f;
    int32_t adc_max = 0;
    // target != null (single runs): the inverse time FFT writes M - target (the same
    // [n_w][n_t] layout) instead of M and, with loss, adds 1/2 sum (M - target)^2 to *loss
    // (FP32 within a warp, FP64 across warps)
    const float* target = nullptr;
    double* loss = nullptr;
};


__host__ __device__ inline int64_t blk_index(int kt, int w, int n)
{
    return ((int64_t)(kt >> 2) * n + w) * kBlockCols + (kt & 3);
}

// H_j(kt, kw) = s * (R_j[kw][kt] + conj(R_j[-kw][-kt])) / 2, stored time-frequency major,
// [n_imp][4 nkb][n_fw] (zero for kt >= nh): the 4 columns of a block are 4 contiguous rows
// of n_fw, so one block's tile is contiguous and a warp reads a column with consecutive
// lanes on consecutive wires.
cudaError_t launch_make_hermitian(const ConvDims& d, const float2* resp, float2* H, float scale,
                                  cudaStream_t s);
// Time-axis real-to-complex FFT of every grid row; writes Shat_j blocked
// [n_imp][nkb][n_w][4].
cudaError_t launch_rows_r2c(const ConvDims& d, const FftPlan& pt, const float* grid,
                            float2* shat, int* flags, cudaStream_t s);
// Same for n_ev events laid out with the ConvDims event strides (direct kernel).
cudaError_t launch_rows_r2c_batch(const ConvDims& d, const FftPlan& pt, const float* grid,
                                  float2* shat, int n_ev, cudaStream_t s);
// Per block of time frequencies: wire FFT of each S_j, times H_j, summed over j, inverse
// wire FFT; writes Mt blocked [nkb][n_w][4].
cudaError_t launch_wire_pass(const ConvDims& d, const FftPlan& pw, const float2* shat,
                             const float2* H, float2* mt, int* flags, cudaStream_t s);
// Wire axes of 32 M points, M in this set, run as one warp per time frequency
// (lanes x registers, no block barriers); others use the block-level engine.
bool wire_warp_supported(int n_fw);
// Twiddles of the warp kernel: [2][n_fw], exp(-2 pi i a b / n_fw) at a * 32 + b (a < M,
// b < 32) and at b * M + a, FP64 rounded to FP32.  Device allocation owned by the caller.
cudaError_t wire_warp_twiddles(int n_fw, float2** dev);
// s2d (n_ev = 1 only): also write the 2D spectra of S (every Shat_j column's wire FFT,
// before the product with H_j), time-frequency major [n_imp][4 nkb][n_fw] complex.
cudaError_t launch_wire_warp(const ConvDims& d, const float2* tw2, const float2* shat,
                             const float2* H, float2* mt, int* flags, cudaStream_t s,
                             int n_ev = 1, float2* s2d = nullptr);
// Adjoint of the wire pass (n_fw = 32 M): reads the time-axis spectra of the forward grid
// (shat) and of G (gt, blocked [nkb][n_w][4]); overwrites shat with the time-axis spectra
// of dL/dS and, if dR is not null, writes dL/dR_j (full [n_imp][n_fw][n_ft] layout).  g2d
// (blocked [nkb][n_fw][4]) receives the 2D spectrum of G on the way.
cudaError_t launch_wire_adjoint_warp(const ConvDims& d, const float2* tw2, const float2* gt,
                                     float2* shat, const float2* H, float2* g2d, float2* dR,
                                     float inv_n, cudaStream_t s);
// dL/dR_j from the forward's kept 2D spectra of S (s2d, [n_imp][4 nkb][n_fw], see
// launch_wire_warp) and G's 2D spectrum (g2d, blocked [nkb][n_fw][4]; part A with dR null
// writes it): the full [n_imp][n_fw][n_ft] layout, Hermitian mirror included.
cudaError_t launch_dr_rows(const ConvDims& d, const float2* s2d, const float2* g2d, float2* dR,
                           float inv_n, cudaStream_t s);
// The same adjoint for any wire FFT size, block-level engine (plan pw): gt, shat, dR as above;
// no 2D spectrum of G is kept.
cudaError_t launch_wire_adjoint_block(const ConvDims& d, const FftPlan& pw, const float2* gt,
                                      float2* shat, const float2* H, float2* dR, float inv_n,
                                      cudaStream_t s);
// TMA view of a blocked spectrum array [n_ev][n_j][nkb][n_w][4] complex (ev_stride complex
// values from one event to the next): a 5-D FP32 tensor map whose box is one row's half
// spectrum over blocked_box_kb(nkb) frequency blocks (4 complex values per block, dense in
// shared memory).  False when the driver offers no encoder or the layout cannot be mapped
// (base not 16-byte aligned); *out is then unspecified.
constexpr int kMapBoxKb = 256;          // the TMA limit on a box dimension
// Frequency blocks per box: nkb itself up to the limit, else the fewest boxes of equal size,
// rounded up to a multiple of 4 blocks (so that every box starts on a 128-byte boundary of a
// dense shared buffer); the last box may reach past nkb (clipped by the copy).
int blocked_box_kb(int nkb);
bool blocked_spectra_map(const float2* base, int n_w, int nkb, int n_j, int n_ev,
                         int64_t ev_stride, ::CUtensorMap_st* out);
// Inverse time-axis FFT of every grid row from blocked spectra [n_imp][nkb][n_w][4].
cudaError_t launch_rows_c2r_grid(const ConvDims& d, const FftPlan& pt, const float2* shat,
                                 float* grid, cudaStream_t s);
// Time-axis complex-to-real inverse FFT of the Hermitian half rows of Mt -> wave.
cudaError_t launch_rows_c2r(const ConvDims& d, const FftPlan& pt, const float2* mt,
                            float* wave, cudaStream_t s);
cudaError_t launch_rows_c2r_batch(const ConvDims& d, const FftPlan& pt, const float2* mt,
                                  const WavePtrs& waves, int n_ev, cudaStream_t s);

// ------------------------------------------------------------------ fused rasterization
// Rasterization inside the time-axis transform: depos are binned by the first wire their rows
// reach, and each transform CTA rasterizes the depos of its wire's neighbourhood straight into
// its shared-memory rows, so that the grid S is never written.
struct Decision;
constexpr size_t kDecisionBytes = 64;   // sizeof(Decision)
constexpr int kFusedSpan = 4;     // a depo reaching over more wires goes to the "wide" bucket
constexpr int kFusedSlots = 24;   // tick weights stored per binned depo (6 four-tick groups)

// Scratch of the binning pass, cap depos.
struct FusedScratch {
    Decision* dec = nullptr;      // [cap] decisions in depo order
    int32_t* pos = nullptr;       // [cap] slot within its bucket, -1 if the depo adds nothing
    int32_t* cnt = nullptr;       // [n_w + 1] bucket counts (zero between calls)
    int32_t* off = nullptr;       // [n_w + 2] bucket offsets, off[n_w + 1] = binned depos
    Decision* sorted = nullptr;   // [cap] decisions in bucket order
    float* wts = nullptr;         // [cap][kFusedSlots] tick weights of `sorted`
    int64_t cap = 0;
};

// What the transform reads of the binning (passed by value).
struct FusedBins {
    const Decision* sorted;
    const float* wts;
    const int32_t* off;
    int32_t n_w;                  // index of the wide bucket
    int64_t cap;                  // entries of sorted / wts
};

// The fused transform fits shared memory for this time-axis plan.
bool fused_supported(const FftPlan& pt);
// Decide and bin every depo (three launches); c.depos_per_block is ignored.
cudaError_t launch_bin_depos(const RasterConsts& c, const DepoArrays& d, int n_imp, int n_w,
                             const FusedScratch& s, int* flags, cudaStream_t st);
// Rasterize the binned depos into every grid row (two rows of one wire per CTA) and
// transform the rows; writes the half spectra to shat (blocked [n_imp][nkb][n_w][4]) as the
// plain transform does.
cudaError_t launch_rows_r2c_fused(const ConvDims& d, const FftPlan& pt, const RasterConsts& c,
                                  const FusedScratch& s, float2* shat, cudaStream_t st);

// Streaming multiprocessors of the current device (cached).
int sm_count();

// A once-per-device flag: kernel attributes (cudaFuncSetAttribute) are set per device, so a
// process that drives several GPUs sets them once on each.
class DeviceOnce {
public:
    // true if the current device has not been marked yet
    bool pending() const { const int d = dev(); return d < 0 || d >= kMax || !done_[d]; }
    void mark() { const int d = dev(); if (d >= 0 && d < kMax) done_[d] = true; }

private:
    static constexpr int kMax = 64;
    static int dev() { int d = -1; return cudaGetDevice(&d) == cudaSuccess ? d : -1; }
    bool done_[kMax] = {};
};

}  // namespace wcsim
