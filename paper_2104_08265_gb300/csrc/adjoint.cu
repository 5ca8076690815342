// Adjoint of the Eq. 2 convolution.
//
// The forward computes M = IFFT2(sum_j H_j FFT2(S_j)) with H_j the Hermitian part of R_j
// (scaled by 1/(n_fw n_ft)).  For a loss L with G = dL/dM:
//   dL/dS_j = IFFT2(conj(H_j) FFT2(G))                (same unnormalised inverse, same scale)
//   dL/dR_j = conj(FFT2(S_j)) FFT2(G) / (n_fw n_ft)    (complex-gradient convention dRe + i dIm)
// The wire-axis adjoint runs as two one-warp-per-time-frequency kernels (n_fw = 32 M, the
// layout of the forward warp kernel), each doing one wire FFT per impact position: part A
// transforms G's column once and, per j, S_j's column, writing dL/dR_j at (kw, kt) and its
// Hermitian mirror (-kw, -kt); part B forms conj(H_j) G^ and transforms it back, overwriting
// S_j's column with the time-axis spectrum of dL/dS_j.  When the forward kept the 2D spectra
// of S, part A transforms G alone and dr_tiles forms dL/dR_j from the kept spectra.
// rows_c2r_grid: the inverse time-axis FFT of those spectra for every grid row.
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>

#include "fft_engine.cuh"
#include "warp_fft.cuh"
#include "wcsim_internal.cuh"

namespace wcsim {
namespace {

constexpr int kWarps = 4;     // = kBlockCols: warp c takes column c of a block

// Adjoint part A, one warp per time frequency kt: G^ = wire FFT of G's time-axis spectrum
// (kept for part B in g2d, blocked [nkb][n_fw][4]); for every j, the wire FFT of S_j and
// dL/dR_j(kw, kt) = conj(S^_j) G^ / n with its Hermitian mirror (-kw, -kt).  G^ stays in
// shared memory; each warp leaves its output column in its own transpose buffer (column c at
// c * TR), from which the rows of dL/dR_j are written 4 adjacent values at a time.
template <int M>
__global__ void __launch_bounds__(kWarps * 32, 3)
k_wire_adjoint_a(ConvDims d, const float2* __restrict__ tw2, const float2* __restrict__ gt,
                 const float2* __restrict__ shat, float2* __restrict__ g2d, float2* __restrict__ dR,
                 float inv_n)
{
    // per-warp region >= 33 M (the transpose tile) with TR = 4 mod 16: the four output
    // columns then start 32 bytes apart modulo 128 and the row-wise reads below are free of
    // bank conflicts
    constexpr int N = 32 * M, TR = 33 * M + ((4 - 33 * M) % 16 + 16) % 16;
    static_assert(TR % 16 == 4 && TR >= 33 * M, "transpose region stride");
    __shared__ float2 s_twf[N];
    __shared__ __align__(16) float2 s_tr[kWarps * TR];
    // dynamic: G^'s columns [4][ld] (warp c's at c * ld), kept for every j
    extern __shared__ __align__(128) unsigned char smraw[];
    float2* s_g = reinterpret_cast<float2*>(smraw);
    load_wire_twiddles<M>(tw2, s_twf, nullptr);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int kb = blockIdx.x, c = warp, kt0 = kb * kBlockCols;
    // impacts j0 <= j < j1 of this CTA (grid y splits the impacts; every part transforms G)
    const int j0 = (int)((int64_t)blockIdx.y * d.n_imp / gridDim.y);
    const int j1 = (int)((int64_t)(blockIdx.y + 1) * d.n_imp / gridDim.y);
    float2* tr = s_tr + warp * TR;
    float2* gcol = s_g + c * tile_ld(N);

    {
        float2 v[M], g[32];
        load_col<M>(gt + (int64_t)kb * d.n_w * kBlockCols, c, d.n_w, lane, v);
        warp_fft_fwd<M>(v, s_twf, tr, lane, g);
        if (lane < M) {
#pragma unroll
            for (int k1 = 0; k1 < 32; ++k1) gcol[lane + M * k1] = g[k1];
        }
    }
    __syncthreads();
    if (blockIdx.y == 0) store_tile_cols(s_g, N, tile_ld(N), g2d + (int64_t)kb * N * kBlockCols);
    if (dR == nullptr || kt0 >= d.nh || j0 >= j1) return;   // uniform per CTA
    const bool vec = (d.n_ft % 2) == 0 && (reinterpret_cast<uintptr_t>(dR) & 15) == 0;
    // S_j's column is loaded one impact ahead: the loads of S_{j+1} are in flight while the
    // rows of dL/dR_j are written
    float2 v[M];
    load_col<M>(shat + ((int64_t)j0 * d.nkb + kb) * d.n_w * kBlockCols, c, d.n_w, lane, v);
    for (int j = j0; j < j1; ++j) {
        float2 u[32];
        __syncthreads();                                  // s_tr is read out
        warp_fft_fwd<M>(v, s_twf, tr, lane, u);
        if (lane < M) {
#pragma unroll
            for (int k1 = 0; k1 < 32; ++k1) {
                const float2 g = gcol[lane + M * k1];
                tr[lane + M * k1] = make_float2(inv_n * (u[k1].x * g.x + u[k1].y * g.y),
                                                inv_n * (u[k1].x * g.y - u[k1].y * g.x));
            }
        }
        __syncthreads();
        if (j + 1 < j1)
            load_col<M>(shat + ((int64_t)(j + 1) * d.nkb + kb) * d.n_w * kBlockCols, c, d.n_w, lane, v);
        float2* dRj = dR + (int64_t)j * N * d.n_ft;
        // direct values (kw, kt0 + cc), kt < nh: pairs of columns as 16-byte stores
        for (int e = threadIdx.x; e < N * 2; e += blockDim.x) {
            const int kw = e >> 1, cc = (e & 1) * 2, kt = kt0 + cc;
            const float2 a = s_tr[cc * TR + kw], b = s_tr[(cc + 1) * TR + kw];
            float2* row = dRj + (int64_t)kw * d.n_ft;
            if (vec && kt + 1 < d.nh) {
                *reinterpret_cast<float4*>(row + kt) = make_float4(a.x, a.y, b.x, b.y);
            } else {
                if (kt < d.nh) row[kt] = a;
                if (kt + 1 < d.nh) row[kt + 1] = b;
            }
        }
        // mirrors (-kw, n_ft - kt) for 1 <= kt <= n_ft - nh, adjacent threads on adjacent
        // columns of one row
        for (int e = threadIdx.x; e < N * kBlockCols; e += blockDim.x) {
            const int kw = e >> 2, cc = 3 - (e & 3), kt = kt0 + cc;
            if (kt >= 1 && d.n_ft - kt >= d.nh) {
                const float2 a = s_tr[cc * TR + kw];
                dRj[(int64_t)((N - kw) % N) * d.n_ft + (d.n_ft - kt)] = make_float2(a.x, -a.y);
            }
        }
    }
}

// Adjoint part B, one warp per time frequency: for every j, conj(H_j) G^ transformed back
// along the wires, written over S_j's block of shat (the time-axis spectrum of dL/dS_j).
// The warps' transpose buffers double as the CTA's output columns ([4][ld]).
template <int M>
__global__ void __launch_bounds__(kWarps * 32, 3)
k_wire_adjoint_b(ConvDims d, const float2* __restrict__ tw2, const float2* __restrict__ g2d,
                 float2* __restrict__ shat, const float2* __restrict__ H)
{
    constexpr int N = 32 * M, LD = tile_ld(N);
    constexpr int TR = 32 * (M + 1);
    static_assert(kWarps * TR >= kBlockCols * LD, "output columns must fit the transpose space");
    __shared__ float2 s_twi[N];
    __shared__ __align__(16) float2 s_tr[kWarps * TR];
    float2* s_out = s_tr;
    load_wire_twiddles<M>(tw2, nullptr, s_twi);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int kb = blockIdx.x, c = warp;
    const int j0 = (int)((int64_t)blockIdx.y * d.n_imp / gridDim.y);
    const int j1 = (int)((int64_t)(blockIdx.y + 1) * d.n_imp / gridDim.y);
    float2* tr = s_tr + warp * TR;

    float2 g[32];
    if (lane < M) {
        const float2* gc = g2d + (int64_t)kb * N * kBlockCols + c;
#pragma unroll
        for (int k1 = 0; k1 < 32; ++k1) g[k1] = __ldg(gc + (int64_t)(lane + M * k1) * kBlockCols);
    }
    for (int j = j0; j < j1; ++j) {
        const int64_t blk = (int64_t)j * d.nkb + kb;
        float2 u[32];
        if (lane < M) {
            const float2* hj = H + (blk * kBlockCols + c) * N;   // column kt of H_j
#pragma unroll
            for (int k1 = 0; k1 < 32; ++k1) {
                const float2 h = __ldg(hj + lane + M * k1);
                u[k1] = make_float2(h.x * g[k1].x + h.y * g[k1].y, h.x * g[k1].y - h.y * g[k1].x);
            }
        }
        float2 v[M];
        warp_fft_inv<M>(u, s_twi, tr, lane, v);
        __syncthreads();                                  // every warp is done with tr
#pragma unroll
        for (int n1 = 0; n1 < M; ++n1) {
            const int w = lane + 32 * n1;
            if (w < d.n_w) s_out[c * LD + w] = v[n1];
        }
        __syncthreads();
        store_tile_cols(s_out, d.n_w, LD, shat + blk * d.n_w * kBlockCols);
        __syncthreads();                                  // s_out is read out
    }
}

template <int FIX>
__global__ void __launch_bounds__(256, FIX == kPlanRuntime ? 2 : 3)
k_rows_c2r_grid(ConvDims d, FftPlan p, const float2* __restrict__ shat, float* __restrict__ grid)
{
    extern __shared__ __align__(128) unsigned char smraw[];
    const int N = p.n;
    float2* X = reinterpret_cast<float2*>(smraw);
    float2* Y = X + padded_len(N);
    // CTA b: impact j = b / npw, wires 2 (b mod npw) and the next one.  Adjacent wires of one
    // impact read adjacent 32-byte chunks of the blocked spectra.
    const int npw = (d.n_w + 1) / 2;
    const int j = blockIdx.x / npw, w0 = 2 * (blockIdx.x % npw), w1 = w0 + 1;
    const bool has1 = w1 < d.n_w;
    const int64_t slab = (int64_t)d.nkb * d.n_w * kBlockCols;
    stage_herm_pair(shat + j * slab, shat + j * slab, w0, has1 ? w1 : w0, has1, d.n_w, d.nh, N, X);
    __syncthreads();
    const float2* z = run_row_plan<true, FIX, 256>(p, X, Y);
    float* o0 = grid + ((int64_t)w0 * d.n_imp + j) * d.n_t;
    float* o1 = grid + ((int64_t)w1 * d.n_imp + j) * d.n_t;
    const bool vec = ((d.n_t & 3) == 0) && ((reinterpret_cast<uintptr_t>(grid) & 15) == 0);
    store_real_pair(z, o0, o1, d.n_t, has1, vec);
}

// dL/dR_j(kw, kt) = conj(S_j^(kw, kt)) G^(kw, kt) / n and its Hermitian mirror (-kw, -kt)
// (as part A writes them), from the 2D spectra of S kept by the forward's wire pass (s2d,
// time-frequency major [n_imp][4 nkb][n_fw]) and G's 2D spectrum (g2d, blocked
// [nkb][n_fw][4]).  A CTA takes a tile of 32 time frequencies x 32 wire frequencies and
// loops over the impacts: each warp reads 4 columns of the tile (consecutive lanes on
// consecutive wire frequencies), the products pass through a padded shared tile, and each
// warp then writes 4 rows of dL/dR_j (32 consecutive time frequencies, 256 bytes) and the
// 4 mirrored rows (reversed, also contiguous): whole lines out, where part A writes 32-byte
// pieces 48 KB apart.  G^'s tile is read once for all impacts.
constexpr int kDrTile = 32;

__global__ void __launch_bounds__(256)
k_dr_tiles(ConvDims d, const float2* __restrict__ s2d, const float2* __restrict__ g2d,
           float2* __restrict__ dR, float inv_n)
{
    __shared__ float2 t[kDrTile][kDrTile + 1];        // [kt][kw], padded
    const int N = d.n_fw, ncol = kBlockCols * d.nkb;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int kt0 = blockIdx.x * kDrTile, kw0 = blockIdx.y * kDrTile;
    const int kw = kw0 + lane;
    // this thread's 4 elements: time frequencies kt0 + 4 warp + i, wire frequency kw
    float2 g[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int kt = kt0 + 4 * warp + i;
        g[i] = (kt < d.nh && kw < N)
                   ? __ldg(g2d + ((int64_t)(kt >> 2) * N + kw) * kBlockCols + (kt & 3))
                   : make_float2(0.f, 0.f);
    }
    // this thread's 4 values of S_j^, loaded one impact ahead
    auto load_s = [&](int j, float2 (&u)[4]) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int kt = kt0 + 4 * warp + i;
            u[i] = (kt < d.nh && kw < N) ? __ldcs(s2d + ((int64_t)j * ncol + kt) * N + kw)
                                         : make_float2(0.f, 0.f);
        }
    };
    float2 un[4];
    load_s(0, un);
    for (int j = 0; j < d.n_imp; ++j) {
        float2 u[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) u[i] = un[i];
        if (j + 1 < d.n_imp) load_s(j + 1, un);
        __syncthreads();                                // the previous impact's tile is read
#pragma unroll
        for (int i = 0; i < 4; ++i)
            t[4 * warp + i][lane] = make_float2(inv_n * (u[i].x * g[i].x + u[i].y * g[i].y),
                                                inv_n * (u[i].x * g[i].y - u[i].y * g[i].x));
        __syncthreads();
        float2* dRj = dR + (int64_t)j * N * d.n_ft;
        const int kt = kt0 + lane;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int r = 4 * warp + i, w = kw0 + r;       // row kw = w, column kt
            if (w >= N) break;
            const float2 v = t[lane][r];
            if (kt < d.nh) __stcs(dRj + (int64_t)w * d.n_ft + kt, v);
            if (kt >= 1 && kt < d.nh && d.n_ft - kt >= d.nh)
                __stcs(dRj + (int64_t)((N - w) % N) * d.n_ft + (d.n_ft - kt), make_float2(v.x, -v.y));
        }
    }
}

#define WCSIM_ADJ_M(X) X(4) X(8) X(15) X(16) X(20) X(24) X(25) X(30)

// Impact groups per frequency block for the one-warp adjoint on `slots` resident CTAs: the s
// in 1 .. 4 that minimises the transform work, (n_imp + s) / (n_imp + 1) (every group also
// transforms G), divided by the fill of the last wave of nkb s CTAs.
int adjoint_split(int nkb, int n_imp, int slots)
{
    int best = 1;
    double best_cost = 1e300;
    for (int sp = 1; sp <= 4 && sp <= n_imp; ++sp) {
        const double waves = (double)nkb * sp / slots;
        const double fill = waves / std::ceil(waves);
        const double cost = (double)(n_imp + sp) / (n_imp + 1) / fill;
        if (cost < best_cost - 1e-9) { best = sp; best_cost = cost; }
    }
    return best;
}

DeviceOnce g_attr;

}  // namespace

cudaError_t launch_wire_adjoint_warp(const ConvDims& d, const float2* tw2, const float2* gt,
                                     float2* shat, const float2* H, float2* g2d, float2* dR,
                                     float inv_n, cudaStream_t s)
{
    // impacts split over grid y: more, shorter CTAs for the same per-CTA footprint
    const int split = d.adj_split > 0 ? (d.adj_split > d.n_imp ? d.n_imp : d.adj_split)
                                      : adjoint_split(d.nkb, d.n_imp, 3 * sm_count());
    switch (d.n_fw / 32) {
#define WCSIM_CASE(MM)                                                                           \
    case MM: {                                                                                   \
        const size_t smem_a = (size_t)kBlockCols * tile_ld(32 * MM) * sizeof(float2);         \
        static DeviceOnce attr_set;                                                             \
        if (attr_set.pending()) {                                                               \
            cudaError_t e = cudaFuncSetAttribute(k_wire_adjoint_a<MM>,                          \
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize,   \
                                                 (int)smem_a);                                  \
            if (e) return e;                                                                    \
            attr_set.mark();                                                                    \
        }                                                                                       \
        const dim3 grid(d.nkb, split), grid_a(d.nkb, dR ? split : 1);                           \
        k_wire_adjoint_a<MM><<<grid_a, kWarps * 32, smem_a, s>>>(d, tw2, gt, shat, g2d, dR, inv_n); \
        k_wire_adjoint_b<MM><<<grid, kWarps * 32, 0, s>>>(d, tw2, g2d, shat, H);                \
        break;                                                                                   \
    }
        WCSIM_ADJ_M(WCSIM_CASE)
#undef WCSIM_CASE
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_dr_rows(const ConvDims& d, const float2* s2d, const float2* g2d, float2* dR,
                           float inv_n, cudaStream_t s)
{
    const dim3 grid((unsigned)((d.nh + kDrTile - 1) / kDrTile),
                    (unsigned)((d.n_fw + kDrTile - 1) / kDrTile));
    k_dr_tiles<<<grid, 256, 0, s>>>(d, s2d, g2d, dR, inv_n);
    return cudaGetLastError();
}

cudaError_t launch_rows_c2r_grid(const ConvDims& d, const FftPlan& pt, const float2* shat,
                                 float* grid, cudaStream_t s)
{
    if (g_attr.pending()) {
        cudaError_t e = cudaFuncSetAttribute(k_rows_c2r_grid<kPlanRuntime>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
        if (!e) e = cudaFuncSetAttribute(k_rows_c2r_grid<kPlan6000>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
        if (e) return e;
        g_attr.mark();
    }
    const int64_t n_ctas = (int64_t)d.n_imp * ((d.n_w + 1) / 2);
    const int fix = fixed_plan_of(pt);
    auto k = fix == kPlan6000 ? k_rows_c2r_grid<kPlan6000> : k_rows_c2r_grid<kPlanRuntime>;
    k<<<(unsigned)n_ctas, 256, row_plan_smem(fix, pt.n), s>>>(d, pt, shat, grid);
    return cudaGetLastError();
}

}  // namespace wcsim
