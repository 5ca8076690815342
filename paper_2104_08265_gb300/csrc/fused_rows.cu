// Rasterization fused into the time-axis transform of Eq. 2 (Sec. 2.1.1 "rasterization" and
// "scatter adding", followed by the FT): the grid S is never written to memory.
//
// Binning (three small launches).  k_bin_count takes every depo's drift and bin decision
// (the same FP64 decision as the plain rasterizer) and counts it into the bucket of the first
// wire its rows reach (a depo reaching over more than kSpan wires goes to one extra "wide"
// bucket); k_bin_scan turns the counts into bucket offsets; k_bin_fill writes the decisions in
// bucket order together with each depo's tick weights, laid out on 4-tick groups (slot s is
// tick 4 floor(k_lo / 4) + s, zero outside the window).
//
// Transform.  A CTA owns two grid rows of one wire, impact positions j and j + 1.  Its
// candidates are the depos of buckets w - kSpan + 1 .. w (one contiguous range) and of the
// wide bucket.  In rounds of one candidate per thread, the CTA finds the candidates whose
// window covers its rows, forms their row weights, and lists (depo, row, 4-tick group) items;
// every thread then takes items, draws the fluctuation of its four bins (the Philox block of
// the plain rasterizer: counter (tick / 4, row, depo id, plane id)) and adds the four values
// into the pair's staging buffer in shared memory.  The buffer then goes through the
// time-axis FFT in place, and the two half spectra are stored as the plain transform stores
// them.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "depo_common.cuh"
#include "fft_engine.cuh"
#include "rng.cuh"
#include "wcsim_internal.cuh"

namespace wcsim {
namespace {

constexpr int kBinThreads = 256;
constexpr int kFusedThreads = 256;
constexpr int kScanThreads = 1024;

__device__ __forceinline__ int bucket_of(const Decision& r, int n_imp, int n_w)
{
    const int wlo = r.r_lo / n_imp, whi = r.r_hi / n_imp;
    return (whi - wlo < kFusedSpan) ? wlo : n_w;
}

__global__ void __launch_bounds__(kBinThreads)
k_bin_count(RasterConsts c, DepoArrays d, int n_imp, int n_w, Decision* __restrict__ dec,
            int32_t* __restrict__ pos, int32_t* __restrict__ cnt, int* flags)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= d.n) return;
    Decision r = decide(c, d, i, flags, true);
    const bool take = r.ok && r.qatt > 0.0f;         // a depo that adds nothing is not binned
    const int b = take ? bucket_of(r, n_imp, n_w) : -1;
    // neighbouring depos of a track mostly share a bucket: one atomic per bucket per warp
    const unsigned active = __activemask();
    const unsigned same = __match_any_sync(active, b);
    const int leader = __ffs(same) - 1;
    const int lane = threadIdx.x & 31;
    int32_t base = 0;
    if (take && lane == leader) base = atomicAdd(cnt + b, __popc(same));
    base = __shfl_sync(active, base, leader);
    int32_t p = -1;
    if (take) {
        r.id = d.id[i];
        p = base + __popc(same & ((1u << lane) - 1u));
        dec[i] = r;
    }
    pos[i] = p;
}

// Exclusive prefix of cnt[0 .. nb) into off[0 .. nb] (off[nb] = total); cnt is left zero for
// the next call.  One CTA of kScanThreads threads, each owning a contiguous run of buckets.
__global__ void __launch_bounds__(kScanThreads)
k_bin_scan(int32_t* __restrict__ cnt, int32_t* __restrict__ off, int nb)
{
    __shared__ int32_t s_warp[kScanThreads / 32];
    const int per = (nb + kScanThreads - 1) / kScanThreads;
    const int b0 = threadIdx.x * per, b1 = min(nb, b0 + per);
    int32_t sum = 0;
    for (int b = b0; b < b1; ++b) sum += cnt[b];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int32_t incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int32_t v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int32_t v = s_warp[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t u = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += u;
        }
        s_warp[lane] = v;                    // inclusive over warps
    }
    __syncthreads();
    int32_t run = incl - sum + (warp > 0 ? s_warp[warp - 1] : 0);
    for (int b = b0; b < b1; ++b) {
        off[b] = run;
        run += cnt[b];
        cnt[b] = 0;
    }
    if (threadIdx.x == kScanThreads - 1) off[nb] = s_warp[kScanThreads / 32 - 1];
}

// Decisions in bucket order, and the tick weights of each on 4-tick groups (when its window
// spans at most kFusedSlots / 4 groups; wider windows are weighted by the transform itself).
__global__ void __launch_bounds__(kBinThreads)
k_bin_fill(RasterConsts c, int64_t n, int64_t cap, int n_imp, int n_w,
           const Decision* __restrict__ dec,
           const int32_t* __restrict__ pos, const int32_t* __restrict__ off,
           Decision* __restrict__ sorted, float* __restrict__ wts)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int32_t p = pos[i];
    if (p < 0) return;
    const Decision r = dec[i];
    const int64_t k = (int64_t)off[bucket_of(r, n_imp, n_w)] + p;
    if (k >= cap) return;                      // never with consistent counts
    sorted[k] = r;
    const int q_lo = r.k_lo >> 2, ng = (r.k_hi >> 2) - q_lo + 1;
    if (ng > kFusedSlots / 4) return;
    const float s_t = (r.st > 0.0f) ? c.dt_f / (1.41421356237309505f * r.st) : 0.0f;
    float4* out = reinterpret_cast<float4*>(wts + k * kFusedSlots);
    float ea = 0.0f;
    if (r.st > 0.0f) ea = edge_erfc((int64_t)r.k_lo - r.i0t, r.frac_t, s_t);
    for (int g = 0; g < kFusedSlots / 4; ++g) {
        float w[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int kk = 4 * (q_lo + g) + e;
            w[e] = 0.0f;
            if (kk >= r.k_lo && kk <= r.k_hi) {
                if (r.st > 0.0f) {
                    const float eb = edge_erfc((int64_t)(kk + 1) - r.i0t, r.frac_t, s_t);
                    w[e] = bin_mass((int64_t)kk - r.i0t, r.frac_t, s_t, ea, eb);
                    ea = eb;
                } else {
                    w[e] = 1.0f;
                }
            }
        }
        out[g] = make_float4(w[0], w[1], w[2], w[3]);
    }
}

// Mass of bin `kk` of an axis (offset from the floor of the position in bins: kk - i0) with
// both edge terms computed here.
__device__ __forceinline__ float bin_mass_direct(int64_t koff, float frac, float s)
{
    return bin_mass(koff, frac, s, edge_erfc(koff, frac, s), edge_erfc(koff + 1, frac, s));
}

// Store the half spectra of the two rows of wire w held in z (row 0 in .x, row 1 in .y after
// the real-pair split) at impact positions s0 and s0 + 1 of the blocked layout
// [n_imp][nkb][n_w][4] (zeros for the padding columns, or everywhere when `zero`).
__device__ __forceinline__ void store_wire_pair(const ConvDims& d, const float2* z, int N, int w,
                                                int s0, bool has1, float2* shat, bool zero)
{
    const int nk = d.nkb * kBlockCols, nh = d.nh;
    const int k0 = threadIdx.x;
    const int64_t row = (int64_t)d.n_w * kBlockCols;
    const int64_t slice = (int64_t)d.nkb * row;
    const int64_t step = (int64_t)(blockDim.x / kBlockCols) * row;
    float2* q0 = shat + (int64_t)s0 * slice + (k0 >> 2) * row + w * kBlockCols + (k0 & 3);
    float2* q1 = q0 + slice;
    const int dp = blockDim.x + (blockDim.x >> 4);
    int pa = pad16(k0), pb = pad16(N - k0);
    for (int k = k0; k < nk; k += blockDim.x, q0 += step, q1 += step, pa += dp, pb -= dp) {
        float2 x0 = make_float2(0.f, 0.f), x1 = x0;
        if (k < nh && !zero) {
            const float2 u = z[pa];
            const float2 v = z[k == 0 ? 0 : pb];
            x0 = make_float2(0.5f * (u.x + v.x), 0.5f * (u.y - v.y));
            x1 = make_float2(0.5f * (u.y + v.y), 0.5f * (v.x - u.x));
        }
        *q0 = x0;
        if (has1) *q1 = x1;
    }
}

// One CTA per (wire, pair of impact positions j, j + 1; the last of an odd count alone).
// FIX: compile-time plan variant.
template <int FIX>
__global__ void __launch_bounds__(kFusedThreads, FIX == kPlanRuntime ? 2 : 3)
k_rows_r2c_fused(ConvDims d, FftPlan p, RasterConsts c, FusedBins b, float2* __restrict__ shat)
{
    extern __shared__ __align__(128) unsigned char smraw[];
    constexpr int T = kFusedThreads;
    const int N = p.n;
    float2* X = reinterpret_cast<float2*>(smraw);
    float2* Y = X + padded_len(N);
    float* zf = reinterpret_cast<float*>(X);          // tick k: row 0 at 2k, row 1 at 2k + 1
    // one round of candidates: the hits, their row weights and item prefix
    __shared__ int32_t s_base[T + 1];
    __shared__ int32_t s_rec[T], s_klo[T];
    __shared__ float s_w[2][T], s_invq[T];
    __shared__ uint32_t s_id[T];
    __shared__ int32_t s_ng[T];
    __shared__ uint8_t s_rows[T];
    __shared__ int32_t s_warp[T / 32];

    const int npj = (d.n_imp + 1) >> 1;
    const int w = blockIdx.x / npj, jp = blockIdx.x - w * npj;
    const int ja = 2 * jp;
    const bool has1 = ja + 1 < d.n_imp;
    const int64_t r0 = (int64_t)w * d.n_imp + ja, r1 = r0 + 1;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

    float4* X4 = reinterpret_cast<float4*>(X);
    for (int i = threadIdx.x; i < (N + 1) / 2; i += T) X4[i] = make_float4(0.f, 0.f, 0.f, 0.f);

    const int32_t c0 = __ldg(b.off + max(0, w - kFusedSpan + 1)), c1 = __ldg(b.off + w + 1);
    const int32_t wd0 = __ldg(b.off + b.n_w), wd1 = __ldg(b.off + b.n_w + 1);
    // (ranges past the scratch capacity never occur with consistent counts; clipped anyway)
    const int32_t cap = (int32_t)min((int64_t)b.cap, (int64_t)INT32_MAX);
    const int32_t n_near = max(0, min(c1, cap) - c0);
    const int32_t n_cand = n_near + max(0, min(wd1, cap) - wd0);
    bool any = false;
    __syncthreads();                                   // buffer cleared
    for (int base = 0; base < n_cand; base += T) {
        const int ci = base + threadIdx.x;
        int items = 0, ng = 0, rows = 0;
        int32_t rec = 0;
        if (ci < n_cand) {
            rec = ci < n_near ? c0 + ci : wd0 + (ci - n_near);
            const Decision* dp = b.sorted + rec;
            const int4 win = *reinterpret_cast<const int4*>(&dp->ok);    // ok, r_lo, r_hi, k_lo
            const bool h0 = win.y <= r0 && r0 <= win.z;
            const bool h1 = has1 && win.y <= r1 && r1 <= win.z;
            if (h0 || h1) {
                const Decision dd = *dp;
                const float s_p = (dd.sp > 0.0f) ? c.dp_f / (1.41421356237309505f * dd.sp) : 0.0f;
                float w0 = 0.0f, w1 = 0.0f;
                if (dd.sp > 0.0f) {
                    // the edges of rows r0, r0 + 1: three erfc terms for both rows
                    const int64_t o0 = r0 - dd.i0p;
                    const float e0 = edge_erfc(o0, dd.frac_p, s_p);
                    const float e1 = edge_erfc(o0 + 1, dd.frac_p, s_p);
                    if (h0) w0 = dd.qw * bin_mass(o0, dd.frac_p, s_p, e0, e1);
                    if (h1) w1 = dd.qw * bin_mass(o0 + 1, dd.frac_p, s_p, e1,
                                                  edge_erfc(o0 + 2, dd.frac_p, s_p));
                } else {
                    w0 = h0 ? dd.qw : 0.0f;
                    w1 = h1 ? dd.qw : 0.0f;
                }
                ng = (dd.k_hi >> 2) - (dd.k_lo >> 2) + 1;
                rows = (h0 ? 1 : 0) | (h1 ? 2 : 0);
                items = ((h0 ? 1 : 0) + (h1 ? 1 : 0)) * ng;
                s_w[0][threadIdx.x] = w0;
                s_w[1][threadIdx.x] = w1;
                s_klo[threadIdx.x] = dd.k_lo;
                s_invq[threadIdx.x] = 1.0f / dd.qatt;
                s_id[threadIdx.x] = dd.id;
            }
        }
        // exclusive prefix of the item counts over the block
        int32_t incl = items;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        if (lane == 31) s_warp[warp] = incl;
        s_rec[threadIdx.x] = rec;
        s_ng[threadIdx.x] = ng;
        s_rows[threadIdx.x] = (uint8_t)rows;
        __syncthreads();
        int32_t before = 0, total = 0;
#pragma unroll
        for (int k = 0; k < T / 32; ++k) {
            const int32_t v = s_warp[k];
            before += (k < warp) ? v : 0;
            total += v;
        }
        s_base[threadIdx.x] = before + incl - items;
        if (threadIdx.x == 0) s_base[T] = total;
        __syncthreads();
        any |= total > 0;
        for (int it = threadIdx.x; it < total; it += T) {
            // the hit holding item `it`: the last h with s_base[h] <= it
            int lo = 0, hi = T - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (s_base[mid] <= it) lo = mid;
                else hi = mid - 1;
            }
            const int h = lo;
            const int local = it - s_base[h];
            const int ngh = s_ng[h];
            const int rm = s_rows[h];
            const int rsel = (local >= ngh) ? 1 : 0;
            const int g = local - rsel * ngh;
            const int row = (rm == 3) ? rsel : (rm == 1 ? 0 : 1);
            const float wr = s_w[row][h];
            const int32_t rec_h = s_rec[h];
            const int q = (s_klo[h] >> 2) + g;
            float4 wt;
            if (ngh <= kFusedSlots / 4) {
                wt = __ldg(reinterpret_cast<const float4*>(b.wts + (int64_t)rec_h * kFusedSlots) + g);
            } else {
                // a window wider than the stored slots: its tick weights are formed here
                const Decision* dp = b.sorted + rec_h;
                const int64_t i0t = dp->i0t;
                const int k_lo = dp->k_lo, k_hi = dp->k_hi;
                const float frac_t = dp->frac_t, st = dp->st;
                const float s_t = (st > 0.0f) ? c.dt_f / (1.41421356237309505f * st) : 0.0f;
                float v4[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int kk = 4 * q + e;
                    v4[e] = 0.0f;
                    if (kk >= k_lo && kk <= k_hi)
                        v4[e] = (st > 0.0f) ? bin_mass_direct((int64_t)kk - i0t, frac_t, s_t) : 1.0f;
                }
                wt = make_float4(v4[0], v4[1], v4[2], v4[3]);
            }
            float v[4] = {wr * wt.x, wr * wt.y, wr * wt.z, wr * wt.w};
            if (c.fluctuate == 1) {
                // normal approximation to Binomial(Q', mean / Q'); zero-mean bins stay zero
                float z[4];
                box_muller4(philox(make_uint4((uint32_t)q, (uint32_t)(row ? r1 : r0), s_id[h],
                                              c.plane_id), c.key0, c.key1), z);
                const float inv_q = s_invq[h];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const float var = v[e] * (1.0f - v[e] * inv_q);
                    v[e] = fmaxf(0.0f, fmaf(sqrt_fast(var), z[e], v[e]));
                }
            }
#pragma unroll
            for (int e = 0; e < 4; ++e)
                if (v[e] != 0.0f && 4 * q + e < d.n_t) atomicAdd(zf + 2 * (4 * q + e) + row, v[e]);
        }
        __syncthreads();                               // the hit list is refilled next round
    }
    const int s0 = ja;
    if (!any) {                                        // nothing deposited: zero spectra
        store_wire_pair(d, X, N, w, s0, has1, shat, true);
        return;
    }
    const float2* z = run_row_plan<false, FIX, T>(p, X, Y);
    store_wire_pair(d, z, N, w, s0, has1, shat, false);
}

// Largest dynamic shared memory a launch of kernel k may ask for on the current device: the
// opt-in limit per block less the kernel's static shared memory.
template <class K>
cudaError_t max_dynamic_smem(K k, int* out)
{
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (!e) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes a;
    if (!e) e = cudaFuncGetAttributes(&a, k);
    if (!e) *out = optin - (int)a.sharedSizeBytes;
    return e;
}

DeviceOnce g_attr;
cudaError_t attrs()
{
    if (!g_attr.pending()) return cudaSuccess;
    int m0 = 0, m1 = 0;
    cudaError_t e = max_dynamic_smem(k_rows_r2c_fused<kPlanRuntime>, &m0);
    if (!e) e = max_dynamic_smem(k_rows_r2c_fused<kPlan6000>, &m1);
    if (!e) e = cudaFuncSetAttribute(k_rows_r2c_fused<kPlanRuntime>, cudaFuncAttributeMaxDynamicSharedMemorySize, m0);
    if (!e) e = cudaFuncSetAttribute(k_rows_r2c_fused<kPlan6000>, cudaFuncAttributeMaxDynamicSharedMemorySize, m1);
    if (!e) g_attr.mark();
    return e;
}

}  // namespace

bool fused_supported(const FftPlan& pt)
{
    const int fix = fixed_plan_of(pt);
    int mx = 0;
    if (max_dynamic_smem(fix == kPlan6000 ? k_rows_r2c_fused<kPlan6000>
                                          : k_rows_r2c_fused<kPlanRuntime>, &mx) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return row_plan_smem(fix, pt.n) <= (size_t)mx;
}

cudaError_t launch_bin_depos(const RasterConsts& c, const DepoArrays& d, int n_imp, int n_w,
                             const FusedScratch& s, int* flags, cudaStream_t st)
{
    if (d.n <= 0) return cudaMemsetAsync(s.off, 0, (size_t)(n_w + 2) * sizeof(int32_t), st);
    const unsigned blocks = (unsigned)((d.n + kBinThreads - 1) / kBinThreads);
    k_bin_count<<<blocks, kBinThreads, 0, st>>>(c, d, n_imp, n_w, s.dec, s.pos, s.cnt, flags);
    k_bin_scan<<<1, kScanThreads, 0, st>>>(s.cnt, s.off, n_w + 1);
    k_bin_fill<<<blocks, kBinThreads, 0, st>>>(c, d.n, s.cap, n_imp, n_w, s.dec, s.pos, s.off,
                                               s.sorted, s.wts);
    return cudaGetLastError();
}

cudaError_t launch_rows_r2c_fused(const ConvDims& d, const FftPlan& pt, const RasterConsts& c,
                                  const FusedScratch& s, float2* shat, cudaStream_t st)
{
    cudaError_t e = attrs();
    if (e) return e;
    FusedBins b;
    b.sorted = s.sorted;
    b.wts = s.wts;
    b.off = s.off;
    b.n_w = d.n_w;
    b.cap = s.cap;
    const int npj = (d.n_imp + 1) / 2;
    const unsigned blocks = (unsigned)(d.n_w * npj);
    const int fix = fixed_plan_of(pt);
    auto k = fix == kPlan6000 ? k_rows_r2c_fused<kPlan6000> : k_rows_r2c_fused<kPlanRuntime>;
    k<<<blocks, kFusedThreads, row_plan_smem(fix, pt.n), st>>>(d, pt, c, b, shat);
    return cudaGetLastError();
}

}  // namespace wcsim
