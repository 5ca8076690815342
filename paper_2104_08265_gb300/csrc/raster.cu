// Drift, rasterization, fluctuation and scatter-add of depos into the impact x tick grid
// (Sec. 2.1.1 "rasterization" and "scatter adding"; drift and diffusion as in Fig. 2;
// fluctuation with a Box-Muller normal as in Sec. 3.3.1).
//
// Work split.  A warp owns 32 consecutive depos.  First every lane takes the FP64 bin
// decision of its own depo (one thread per depo: FP64 is scarce on this part, so it is
// never evaluated redundantly by a whole warp).  Then the warp walks its 32 depos one by
// one: lanes compute the per-bin 1D weights of the depo's patch into shared memory (FP32
// erf/erfc of bin-edge offsets), then stride over the patch bins, form the value
// Q' * w_p * w_t (optionally fluctuated) and add it into the grid with a fire-and-forget
// global reduction.  Adjacent lanes take adjacent ticks of a row, so the reductions of a
// warp land in a few contiguous sectors.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "wcsim_internal.cuh"

namespace wcsim {
namespace {

constexpr int kWarps = 8;       // warps per block
constexpr int kWmax = 64;       // weights per axis held per patch tile

struct Decision {
    int32_t ok;                 // covers >= 1 bin and carries charge
    int32_t r_lo, r_hi, k_lo, k_hi;
    int64_t i0p, i0t;           // floor of the depo position in bin units
    float frac_p, frac_t;       // position - floor, FP32
    float sp, st;               // sigma_T [mm], sigma_t [us] (FP32)
    float qatt;                 // Q' = Q exp(-t_d / lifetime)
};

// One axis of the bin decision.  Every operation is an explicitly rounded IEEE operation
// (no contraction), so that the result is a function of the inputs alone.
__device__ __forceinline__ bool axis_window(double x, float hw, int64_t n, int32_t& lo,
                                            int32_t& hi, int64_t& i0i, float& frac)
{
    if (!(x > -1e12 && x < 1e12)) return false;
    double i0 = floor(x);
    frac = __double2float_rn(__dsub_rn(x, i0));
    float a = __fsub_rn(frac, hw);
    float b = __fadd_rn(frac, hw);
    double l = __dadd_rn(i0, floor((double)a));
    double h = __dadd_rn(i0, floor((double)b));
    if (l < 0.0) l = 0.0;
    if (h > (double)(n - 1)) h = (double)(n - 1);
    if (l > h) return false;
    lo = (int32_t)l;
    hi = (int32_t)h;
    i0i = (int64_t)i0;
    return true;
}

// Drift (t_a = t + t_d, Q' = Q e^{-t_d/tau}, sigma = sqrt(2 D t_d)) and the window of bins
// whose span meets [mu - n sigma, mu + n sigma], clipped to the grid.
__device__ __forceinline__ Decision decide(const RasterConsts& c, const DepoArrays& d,
                                           int64_t i, int* flags)
{
    Decision r;
    r.ok = 0;
    const double p = d.p[i], t = d.t[i], td = d.td[i];
    const float q = d.q[i];
    if (!(td >= 0.0) || !isfinite(p) || !isfinite(t) || !isfinite(td) || !(q >= 0.0f) ||
        !isfinite(q)) {
        atomicOr(flags, 1);
        return r;
    }
    if (!(q > 0.0f)) return r;
    const float td_f = __double2float_rn(td);
    r.sp = __fsqrt_rn(__fmul_rn(c.two_dt, td_f));
    r.st = __fmul_rn(__fsqrt_rn(__fmul_rn(c.two_dl, td_f)), c.inv_v);
    const float hw_p = __fmul_rn(__fmul_rn(c.nsig, r.sp), c.inv_dp_f);
    const float hw_t = __fmul_rn(__fmul_rn(c.nsig, r.st), c.inv_dt_f);
    const double ta = __dadd_rn(t, td);
    const double xp = __dmul_rn(__dsub_rn(p, c.p0), c.inv_dp);
    const double xt = __dmul_rn(__dsub_rn(ta, c.t0), c.inv_dt);
    if (!axis_window(xp, hw_p, c.n_rows, r.r_lo, r.r_hi, r.i0p, r.frac_p)) return r;
    if (!axis_window(xt, hw_t, c.n_ticks, r.k_lo, r.k_hi, r.i0t, r.frac_t)) return r;
    r.qatt = q * expf(-td_f * c.inv_tau);
    r.ok = 1;
    return r;
}

// Gaussian mass of bin k: Phi(b) - Phi(a), in units where u = offset / (sqrt(2) sigma);
// the erfc forms keep relative precision in the tails.  koff = k - floor(position).
__device__ __forceinline__ float bin_weight(int64_t koff, float frac, float s)
{
    const float ua = ((float)koff - frac) * s;
    const float ub = ((float)(koff + 1) - frac) * s;
    if (ua >= 0.0f) return 0.5f * (erfcf(ua) - erfcf(ub));
    if (ub <= 0.0f) return 0.5f * (erfcf(-ub) - erfcf(-ua));
    return 0.5f * (erff(ub) - erff(ua));
}

// Philox4x32-10 (Salmon et al., SC'11): 10 rounds of the multiply-xor bijection with a
// Weyl-sequence key schedule.
__device__ __forceinline__ uint4 philox(uint4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int i = 0; i < 10; ++i) {
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// Standard normal from two 32-bit words (Box & Muller 1958), u = (x + 1/2) 2^-32.
__device__ __forceinline__ float box_muller(uint32_t x0, uint32_t x1)
{
    const float u1 = fmaf((float)x0, 2.3283064365386963e-10f, 1.1641532182693481e-10f);
    const float u2 = fmaf((float)x1, 2.3283064365386963e-10f, 1.1641532182693481e-10f);
    return sqrtf(-2.0f * logf(u1)) * cospif(2.0f * u2);
}

__global__ void __launch_bounds__(kWarps * 32)
k_rasterize(RasterConsts c, DepoArrays d, float* __restrict__ grid, int* flags)
{
    __shared__ float s_wp[kWarps][kWmax];
    __shared__ float s_wt[kWarps][kWmax];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t base = ((int64_t)blockIdx.x * kWarps + warp) * 32;
    if (base >= d.n) return;

    Decision me;
    me.ok = 0;
    uint32_t my_id = 0;
    if (base + lane < d.n) {
        me = decide(c, d, base + lane, flags);
        my_id = d.id[base + lane];
    }
    unsigned todo = __ballot_sync(0xffffffffu, me.ok != 0);
    float* wp = s_wp[warp];
    float* wt = s_wt[warp];

    while (todo) {
        const int src = __ffs(todo) - 1;
        todo &= todo - 1;
        const int32_t r_lo = __shfl_sync(0xffffffffu, me.r_lo, src);
        const int32_t r_hi = __shfl_sync(0xffffffffu, me.r_hi, src);
        const int32_t k_lo = __shfl_sync(0xffffffffu, me.k_lo, src);
        const int32_t k_hi = __shfl_sync(0xffffffffu, me.k_hi, src);
        const int64_t i0p = __shfl_sync(0xffffffffu, me.i0p, src);
        const int64_t i0t = __shfl_sync(0xffffffffu, me.i0t, src);
        const float frac_p = __shfl_sync(0xffffffffu, me.frac_p, src);
        const float frac_t = __shfl_sync(0xffffffffu, me.frac_t, src);
        const float sp = __shfl_sync(0xffffffffu, me.sp, src);
        const float st = __shfl_sync(0xffffffffu, me.st, src);
        const float qatt = __shfl_sync(0xffffffffu, me.qatt, src);
        const uint32_t id = __shfl_sync(0xffffffffu, my_id, src);
        if (!(qatt > 0.0f)) continue;      // Q' underflowed: nothing to add
        // u = offset_in_bins * bin / (sqrt(2) sigma); sigma == 0 puts all weight in the
        // single bin of the window.
        const float s_p = (sp > 0.0f) ? c.dp_f / (1.41421356237309505f * sp) : 0.0f;
        const float s_t = (st > 0.0f) ? c.dt_f / (1.41421356237309505f * st) : 0.0f;

        for (int32_t r0 = r_lo; r0 <= r_hi; r0 += kWmax) {
            const int nr = min(kWmax, r_hi - r0 + 1);
            for (int32_t k0 = k_lo; k0 <= k_hi; k0 += kWmax) {
                const int nt = min(kWmax, k_hi - k0 + 1);
                for (int e = lane; e < nr; e += 32)
                    wp[e] = qatt * ((sp > 0.0f) ? bin_weight((int64_t)(r0 + e) - i0p, frac_p, s_p)
                                                : 1.0f);
                for (int e = lane; e < nt; e += 32)
                    wt[e] = (st > 0.0f) ? bin_weight((int64_t)(k0 + e) - i0t, frac_t, s_t) : 1.0f;
                __syncwarp();
                const float inv_nt = 1.0f / (float)nt;
                for (int b = lane; b < nr * nt; b += 32) {
                    const int ir = (int)(((float)b + 0.5f) * inv_nt);
                    const int ik = b - ir * nt;
                    const int64_t r = r0 + ir;
                    const int32_t k = k0 + ik;
                    float val = wp[ir] * wt[ik];
                    if (c.fluctuate) {
                        // normal approximation to Binomial(Q', mean / Q')
                        const uint4 x = philox(make_uint4((uint32_t)k, (uint32_t)r, id, c.plane_id),
                                               c.key0, c.key1);
                        const float z = box_muller(x.x, x.y);
                        const float var = fmaxf(0.0f, val * (1.0f - val / qatt));
                        val = fmaxf(0.0f, val + sqrtf(var) * z);
                    }
                    atomicAdd(grid + r * c.n_ticks + k, val);
                }
                __syncwarp();
            }
        }
    }
}

__global__ void k_windows(RasterConsts c, DepoArrays d, int32_t* __restrict__ out, int* flags)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= d.n) return;
    Decision r = decide(c, d, i, flags);
    int4 v = r.ok ? make_int4(r.r_lo, r.r_hi, r.k_lo, r.k_hi) : make_int4(-1, -1, -1, -1);
    reinterpret_cast<int4*>(out)[i] = v;
}

}  // namespace

cudaError_t launch_rasterize(const RasterConsts& c, const DepoArrays& d, float* grid,
                             int* flags, cudaStream_t s)
{
    if (d.n <= 0) return cudaSuccess;
    const int64_t per_block = kWarps * 32;
    const int64_t blocks = (d.n + per_block - 1) / per_block;
    k_rasterize<<<(unsigned)blocks, kWarps * 32, 0, s>>>(c, d, grid, flags);
    return cudaGetLastError();
}

cudaError_t launch_windows(const RasterConsts& c, const DepoArrays& d, int32_t* out,
                           int* flags, cudaStream_t s)
{
    if (d.n <= 0) return cudaSuccess;
    const int64_t blocks = (d.n + 255) / 256;
    k_windows<<<(unsigned)blocks, 256, 0, s>>>(c, d, out, flags);
    return cudaGetLastError();
}

}  // namespace wcsim
