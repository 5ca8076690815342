// Drift, rasterization, fluctuation and scatter-add of depos into the impact x tick grid
// (Sec. 2.1.1 "rasterization" and "scatter adding"; drift and diffusion as in Fig. 2;
// fluctuation with a Box-Muller normal as in Sec. 4.3.1).
//
// Work split.  A block of 8 warps owns KD consecutive depos (32 by default; 64 or 128 when
// the autotuner finds them faster; the adjoint uses 64).  Threads 0..KD-1 take the FP64 bin
// decision of one depo each (one thread per depo: FP64 is scarce on this part, so it is
// never evaluated redundantly by a whole warp) and park it in shared memory.  Each group of
// 8 lanes then walks KD / 32 of the block's depos (the four groups of a warp work on four
// depos side by side): its lanes compute one erfc per bin edge of the patch (rows and ticks
// together), difference them into the per-bin 1D weights in shared memory and stride over
// (row, 4-tick group) items.
// An item draws one Philox block for its four ticks when fluctuating (four Box-Muller
// normals), forms Q' w_p w_t per bin and adds the four values into the grid with one
// vector reduction.  The exact binomial fluctuation (an instance of its own) strides over
// single bins instead: each draw walks its bin's CDF, and neighbouring ticks, whose walks
// cost alike, then run side by side in a group.  With renormalisation the weights of each
// axis are divided by the mass of its unclipped n-sigma window (folded into the per-depo
// scale of the decision).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "binomial.cuh"
#include "depo_common.cuh"
#include "rng.cuh"
#include "wcsim_internal.cuh"

namespace wcsim {
namespace {

constexpr int kWarps = 8;       // warps per block
constexpr int kDepos = 64;      // depos per block
constexpr int kWmax = 64;       // weights per axis held per patch tile

// Exact binomial fluctuation of the bin (row r, tick k) with mean v: x ~ Binomial(N, p) with
// N = rint(Q') whole electrons and p = v / Q', drawn by inversion at the 23-bit uniform of
// word k mod 4 of the bin's Philox block (the block the normal approximation uses).  A bin
// whose variance N p (1 - p) exceeds 65536, or N above 2^24, takes the normal
// approximation instead.
__device__ __forceinline__ float binomial_bin(const RasterConsts& c, const Decision& dd, int k,
                                              int64_t r, float v, float inv_q, const float* stirl)
{
    const uint4 x = philox(make_uint4((uint32_t)(k >> 2), (uint32_t)r, dd.id, c.plane_id),
                           c.key0, c.key1);
    const int e = k & 3;
    const float n = rintf(dd.qatt);
    const float p = fminf(1.0f, v * inv_q);
    if (n > 16777216.0f || n * p * (1.0f - p) > 65536.0f) {
        float z[4];
        box_muller4(x, z);
        const float ze = e == 0 ? z[0] : e == 1 ? z[1] : e == 2 ? z[2] : z[3];
        const float var = v * (1.0f - v * inv_q);
        return fmaxf(0.0f, fmaf(sqrt_fast(var), ze, v));
    }
    if (n == 0.0f) return 0.0f;
    if (p >= 1.0f) return n;
    const uint32_t w = e == 0 ? x.x : e == 1 ? x.y : e == 2 ? x.z : x.w;
    return binomial_inverse(n, p, uniform23(w), stirl);
}

// The rasterization tiles (KD depos per CTA, G lanes per depo) the autotuner chooses from.
// With G = 8 the four groups of a warp work on four depos side by side (a patch of ~17 rows x
// 3 four-tick groups, ~47 items, fills six rounds of 8 lanes); with G = 32 a warp takes one
// depo at a time (two rounds, but no groups diverging inside the warp).
#define WCSIM_RASTER_TILES(X) X(32, 8) X(64, 8) X(128, 8) X(256, 8) X(64, 16) X(128, 16) \
    X(256, 16) X(64, 32) X(128, 32) X(256, 32)

// The depos [blk * KD, blk * KD + KD) of one event, by one CTA of kWarps warps, G lanes per
// depo.  BIN: the exact binomial fluctuation (an instance of its own, so that the other
// modes keep their registers).
template <int KD, int G, bool BIN>
__device__ __forceinline__ void rasterize_block(const RasterConsts& c, const DepoArrays& d,
                                                float* __restrict__ grid, int* flags, int64_t blk)
{
    static_assert(KD <= kWarps * 32, "one deciding thread per depo");
    static_assert(G == 8 || G == 16 || G == 32, "lanes per depo");
    constexpr int NG = kWarps * 32 / G;
    __shared__ Decision s_dec[KD];
    __shared__ float s_wp[NG][kWmax];
    // tick weights of a tile laid out on 4-tick groups: slot p is tick 4 q_lo + p (zero
    // outside the window), so that an item reads its four weights with one 16-byte load
    __shared__ __align__(16) float s_wt[NG][kWmax + 8];
    __shared__ float s_edge[NG][2 * (kWmax + 1)];        // row edges, then tick edges
    __shared__ float s_stirl[BIN ? 16 : 1];              // the binomial's small-count table
    if (BIN && threadIdx.x == 0) {
#pragma unroll
        for (int m = 0; m < 16; ++m) s_stirl[m] = c.stirl[m];    // constant indices: no local copy
    }
    const int gl = threadIdx.x % G, grp = threadIdx.x / G;
    // the lanes of this group within its warp
    const unsigned gmask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << ((threadIdx.x & 31) & ~(G - 1)));
    const int64_t base = blk * KD;
    if (threadIdx.x < KD) {
        Decision r;
        r.ok = 0;
        const int64_t i = base + threadIdx.x;
        if (i < d.n) {
            r = decide(c, d, i, flags, true);
            r.id = d.id[i];
        }
        s_dec[threadIdx.x] = r;
    }
    __syncthreads();
    // 16-byte reductions need 4-tick groups to start on 16-byte boundaries
    const bool vec4 = ((c.n_ticks & 3) == 0) && ((reinterpret_cast<uintptr_t>(grid) & 15) == 0);
    float* wp = s_wp[grp];
    float* wt = s_wt[grp];
    float* ed = s_edge[grp];

    for (int i = grp; i < KD; i += NG) {
        const Decision dd = s_dec[i];
        if (!dd.ok || !(dd.qatt > 0.0f)) continue;    // nothing, or Q' underflowed
        // u = offset_in_bins * bin / (sqrt(2) sigma); sigma == 0 puts all weight in the
        // single bin of the window.
        const float s_p = (dd.sp > 0.0f) ? c.dp_f / (1.41421356237309505f * dd.sp) : 0.0f;
        const float s_t = (dd.st > 0.0f) ? c.dt_f / (1.41421356237309505f * dd.st) : 0.0f;
        const float inv_q = 1.0f / dd.qatt;

        for (int32_t r0 = dd.r_lo; r0 <= dd.r_hi; r0 += kWmax) {
            const int nr = min(kWmax, dd.r_hi - r0 + 1);
            for (int32_t k0 = dd.k_lo; k0 <= dd.k_hi; k0 += kWmax) {
                const int nt = min(kWmax, dd.k_hi - k0 + 1);
                // one erfc per bin edge: nr + 1 row edges and nt + 1 tick edges
                for (int e = gl; e < nr + nt + 2; e += G) {
                    float v;
                    if (e <= nr) v = edge_erfc((int64_t)(r0 + e) - dd.i0p, dd.frac_p, s_p);
                    else v = edge_erfc((int64_t)(k0 + e - nr - 1) - dd.i0t, dd.frac_t, s_t);
                    ed[e] = v;
                }
                const int q_lo = k0 >> 2, q_hi = (k0 + nt - 1) >> 2;
                const int nq = q_hi - q_lo + 1;
                const int koff = k0 - 4 * q_lo;            // slot of tick k0
                __syncwarp(gmask);
                for (int e = gl; e < nr + 4 * nq; e += G) {
                    if (e < nr) {
                        wp[e] = dd.qw * ((dd.sp > 0.0f)
                                    ? bin_mass((int64_t)(r0 + e) - dd.i0p, dd.frac_p, s_p, ed[e], ed[e + 1])
                                    : 1.0f);
                    } else {
                        const int k = e - nr - koff;
                        float w = 0.0f;
                        if (k >= 0 && k < nt)
                            w = (dd.st > 0.0f) ? bin_mass((int64_t)(k0 + k) - dd.i0t, dd.frac_t, s_t,
                                                          ed[nr + 1 + k], ed[nr + 2 + k])
                                               : 1.0f;
                        wt[e - nr] = w;
                    }
                }
                __syncwarp(gmask);
                if constexpr (BIN) {
                    // one bin per lane: neighbouring ticks cost alike, so the group's lanes
                    // walk their CDFs side by side, and no lane chains four draws
                    const float inv_nt = 1.0f / (float)nt;
                    for (int b = gl; b < nr * nt; b += G) {
                        const int ir = (int)(((float)b + 0.5f) * inv_nt);
                        const int ik = b - ir * nt;
                        const int64_t r = r0 + ir;
                        const float v = wp[ir] * wt[ik + koff];
                        if (!(v > 0.0f)) continue;
                        atomicAdd(grid + r * c.n_ticks + (k0 + ik),
                                  binomial_bin(c, dd, k0 + ik, r, v, inv_q, s_stirl));
                    }
                    __syncwarp(gmask);
                    continue;
                }
                const float inv_nq = 1.0f / (float)nq;
                for (int item = gl; item < nr * nq; item += G) {
                    const int ir = (int)(((float)item + 0.5f) * inv_nq);
                    const int iq = item - ir * nq;
                    const int64_t r = r0 + ir;
                    const int kq = (q_lo + iq) * 4;
                    const float w = wp[ir];
                    const float4 t4 = reinterpret_cast<const float4*>(wt)[iq];
                    float v[4] = {w * t4.x, w * t4.y, w * t4.z, w * t4.w};
                    if (c.fluctuate == 1) {
                        // normal approximation to Binomial(Q', mean / Q'); zero-mean bins
                        // (outside the window) stay zero
                        float z[4];
                        box_muller4(philox(make_uint4((uint32_t)(q_lo + iq), (uint32_t)r, dd.id,
                                                      c.plane_id), c.key0, c.key1), z);
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            const float var = v[e] * (1.0f - v[e] * inv_q);
                            v[e] = fmaxf(0.0f, fmaf(sqrt_fast(var), z[e], v[e]));
                        }
                    }
                    float* dst = grid + r * c.n_ticks + kq;
                    if (vec4) {
                        atomicAdd(reinterpret_cast<float4*>(dst), make_float4(v[0], v[1], v[2], v[3]));
                    } else {
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            const int ik = kq + e - k0;
                            if (ik >= 0 && ik < nt) atomicAdd(dst + e, v[e]);
                        }
                    }
                }
                __syncwarp(gmask);
            }
        }
    }
}

template <int KD, int G, bool BIN>
__global__ void __launch_bounds__(kWarps * 32)
k_rasterize(RasterConsts c, DepoArrays d, float* __restrict__ grid, int* flags)
{
    rasterize_block<KD, G, BIN>(c, d, grid, flags, blockIdx.x);
}

// Several events of one plane: CTA b belongs to the event whose block range holds b.
template <int KD, int G, bool BIN>
__global__ void __launch_bounds__(kWarps * 32)
k_rasterize_batch(RasterConsts c, BatchEvents ev, int* flags)
{
    int e = 0;
    while (e + 1 < ev.n && ev.block_start[e + 1] <= (int)blockIdx.x) ++e;
    c.key0 = ev.key0[e];
    c.key1 = ev.key1[e];
    rasterize_block<KD, G, BIN>(c, ev.d[e], ev.grid[e], flags,
                                (int64_t)blockIdx.x - ev.block_start[e]);
}

// Every event of a batch over a work queue: each CTA pops (event, depo block) items until the
// queue is empty (events of different planes carry their own constants).
template <int KD, int G, bool BIN>
__global__ void __launch_bounds__(kWarps * 32)
k_rasterize_queue(QueueEvents q, int* queue)
{
    __shared__ int s_item;
    const int total = q.block_start[q.n];
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(queue, 1);
        __syncthreads();
        const int item = s_item;
        __syncthreads();                   // every thread has the item before s_item is reused
        if (item >= total) break;
        int e = 0;
        while (e + 1 < q.n && q.block_start[e + 1] <= item) ++e;
        rasterize_block<KD, G, BIN>(q.c[e], q.d[e], q.grid[e], q.flags[e],
                                    (int64_t)item - q.block_start[e]);
        __syncthreads();                   // the block's shared tiles are reused by the next item
    }
}

// Sum over the G lanes of a lane group (mask: the group's lanes), in every lane of it.
template <int G>
__device__ __forceinline__ float group_sum(float v, unsigned mask)
{
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(mask, v, o);
    return v;
}

// Renormalisation factors of one depo for the adjoint: 1 / T and the telescoped dT/dmu,
// dT/dsigma per axis (rows, then ticks), T the unclipped window's mass between its outer
// edges: dT/dmu = -(phi(B') - phi(A')) / sigma, dT/dsigma = -(B' phi(B') - A' phi(A')) /
// sigma.  The identity (1, 0, 0) when renormalisation is off or sigma == 0.
__device__ __forceinline__ void renorm_factors(const RasterConsts& c, const Decision& r, float* f)
{
    f[0] = 1.0f; f[1] = 0.0f; f[2] = 0.0f;
    f[3] = 1.0f; f[4] = 0.0f; f[5] = 0.0f;
    if (!c.renorm || !r.ok) return;
#pragma unroll
    for (int ax = 0; ax < 2; ++ax) {
        const float sg = ax ? r.st : r.sp;
        if (!(sg > 0.0f)) continue;
        const float bin = ax ? c.dt_f : c.dp_f;
        const float s = bin / (1.41421356237309505f * sg);
        const float hw = __fmul_rn(__fmul_rn(c.nsig, sg), ax ? c.inv_dt_f : c.inv_dp_f);
        const float frac = ax ? r.frac_t : r.frac_p;
        const float ua = outer_edge_u(frac, hw, s, false), ub = outer_edge_u(frac, hw, s, true);
        const float pa = 0.398942280401432678f * expf(-ua * ua);
        const float pb = 0.398942280401432678f * expf(-ub * ub);
        const float isg = 1.0f / sg;
        f[3 * ax + 0] = 1.0f / span_mass(ua, ub, erfcf(fabsf(ua)), erfcf(fabsf(ub)));
        f[3 * ax + 1] = -(pb - pa) * isg;
        f[3 * ax + 2] = -1.41421356237309505f * (ub * pb - ua * pa) * isg;
    }
}

// Per depo (a half warp each, so that the per-group tiles fit static shared memory):
// recompute the patch weights and their mu / sigma derivatives, gather dL/dS over the patch
// and apply the chain rule through Q' = Q exp(-t_d / tau), t_a = t + t_d and
// sigma = sqrt(2 D t_d).  The global sums are reduced per block in FP64.
template <bool RN>
__global__ void __launch_bounds__(kWarps * 32, 3)
k_depo_adjoint(RasterConsts c, DepoArrays d, const float* __restrict__ dgrid, DepoGrads g,
               int* flags)
{
    // 8 lanes per depo (as the forward's default tile; 16 lanes took 84 against 74 us on the
    // 960 x 6000 plane); patch tiles of at most kTile rows x kTile ticks
    constexpr int G = 8, NG = kWarps * 32 / G, kTile = 32;
    __shared__ Decision s_dec[kDepos];
    // wp, dwp/dmu, dwp/dsig per row; wt, dwt/dmu, dwt/dsig per tick laid out on 4-tick
    // groups (slot p is tick 4 q_lo + p, zero outside the window)
    __shared__ float s_w[NG][3][kTile];
    __shared__ __align__(16) float s_t[NG][3][kTile + 8];
    // per bin edge u: erfc|u|, phi(u) = exp(-u^2) / sqrt(2 pi) and u phi(u); rows then ticks
    __shared__ float s_e[NG][3][2 * (kTile + 1)];
    // per depo, the FP32 factors of its terms in the three global sums (dL/dsigma_L,
    // sigma_L; dL/dsigma_T, sigma_T; dL/dQ', Q'), zero for depos that add nothing
    __shared__ float s_gt[kDepos][6];
    // per depo, the renormalisation factors of its rows and ticks: 1 / T, dT/dmu, dT/dsigma
    // (an instance of its own, so that the plain adjoint keeps its registers)
    __shared__ float s_rn[RN ? kDepos : 1][6];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gl = threadIdx.x % G, grp = threadIdx.x / G;
    const unsigned gmask = ((1u << G) - 1u) << (lane & ~(G - 1));
    const int64_t base = (int64_t)blockIdx.x * kDepos;
    if (threadIdx.x < kDepos) {
        Decision r;
        r.ok = 0;
        const int64_t i = base + threadIdx.x;
        if (i < d.n) {
            r = decide(c, d, i, flags);
            r.id = d.id[i];
        }
        s_dec[threadIdx.x] = r;
        if (RN) renorm_factors(c, r, s_rn[threadIdx.x]);
#pragma unroll
        for (int k = 0; k < 6; ++k) s_gt[threadIdx.x][k] = 0.0f;
    }
    __syncthreads();
    float* wp = s_w[grp][0];
    float* wpm = s_w[grp][1];
    float* wps = s_w[grp][2];
    float* wt = s_t[grp][0];
    float* wtm = s_t[grp][1];
    float* wts = s_t[grp][2];
    float* eE = s_e[grp][0];
    float* eP = s_e[grp][1];
    float* eU = s_e[grp][2];
    const bool vec4 = ((c.n_ticks & 3) == 0) && ((reinterpret_cast<uintptr_t>(dgrid) & 15) == 0);

    for (int i = grp; i < kDepos; i += NG) {
        const int64_t gi = base + i;
        if (gi >= d.n) break;
        const Decision dd = s_dec[i];
        float a_q = 0.f, a_pm = 0.f, a_ps = 0.f, a_tm = 0.f, a_ts = 0.f;
        if (dd.ok && dd.qatt > 0.0f) {
            const float s_p = (dd.sp > 0.0f) ? c.dp_f / (1.41421356237309505f * dd.sp) : 0.0f;
            const float s_t = (dd.st > 0.0f) ? c.dt_f / (1.41421356237309505f * dd.st) : 0.0f;
            const float isp = (dd.sp > 0.0f) ? 1.0f / dd.sp : 0.0f;
            const float ist = (dd.st > 0.0f) ? 1.0f / dd.st : 0.0f;
            // renormalised weights w / T and their derivatives by the quotient rule,
            // (dw - (w / T) dT) / T (the identity when renormalisation is off)
            const float* rn = s_rn[RN ? i : 0];
            for (int32_t r0 = dd.r_lo; r0 <= dd.r_hi; r0 += kTile) {
                const int nr = min(kTile, dd.r_hi - r0 + 1);
                for (int32_t k0 = dd.k_lo; k0 <= dd.k_hi; k0 += kTile) {
                    const int nt = min(kTile, dd.k_hi - k0 + 1);
                    const int q_lo = k0 >> 2, q_hi = (k0 + nt - 1) >> 2, nq = q_hi - q_lo + 1;
                    const int koff = k0 - 4 * q_lo;        // slot of tick k0
                    // edge terms: nr + 1 row edges, nt + 1 tick edges
                    for (int e = gl; e < nr + nt + 2; e += G) {
                        const float u = (e <= nr) ? ((float)((int64_t)(r0 + e) - dd.i0p) - dd.frac_p) * s_p
                                                  : ((float)((int64_t)(k0 + e - nr - 1) - dd.i0t) - dd.frac_t) * s_t;
                        const float ph = 0.398942280401432678f * expf(-u * u);
                        eE[e] = erfcf(fabsf(u));
                        eP[e] = ph;
                        eU[e] = u * ph;
                    }
                    __syncwarp(gmask);
                    // w = Phi(b') - Phi(a'); dw/dmu = -(phi(b') - phi(a')) / sigma;
                    // dw/dsigma = -(b' phi(b') - a' phi(a')) / sigma, with b' = sqrt(2) ub
                    for (int e = gl; e < nr + 4 * nq; e += G) {
                        if (e < nr) {
                            float w = 1.0f, m = 0.0f, sg = 0.0f;
                            if (dd.sp > 0.0f) {
                                w = bin_mass((int64_t)(r0 + e) - dd.i0p, dd.frac_p, s_p, eE[e], eE[e + 1]);
                                m = -(eP[e + 1] - eP[e]);
                                sg = -1.41421356237309505f * (eU[e + 1] - eU[e]);
                            }
                            if (RN) {
                                const float wn = w * rn[0];
                                wp[e] = wn;
                                wpm[e] = (m * isp - wn * rn[1]) * rn[0];
                                wps[e] = (sg * isp - wn * rn[2]) * rn[0];
                            } else {
                                wp[e] = w;
                                wpm[e] = m * isp;
                                wps[e] = sg * isp;
                            }
                        } else {
                            const int k = e - nr - koff, a = nr + 1 + k;
                            float w = 0.0f, m = 0.0f, sg = 0.0f;
                            if (k >= 0 && k < nt) {
                                if (dd.st > 0.0f) {
                                    w = bin_mass((int64_t)(k0 + k) - dd.i0t, dd.frac_t, s_t, eE[a], eE[a + 1]);
                                    m = -(eP[a + 1] - eP[a]);
                                    sg = -1.41421356237309505f * (eU[a + 1] - eU[a]);
                                } else {
                                    w = 1.0f;
                                }
                            }
                            if (RN) {
                                const float wn = w * rn[3];
                                wt[e - nr] = wn;
                                wtm[e - nr] = (m * ist - wn * rn[4]) * rn[3];
                                wts[e - nr] = (sg * ist - wn * rn[5]) * rn[3];
                            } else {
                                wt[e - nr] = w;
                                wtm[e - nr] = m * ist;
                                wts[e - nr] = sg * ist;
                            }
                        }
                    }
                    __syncwarp(gmask);
                    if (vec4) {
                        // (row, 4-tick group) items: one 16-byte load of dL/dS per item
                        const float inv_nq = 1.0f / (float)nq;
                        for (int item = gl; item < nr * nq; item += G) {
                            const int ir = (int)(((float)item + 0.5f) * inv_nq);
                            const int iq = item - ir * nq;
                            const int kq = (q_lo + iq) * 4;
                            const float4 sv = __ldg(reinterpret_cast<const float4*>(
                                dgrid + (int64_t)(r0 + ir) * c.n_ticks + kq));
                            const float4 w4 = reinterpret_cast<const float4*>(wt)[iq];
                            const float4 m4 = reinterpret_cast<const float4*>(wtm)[iq];
                            const float4 g4 = reinterpret_cast<const float4*>(wts)[iq];
                            const float A = sv.x * w4.x + sv.y * w4.y + sv.z * w4.z + sv.w * w4.w;
                            const float B = sv.x * m4.x + sv.y * m4.y + sv.z * m4.z + sv.w * m4.w;
                            const float C = sv.x * g4.x + sv.y * g4.y + sv.z * g4.z + sv.w * g4.w;
                            const float pw = wp[ir];
                            a_q += pw * A;
                            a_pm += wpm[ir] * A;
                            a_ps += wps[ir] * A;
                            a_tm += pw * B;
                            a_ts += pw * C;
                        }
                    } else {
                        const float inv_nt = 1.0f / (float)nt;
                        for (int b = gl; b < nr * nt; b += G) {
                            const int ir = (int)(((float)b + 0.5f) * inv_nt);
                            const int ik = b - ir * nt;
                            const float sv = __ldg(dgrid + (int64_t)(r0 + ir) * c.n_ticks + (k0 + ik));
                            const float pw = wp[ir], tw = wt[ik + koff];
                            a_q += sv * pw * tw;
                            a_pm += sv * wpm[ir] * tw;
                            a_ps += sv * wps[ir] * tw;
                            a_tm += sv * pw * wtm[ik + koff];
                            a_ts += sv * pw * wts[ik + koff];
                        }
                    }
                    __syncwarp(gmask);
                }
            }
            a_q = group_sum<G>(a_q, gmask);
            a_pm = group_sum<G>(a_pm, gmask);
            a_ps = group_sum<G>(a_ps, gmask);
            a_tm = group_sum<G>(a_tm, gmask);
            a_ts = group_sum<G>(a_ts, gmask);
        }
        if (gl == 0) {
            const float qa = dd.ok ? dd.qatt : 0.0f;
            const float att = (dd.ok && qa > 0.0f) ? qa / d.q[gi] : 0.0f;
            const float dst = qa * a_ps, dsl = qa * a_ts * c.inv_v;
            if (g.dq) g.dq[gi] = a_q * att;
            if (g.dp) g.dp[gi] = qa * a_pm;
            if (g.dt) g.dt[gi] = qa * a_tm;
            if (g.dsl) g.dsl[gi] = dsl;
            if (g.dst) g.dst[gi] = dst;
            if (dd.ok && qa > 0.0f) {
                s_gt[i][0] = dsl;
                s_gt[i][1] = dd.st;
                s_gt[i][2] = dst;
                s_gt[i][3] = dd.sp;
                s_gt[i][4] = a_q;
                s_gt[i][5] = qa;
            }
        }
    }
    __syncthreads();
    // The global sums, by one warp for the whole block (FP64 is scarce on this part: one
    // warp instruction per 32 depos).  sigma = sqrt(2 D t_d) gives dsigma/dD = sigma / (2 D)
    // (sigma_L = v sigma_t in mm); dQ'/dtau = Q' t_d / tau^2.  Products of two FP32 values
    // are exact in FP64.
    if (warp == 0 && g.dglobal) {
        double a0 = 0.0, a1 = 0.0, a2 = 0.0;
        for (int i = lane; i < kDepos; i += 32) {
            if (!(s_gt[i][5] > 0.0f)) continue;
            a0 += (double)s_gt[i][0] * (double)s_gt[i][1];
            a1 += (double)s_gt[i][2] * (double)s_gt[i][3];
            a2 += (double)s_gt[i][4] * (double)s_gt[i][5] * d.td[base + i];
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            a0 += __shfl_xor_sync(0xffffffffu, a0, o);
            a1 += __shfl_xor_sync(0xffffffffu, a1, o);
            a2 += __shfl_xor_sync(0xffffffffu, a2, o);
        }
        if (lane == 0) {
            if (c.DL > 0.0) atomicAdd(g.dglobal + 0, a0 * c.v / (2.0 * c.DL));
            if (c.DT > 0.0) atomicAdd(g.dglobal + 1, a1 / (2.0 * c.DT));
            atomicAdd(g.dglobal + 2, a2 / (c.tau * c.tau));
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

bool raster_tile_supported(int depos_per_block, int lanes_per_depo)
{
#define WCSIM_TILE_CASE(KD, G) if (depos_per_block == KD && lanes_per_depo == G) return true;
    WCSIM_RASTER_TILES(WCSIM_TILE_CASE)
#undef WCSIM_TILE_CASE
    return false;
}

cudaError_t launch_rasterize(const RasterConsts& c, const DepoArrays& d, float* grid,
                             int* flags, cudaStream_t s)
{
    if (d.n <= 0) return cudaSuccess;
    if (!raster_tile_supported(c.depos_per_block, c.lanes_per_depo)) return cudaErrorInvalidValue;
    const unsigned blocks = (unsigned)rasterize_blocks(d.n, c.depos_per_block);
#define WCSIM_TILE_CASE(KD, G)                                                                 \
    if (c.depos_per_block == KD && c.lanes_per_depo == G) {                                    \
        if (c.fluctuate == 2)                                                                  \
            k_rasterize<KD, G, true><<<blocks, kWarps * 32, 0, s>>>(c, d, grid, flags);        \
        else                                                                                   \
            k_rasterize<KD, G, false><<<blocks, kWarps * 32, 0, s>>>(c, d, grid, flags);       \
    }
    WCSIM_RASTER_TILES(WCSIM_TILE_CASE)
#undef WCSIM_TILE_CASE
    return cudaGetLastError();
}

int rasterize_blocks(int64_t n_depos, int depos_per_block)
{
    const int kd = depos_per_block > 0 ? depos_per_block : 64;
    return (int)((n_depos + kd - 1) / kd);
}

cudaError_t launch_rasterize_batch(const RasterConsts& c, const BatchEvents& ev, int* flags,
                                   cudaStream_t s)
{
    const int blocks = ev.block_start[ev.n];
    if (blocks <= 0) return cudaSuccess;
    if (!raster_tile_supported(c.depos_per_block, c.lanes_per_depo)) return cudaErrorInvalidValue;
#define WCSIM_TILE_CASE(KD, G)                                                                 \
    if (c.depos_per_block == KD && c.lanes_per_depo == G) {                                    \
        if (c.fluctuate == 2)                                                                  \
            k_rasterize_batch<KD, G, true><<<blocks, kWarps * 32, 0, s>>>(c, ev, flags);       \
        else                                                                                   \
            k_rasterize_batch<KD, G, false><<<blocks, kWarps * 32, 0, s>>>(c, ev, flags);      \
    }
    WCSIM_RASTER_TILES(WCSIM_TILE_CASE)
#undef WCSIM_TILE_CASE
    return cudaGetLastError();
}

cudaError_t launch_rasterize_queue(const QueueEvents& q, int* queue, cudaStream_t s)
{
    const int total = q.block_start[q.n];
    if (q.n <= 0 || total <= 0) return cudaSuccess;
    const RasterConsts& c = q.c[0];
    if (!raster_tile_supported(c.depos_per_block, c.lanes_per_depo)) return cudaErrorInvalidValue;
    cudaError_t e = cudaMemsetAsync(queue, 0, sizeof(int), s);
    if (e) return e;
#define WCSIM_TILE_CASE(KD, G)                                                                 \
    if (c.depos_per_block == KD && c.lanes_per_depo == G) {                                    \
        auto k = (c.fluctuate == 2) ? k_rasterize_queue<KD, G, true>                           \
                                    : k_rasterize_queue<KD, G, false>;                         \
        int per_sm = 0;                                                                        \
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kWarps * 32, 0)))   \
            return e;                                                                          \
        const int resident = (per_sm > 0 ? per_sm : 1) * sm_count();                           \
        k<<<total < resident ? total : resident, kWarps * 32, 0, s>>>(q, queue);               \
    }
    WCSIM_RASTER_TILES(WCSIM_TILE_CASE)
#undef WCSIM_TILE_CASE
    return cudaGetLastError();
}

cudaError_t launch_depo_adjoint(const RasterConsts& c, const DepoArrays& d, const float* dgrid,
                                const DepoGrads& g, int* flags, cudaStream_t s)
{
    if (d.n <= 0) return cudaSuccess;
    const int64_t blocks = (d.n + kDepos - 1) / kDepos;
    if (c.renorm) k_depo_adjoint<true><<<(unsigned)blocks, kWarps * 32, 0, s>>>(c, d, dgrid, g, flags);
    else k_depo_adjoint<false><<<(unsigned)blocks, kWarps * 32, 0, s>>>(c, d, dgrid, g, flags);
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
