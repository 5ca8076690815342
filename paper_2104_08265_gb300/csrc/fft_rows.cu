// Time-axis transforms of Eq. 2: forward real-to-complex FFT of every grid row and inverse
// complex-to-real FFT of every wire's spectrum.  Two real rows ride in one complex FFT
// (z = x0 + i x1); their spectra are separated with X0 = (Z[k] + conj Z[-k]) / 2,
// X1 = (Z[k] - conj Z[-k]) / 2i.
//
// rows_r2c (direct, the default) takes one pair of rows per CTA: both rows are loaded into
// shared memory with batched 16-byte loads (scalar loads when rows are not 16-byte aligned),
// a pair with no nonzero value stores zero spectra at once, and otherwise every pass of the
// plan runs in shared memory (in place, in one buffer, for the compile-time 6000-point plan;
// between two buffers for runtime plans); the CTA also asks L2 for the rows of the CTA
// expected to follow it on the SM.  The two half spectra are separated into flat shared rows
// and leave through TMA tensor box stores (per-thread stores with WCSIM_SPECTRA_TMA=0).
// rows_r2c (staged, chosen by the autotuner or
// WCSIM_ROWS_KERNEL) is persistent: one CTA per SM walks pairs of rows, and one bulk copy
// brings both rows of the next pair into a two-stage shared buffer while the previous pair
// is transformed.  The inverse kernel stages its Hermitian input (each element read once,
// its mirror written from the same load) and writes 4 ticks per 16-byte store, or, given a
// target frame, the residual M - target and its sum of squares.
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include "async_copy.cuh"
#include "fft_engine.cuh"
#include "wcsim_internal.cuh"

namespace wcsim {
namespace {

constexpr int kStagedThreads = 512;
constexpr int kDirectThreads = 256;
constexpr size_t kMaxSmem = 227 * 1024;

// First-pass source: element i of z = x0 + i x1 (zero beyond the frame), from a pair of rows
// (row 0 then row 1) staged in shared memory.
struct StagedPairLd {
    const float* t;
    int n_t;
    bool has1;
    __device__ __forceinline__ float2 operator()(int, int i) const
    {
        if (i >= n_t) return make_float2(0.f, 0.f);
        return make_float2(t[i], has1 ? t[n_t + i] : 0.f);
    }
};

// Stage z[i] = x0[i] + i x1[i], i < n (zero beyond n_t, x1 = 0 when g1 is null), into the
// unpadded shared buffer z (16-byte aligned; read back through FlatLd).  With vec (rows
// 16-byte aligned, n_t a multiple of 4) each thread issues its 16-byte loads in batches of
// kU per row before storing them.  With clear the
// rows are left zero (consume and clear): only the groups that hold a nonzero value are
// written, so the untouched part of a sparse grid costs no writes.  Returns whether this
// thread saw a nonzero value.  Ends without a barrier.
__device__ __forceinline__ bool stage_real_pair(float* g0, float* g1, int n_t, int n, bool vec,
                                                bool clear, float2* z)
{
    bool any = false;
    for (int i = n_t + threadIdx.x; i < n; i += blockDim.x) z[i] = make_float2(0.f, 0.f);
    float4* z4 = reinterpret_cast<float4*>(z);
    if (vec) {
        constexpr int kU = 6;
        const int nq = n_t >> 2;
        float4* q0 = reinterpret_cast<float4*>(g0);
        float4* q1 = reinterpret_cast<float4*>(g1);
        const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
        auto nz = [](const float4& v) { return v.x != 0.f || v.y != 0.f || v.z != 0.f || v.w != 0.f; };
        for (int base = threadIdx.x; base < nq; base += kU * blockDim.x) {
            float4 a[kU], b[kU];
#pragma unroll
            for (int u = 0; u < kU; ++u) {
                const int q = base + u * blockDim.x;
                a[u] = b[u] = zero;
                if (q < nq) {
                    a[u] = q0[q];
                    if (g1) b[u] = q1[q];
                }
            }
#pragma unroll
            for (int u = 0; u < kU; ++u) {
                const int q = base + u * blockDim.x;
                if (q < nq) {
                    z4[2 * q] = make_float4(a[u].x, b[u].x, a[u].y, b[u].y);
                    z4[2 * q + 1] = make_float4(a[u].z, b[u].z, a[u].w, b[u].w);
                    const bool na = nz(a[u]), nb = nz(b[u]);
                    any |= na | nb;
                    if (clear) {
                        if (na) q0[q] = zero;
                        if (g1 && nb) q1[q] = zero;
                    }
                }
            }
        }
    } else {
        for (int i = threadIdx.x; i < n_t; i += blockDim.x) {
            const float x0 = g0[i], x1 = g1 ? g1[i] : 0.f;
            z[i] = make_float2(x0, x1);
            any |= (x0 != 0.f) | (x1 != 0.f);
            if (clear) {
                if (x0 != 0.f) g0[i] = 0.f;
                if (x1 != 0.f) g1[i] = 0.f;
            }
        }
    }
    return any;
}

// Separate the two real rows' half spectra and store them in the blocked layout (zeros in
// the padding columns nh .. 4 nkb - 1).  Consecutive lanes take consecutive frequencies, so
// the shared reads are free of conflicts and every 4 lanes fill one 32-byte sector per row.
// The block size is a multiple of 16, so the output addresses and the padded shared indices
// of k and N - k advance by constants from one iteration to the next.
__device__ __forceinline__ void store_pair_spectra(const ConvDims& d, const float2* z, int N,
                                                   int64_t r0, bool has1, float2* shat,
                                                   bool zero = false)
{
    const int w0 = (int)(r0 / d.n_imp), j0 = (int)(r0 % d.n_imp);
    const int64_t r1 = r0 + 1;
    const int w1 = (int)(r1 / d.n_imp), j1 = (int)(r1 % d.n_imp);
    const int nk = d.nkb * kBlockCols, nh = d.nh;
    const int k0 = threadIdx.x;
    const int64_t row = (int64_t)d.n_w * kBlockCols;                  // one block of columns
    const int64_t step = (int64_t)(blockDim.x / kBlockCols) * row;
    float2* q0 = shat + (int64_t)j0 * d.nkb * row + (k0 >> 2) * row + w0 * kBlockCols + (k0 & 3);
    float2* q1 = shat + (int64_t)j1 * d.nkb * row + (k0 >> 2) * row + w1 * kBlockCols + (k0 & 3);
    const int dp = blockDim.x + (blockDim.x >> 4);                      // pad16 step
    int pa = pad16(k0), pb = pad16(N - k0);
    for (int k = k0; k < nk; k += blockDim.x, q0 += step, q1 += step, pa += dp, pb -= dp) {
        float2 x0 = make_float2(0.f, 0.f), x1 = x0;
        if (k < nh && !zero) {
            const float2 a = z[pa];
            const float2 b = z[k == 0 ? 0 : pb];
            x0 = make_float2(0.5f * (a.x + b.x), 0.5f * (a.y - b.y));
            x1 = make_float2(0.5f * (a.y + b.y), 0.5f * (b.x - a.x));
        }
        *q0 = x0;
        if (has1) *q1 = x1;
    }
}

// Shared offset (complex values) of row 1's flat half spectrum: 4 nkb rounded up to 128 bytes.
__host__ __device__ inline int flat_row1(int nkb) { return (kBlockCols * nkb + 15) & ~15; }

// The first 128-byte aligned complex slot at or after p (a TMA box in shared memory starts
// on a 128-byte boundary): at most kFlatSlack slots further.
constexpr int kFlatSlack = 15;
__device__ __forceinline__ float2* align128(float2* p)
{
    const uint32_t a = smem_u32(p);
    return p + (((128u - (a & 127u)) & 127u) >> 3);
}

// Separate the pair's half spectra as store_pair_spectra does, into flat shared rows for the
// TMA box stores: row 0's X0[k] at f[k], row 1's X1[k] at f[o1 + k], zeros for nh <= k < nk.
// NI > 0: f may alias z; every thread first reads its NI frequencies k = tid + i T (NI T >= nh)
// into registers, the block synchronises, then writes.  NI = 0: f and z are distinct buffers.
// Ends with a proxy fence and a block barrier (the async proxy may then read f).
template <int NI, int T>
__device__ __forceinline__ void separate_flat(const float2* z, int N, int nh, int nk, int o1,
                                              float2* f)
{
    auto sep = [&](int k, float2& x0, float2& x1) {
        const float2 a = z[pad16(k)];
        const float2 b = z[k == 0 ? 0 : pad16(N - k)];
        x0 = make_float2(0.5f * (a.x + b.x), 0.5f * (a.y - b.y));
        x1 = make_float2(0.5f * (a.y + b.y), 0.5f * (b.x - a.x));
    };
    if constexpr (NI > 0) {
        float2 a0[NI], a1[NI];
#pragma unroll
        for (int i = 0; i < NI; ++i) {
            const int k = threadIdx.x + i * T;
            if (k < nh) sep(k, a0[i], a1[i]);
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < NI; ++i) {
            const int k = threadIdx.x + i * T;
            if (k < nh) {
                f[k] = a0[i];
                f[o1 + k] = a1[i];
            }
        }
    } else {
        for (int k = threadIdx.x; k < nh; k += T) {
            float2 x0, x1;
            sep(k, x0, x1);
            f[k] = x0;
            f[o1 + k] = x1;
        }
    }
    for (int k = nh + threadIdx.x; k < nk; k += T) f[k] = f[o1 + k] = make_float2(0.f, 0.f);
    fence_proxy_async_smem();
    __syncthreads();
}

// One thread stores the flat rows f (row 0) and f + o1 (row 1, if has1) of rows r0, r0 + 1 of
// event ev through the tensor map, bk frequency blocks per box, and waits until the copies
// have read shared memory.  Boxes past nkb are clipped by the copy.
__device__ __forceinline__ void tma_store_pair(const ConvDims& d, const CUtensorMap* map,
                                               const float2* f, int o1, int bk, int64_t r0,
                                               bool has1, int ev)
{
    const int w0 = (int)(r0 / d.n_imp), j0 = (int)(r0 % d.n_imp);
    const int w1 = (int)((r0 + 1) / d.n_imp), j1 = (int)((r0 + 1) % d.n_imp);
    for (int kb = 0; kb < d.nkb; kb += bk) {
        tma_store_5d(map, f + kBlockCols * kb, 0, w0, kb, j0, ev);
        if (has1) tma_store_5d(map, f + o1 + kBlockCols * kb, 0, w1, kb, j1, ev);
    }
    bulk_commit();
    bulk_wait_read();
}

__host__ __device__ inline size_t staged_smem(int n_t, int n)
{
    return 2 * 2 * (size_t)n_t * sizeof(float) + 2 * (size_t)padded_len(n) * sizeof(float2) +
           2 * sizeof(uint64_t);
}

__global__ void __launch_bounds__(kStagedThreads, 1)
k_rows_r2c_staged(ConvDims d, FftPlan p, const float* __restrict__ grid, float2* __restrict__ shat,
                  int* flags)
{
    extern __shared__ __align__(128) unsigned char smraw[];
    const int N = p.n;
    float* st = reinterpret_cast<float*>(smraw);           // stage s at st + s * 2 n_t
    float2* X = reinterpret_cast<float2*>(st + 4 * d.n_t);
    float2* Y = X + padded_len(N);
    uint64_t* bar = reinterpret_cast<uint64_t*>(Y + padded_len(N));
    const int64_t n_rows = (int64_t)d.n_w * d.n_imp;
    const int64_t n_pairs = (n_rows + 1) / 2;
    const int n_items = (n_pairs > (int64_t)blockIdx.x)
                            ? (int)((n_pairs - 1 - blockIdx.x) / gridDim.x + 1) : 0;
    const int tid = threadIdx.x;

    auto issue = [&](int i) {
        const int64_t r0 = 2 * ((int64_t)blockIdx.x + (int64_t)i * gridDim.x);
        const uint32_t bytes = (uint32_t)((r0 + 1 < n_rows ? 2 : 1) * d.n_t * sizeof(float));
        mbar_arrive_expect_tx(&bar[i & 1], bytes);
        bulk_g2s(st + (i & 1) * 2 * d.n_t, grid + r0 * d.n_t, bytes, &bar[i & 1]);
    };

    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (tid == 0) {
        if (n_items > 0) issue(0);
        if (n_items > 1) issue(1);
    }
    int i = 0;
    for (; i < n_items; ++i) {
        const int s = i & 1;
        const int64_t r0 = 2 * ((int64_t)blockIdx.x + (int64_t)i * gridDim.x);
        const bool has1 = r0 + 1 < n_rows;
        const bool landed = mbar_wait(&bar[s], (i >> 1) & 1, d.wait_ns);
        if (!__syncthreads_and(landed)) break;
        const float2* z = run_plan<false, 0>(p, StagedPairLd{st + s * 2 * d.n_t, d.n_t, has1}, X, Y);
        if (tid == 0 && i + 2 < n_items) {     // stage s was read by the first pass only
            fence_proxy_async_smem();
            issue(i + 2);
        }
        store_pair_spectra(d, z, N, r0, has1, shat);
        __syncthreads();
    }
    if (i < n_items && tid == 0) {
        atomicOr(flags, kErrTimeout);
        for (int k = i; k < n_items && k < i + 2; ++k) mbar_wait(&bar[k & 1], (k >> 1) & 1);
    }
}

// pf_ahead > 0: CTA b first asks L2 for the rows of pair b + pf_ahead (the CTA that will
// most likely take over its slot once it retires), so that pair's first pass reads L2.
// FIX: compile-time plan variant (fixed_plan_of(p)).
// bk > 0: the half spectra leave through TMA box stores of bk frequency blocks (map: the
// blocked spectra, events along its last dimension); bk = 0: plain stores.
template <int FIX>
__global__ void __launch_bounds__(kDirectThreads, FIX == kPlanRuntime ? 2 : 3)
k_rows_r2c_direct(ConvDims d, FftPlan p, float* __restrict__ grid, float2* __restrict__ shat,
                  int pf_ahead, const __grid_constant__ CUtensorMap map, int bk)
{
    extern __shared__ __align__(128) unsigned char smraw[];
    const int N = p.n;
    float2* X = reinterpret_cast<float2*>(smraw);
    float2* Y = X + padded_len(N);
    const int64_t n_rows = (int64_t)d.n_w * d.n_imp;
    const int64_t r0 = 2 * (int64_t)blockIdx.x;
    const bool has1 = r0 + 1 < n_rows;
    grid += blockIdx.y * d.ev_grid;          // event of a batched launch (0 otherwise)
    shat += blockIdx.y * d.ev_shat;
    if (pf_ahead > 0 && threadIdx.x == 0) {
        const int64_t q0 = r0 + 2 * (int64_t)pf_ahead;
        if (q0 < n_rows) {
            const int nq = (q0 + 1 < n_rows) ? 2 : 1;
            bulk_prefetch_l2(grid + q0 * d.n_t, (uint32_t)(nq * d.n_t * sizeof(float)));
        }
    }
    const bool vec = ((d.n_t & 3) == 0) && ((reinterpret_cast<uintptr_t>(grid) & 15) == 0);
    float* g0 = grid + r0 * d.n_t;
    const bool any = stage_real_pair(g0, has1 ? g0 + d.n_t : nullptr, d.n_t, N, vec,
                                     d.clear_input != 0, X);
    // the transform of two all-zero rows is zero: store zero spectra and skip the passes
    if (!__syncthreads_or(any)) {
        store_pair_spectra(d, X, N, r0, has1, shat, true);
        return;
    }
    const float2* z = run_row_plan<false, FIX, kDirectThreads>(p, X, Y);
    if (bk > 0) {
        const int o1 = flat_row1(d.nkb);
        if constexpr (FIX == kPlan6000) {
            constexpr int NI = (6000 / 2 + 1 + kDirectThreads - 1) / kDirectThreads;
            float2* f = align128(X);
            separate_flat<NI, kDirectThreads>(z, N, d.nh, kBlockCols * d.nkb, o1, f);
            if (threadIdx.x == 0) tma_store_pair(d, &map, f, o1, bk, r0, has1, blockIdx.y);
        } else {
            float2* f = align128((z == X) ? Y : X);
            separate_flat<0, kDirectThreads>(z, N, d.nh, kBlockCols * d.nkb, o1, f);
            if (threadIdx.x == 0) tma_store_pair(d, &map, f, o1, bk, r0, has1, blockIdx.y);
        }
        return;
    }
    store_pair_spectra(d, z, N, r0, has1, shat);
}

template <int FIX>
__global__ void __launch_bounds__(kDirectThreads, FIX == kPlanRuntime ? 2 : 3)
k_rows_c2r(ConvDims d, FftPlan p, const float2* __restrict__ mt, WavePtrs waves)
{
    extern __shared__ __align__(128) unsigned char smraw[];
    const int N = p.n;
    mt += blockIdx.y * d.ev_mt;              // event of a batched launch (0 otherwise)
    float* __restrict__ wave = waves.p[blockIdx.y];
    float2* X = reinterpret_cast<float2*>(smraw);
    float2* Y = X + padded_len(N);
    const int w0 = 2 * blockIdx.x, w1 = w0 + 1;
    const bool has1 = w1 < d.n_w;
    if (d.target && threadIdx.x == 0 && (d.n_t & 3) == 0 &&
        (reinterpret_cast<uintptr_t>(d.target) & 15) == 0) {
        // the target rows this CTA subtracts at the end: into L2 while it transforms
        bulk_prefetch_l2(d.target + (int64_t)w0 * d.n_t,
                         (uint32_t)((has1 ? 2 : 1) * d.n_t * sizeof(float)));
    }
    stage_herm_pair(mt, mt, w0, has1 ? w1 : w0, has1, d.n_w, d.nh, N, X, d.noise_amp,
                    d.noise_seed + (uint64_t)waves.ev[blockIdx.y], d.plane_id);
    __syncthreads();
    const float2* z = run_row_plan<true, FIX, kDirectThreads>(p, X, Y);
    if (d.adc_max > 0) {                       // digitized: uint16 codes at the same rows
        uint16_t* adc = reinterpret_cast<uint16_t*>(wave);
        uint16_t* a0 = adc + (int64_t)w0 * d.n_t;
        const bool vec = ((d.n_t & 3) == 0) && ((reinterpret_cast<uintptr_t>(adc) & 7) == 0);
        store_real_pair_adc(z, a0, a0 + d.n_t, d.n_t, has1, vec, d.adc_gain, d.adc_pedestal,
                            (float)d.adc_max);
        return;
    }
    float* o0 = wave + (int64_t)w0 * d.n_t;
    if (d.target) {                            // residual M - target, and 1/2 sum of squares
        const float* t0 = d.target + (int64_t)w0 * d.n_t;
        const bool vec = ((d.n_t & 3) == 0) &&
                         (((reinterpret_cast<uintptr_t>(wave) | reinterpret_cast<uintptr_t>(d.target)) & 15) == 0);
        float ss = store_residual_pair(z, o0, o0 + d.n_t, t0, t0 + d.n_t, d.n_t, has1, vec);
        if (d.loss) {                          // one FP64 addition per warp (no static
#pragma unroll                                         // shared memory: see attrs())
            for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
            if ((threadIdx.x & 31) == 0) atomicAdd(d.loss, 0.5 * (double)ss);
        }
        return;
    }
    const bool vec = ((d.n_t & 3) == 0) && ((reinterpret_cast<uintptr_t>(wave) & 15) == 0);
    store_real_pair(z, o0, o0 + d.n_t, d.n_t, has1, vec);
}

// CTAs of the direct R2C kernel k resident on the whole GPU with smem bytes each, when its
// rows may be prefetched with bulk copies (16-byte aligned rows); 0 otherwise.
template <class K>
int r2c_prefetch_ahead(const ConvDims& d, const float* grid, K k, size_t smem)
{
    if ((d.n_t % 4) != 0 || (reinterpret_cast<uintptr_t>(grid) & 15) != 0) return 0;
    if (d.ev_grid % 4 != 0) return 0;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kDirectThreads, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return per_sm * sm_count();
}

// The TMA store setup of the direct R2C kernel for n_ev events of spectra at shat: the map
// and its box size, or bk = 0 (plain stores) when disabled, unmappable, or when the flat rows
// plus the clipped tail of the last box, from a 128-byte aligned start, do not fit one
// padded_len(n) buffer.
int r2c_store_map(const ConvDims& d, const FftPlan& pt, int fix, const float2* shat, int n_ev,
                  CUtensorMap* map)
{
    memset(map, 0, sizeof(*map));
    if (!d.spectra_tma) return 0;
    const int bk = blocked_box_kb(d.nkb);
    const int64_t span = (int64_t)((d.nkb + bk - 1) / bk) * bk * kBlockCols;
    if (kFlatSlack + flat_row1(d.nkb) + span > (int64_t)padded_len(pt.n)) return 0;
    (void)fix;   // both plan variants write the flat rows into one padded_len(n) buffer
    if (!blocked_spectra_map(shat, d.n_w, d.nkb, d.n_imp, n_ev, d.ev_shat, map)) return 0;
    return bk;
}

// The row kernels declare no static shared memory: the dynamic limit set here is the whole
// per-block opt-in limit, which a static array would push over (the attribute call fails).
DeviceOnce g_attr;
cudaError_t attrs()
{
    if (!g_attr.pending()) return cudaSuccess;
    const int mx = (int)kMaxSmem;
    cudaError_t e = cudaFuncSetAttribute(k_rows_r2c_staged, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    if (!e) e = cudaFuncSetAttribute(k_rows_r2c_direct<kPlanRuntime>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    if (!e) e = cudaFuncSetAttribute(k_rows_r2c_direct<kPlan6000>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    if (!e) e = cudaFuncSetAttribute(k_rows_c2r<kPlanRuntime>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    if (!e) e = cudaFuncSetAttribute(k_rows_c2r<kPlan6000>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    if (!e) g_attr.mark();
    return e;
}

}  // namespace

cudaError_t launch_rows_r2c(const ConvDims& d, const FftPlan& pt, const float* grid,
                            float2* shat, int* flags, cudaStream_t s)
{
    cudaError_t e = attrs();
    if (e) return e;
    const int64_t n_rows = (int64_t)d.n_w * d.n_imp;
    const int64_t n_pairs = (n_rows + 1) / 2;
    const size_t smem = staged_smem(d.n_t, pt.n);
    const bool aligned = (d.n_t % 4 == 0) && ((reinterpret_cast<uintptr_t>(grid) & 15) == 0);
    if (d.rows_variant == 1 && aligned && smem <= kMaxSmem) {
        const int grid_n = n_pairs < sm_count() ? (int)n_pairs : sm_count();
        k_rows_r2c_staged<<<grid_n, kStagedThreads, smem, s>>>(d, pt, grid, shat, flags);
    } else {
        // the kernel writes the grid only with d.clear_input (consume and clear)
        const int fix = fixed_plan_of(pt);
        auto k = fix == kPlan6000 ? k_rows_r2c_direct<kPlan6000> : k_rows_r2c_direct<kPlanRuntime>;
        const size_t sm = row_plan_smem(fix, pt.n);
        CUtensorMap map;
        const int bk = r2c_store_map(d, pt, fix, shat, 1, &map);
        k<<<(unsigned)n_pairs, kDirectThreads, sm, s>>>(d, pt, const_cast<float*>(grid), shat,
                                                        r2c_prefetch_ahead(d, grid, k, sm), map, bk);
    }
    return cudaGetLastError();
}

cudaError_t launch_rows_c2r(const ConvDims& d, const FftPlan& pt, const float2* mt,
                            float* wave, cudaStream_t s)
{
    WavePtrs w;
    w.p[0] = wave;
    w.ev[0] = 0;
    return launch_rows_c2r_batch(d, pt, mt, w, 1, s);
}

cudaError_t launch_rows_c2r_batch(const ConvDims& d, const FftPlan& pt, const float2* mt,
                                  const WavePtrs& waves, int n_ev, cudaStream_t s)
{
    cudaError_t e = attrs();
    if (e) return e;
    const dim3 grid((unsigned)((d.n_w + 1) / 2), (unsigned)n_ev);
    const int fix = fixed_plan_of(pt);
    auto k = fix == kPlan6000 ? k_rows_c2r<kPlan6000> : k_rows_c2r<kPlanRuntime>;
    k<<<grid, kDirectThreads, row_plan_smem(fix, pt.n), s>>>(d, pt, mt, waves);
    return cudaGetLastError();
}

cudaError_t launch_rows_r2c_batch(const ConvDims& d, const FftPlan& pt, const float* grid,
                                  float2* shat, int n_ev, cudaStream_t s)
{
    cudaError_t e = attrs();
    if (e) return e;
    const int64_t n_pairs = ((int64_t)d.n_w * d.n_imp + 1) / 2;
    const dim3 g((unsigned)n_pairs, (unsigned)n_ev);
    const int fix = fixed_plan_of(pt);
    auto k = fix == kPlan6000 ? k_rows_r2c_direct<kPlan6000> : k_rows_r2c_direct<kPlanRuntime>;
    const size_t sm = row_plan_smem(fix, pt.n);
    CUtensorMap map;
    const int bk = r2c_store_map(d, pt, fix, shat, n_ev, &map);
    k<<<g, kDirectThreads, sm, s>>>(d, pt, const_cast<float*>(grid), shat,
                                    r2c_prefetch_ahead(d, grid, k, sm), map, bk);
    return cudaGetLastError();
}

}  // namespace wcsim
