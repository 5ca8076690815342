// Wire-axis part of Eq. 2 for wire FFT sizes that are not 32 M (the one-warp-per-column
// kernel of fft_wire_warp.cu covers those), and the response preparation (make_hermitian:
// the Hermitian half of R, scaled, transposed into the time-frequency-major H).
//
// wire_pass is persistent: one CTA per SM walks work items (block kb of 4 time
// frequencies, impact position j).  For each item it bulk-copies the contiguous tiles
// Shat_j(kb) and H_j(kb) into a two-stage shared buffer (the copy of item i + 1 runs while
// item i is transformed), transforms the 4 columns along the wire axis, multiplies by H_j
// and accumulates over j in shared memory; after the last j of a block it transforms the
// sum back along the wire axis and writes the block of Mt.
#include <cuda_runtime.h>
#include <stdint.h>

#include "async_copy.cuh"
#include "fft_engine.cuh"
#include "wcsim_internal.cuh"

namespace wcsim {
namespace {

constexpr int kThreads = 512;
constexpr int LOGB = 2;                 // 4 columns per block (kBlockCols)

// First-pass source: dense staged tile [w][4], zero for padded wires w >= n_w.
struct StagedTileLd {
    const float2* t;
    int n_w;
    __device__ __forceinline__ float2 operator()(int c, int w) const
    {
        return (w < n_w) ? t[(w << LOGB) + c] : make_float2(0.f, 0.f);
    }
};

// Stage s holds the Shat tile at st + s * stage and the H tile right after it.
struct WireSmem {
    float2* st;
    int stage;
    float2 *X, *Y, *acc;
    uint64_t* bar;
    __device__ __forceinline__ float2* st_s(int s) const { return st + s * stage; }
    __device__ __forceinline__ float2* st_h(int s, int n_w) const { return st + s * stage + n_w * kBlockCols; }
};

__host__ __device__ inline size_t wire_smem_bytes(int n_w, int n_fw)
{
    const size_t tile = (size_t)(n_w + n_fw) * kBlockCols * sizeof(float2);
    const size_t buf = (size_t)padded_len(n_fw) * kBlockCols * sizeof(float2);
    return 2 * tile + 3 * buf + 2 * sizeof(uint64_t);
}

__device__ inline WireSmem carve(unsigned char* base, int n_w, int n_fw)
{
    WireSmem m;
    float2* p = reinterpret_cast<float2*>(base);
    const int pl = padded_len(n_fw) * kBlockCols;
    m.st = p;
    m.stage = (n_w + n_fw) * kBlockCols;
    p += 2 * m.stage;
    m.X = p; p += pl;
    m.Y = p; p += pl;
    m.acc = p; p += pl;
    m.bar = reinterpret_cast<uint64_t*>(p);
    return m;
}

__global__ void __launch_bounds__(kThreads, 1)
k_wire_pass(ConvDims d, FftPlan p, const float2* __restrict__ shat, const float2* __restrict__ H,
            float2* __restrict__ mt, int* flags)
{
    extern __shared__ __align__(128) unsigned char smraw[];
    const int N = p.n;
    WireSmem sm = carve(smraw, d.n_w, N);
    const int tid = threadIdx.x;
    const int my_blocks = (d.nkb > (int)blockIdx.x) ? (d.nkb - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    const int n_items = my_blocks * d.n_imp;
    const uint32_t bytes_s = (uint32_t)(d.n_w * kBlockCols * sizeof(float2));
    const uint32_t bytes_h = (uint32_t)(N * kBlockCols * sizeof(float2));

    auto issue = [&](int i) {           // thread 0: start the copies of item i
        const int kb = blockIdx.x + (i / d.n_imp) * gridDim.x, j = i % d.n_imp, s = i & 1;
        const int64_t blk = (int64_t)j * d.nkb + kb;
        mbar_arrive_expect_tx(&sm.bar[s], bytes_s + bytes_h);
        bulk_g2s(sm.st_s(s), shat + blk * d.n_w * kBlockCols, bytes_s, &sm.bar[s]);
        bulk_g2s(sm.st_h(s, d.n_w), H + blk * N * kBlockCols, bytes_h, &sm.bar[s]);
    };

    if (tid == 0) {
        mbar_init(&sm.bar[0], 1);
        mbar_init(&sm.bar[1], 1);
        fence_mbar_init();
    }
    const int plen = padded_len(N) * kBlockCols;
    for (int e = tid; e < plen; e += blockDim.x) sm.acc[e] = make_float2(0.f, 0.f);
    __syncthreads();
    if (tid == 0) {
        if (n_items > 0) issue(0);
        if (n_items > 1) issue(1);
    }

    int i = 0;
    for (; i < n_items; ++i) {
        const int s = i & 1, j = i % d.n_imp;
        const int kb = blockIdx.x + (i / d.n_imp) * gridDim.x;
        const bool landed = mbar_wait(&sm.bar[s], (i >> 1) & 1, d.wait_ns);
        if (!__syncthreads_and(landed)) break;
        const float2* z = run_plan<false, LOGB>(p, StagedTileLd{sm.st_s(s), d.n_w}, sm.X, sm.Y);
        const float2* h = sm.st_h(s, d.n_w);     // [4][N]
        for (int e = tid; e < N * kBlockCols; e += blockDim.x) {
            const int c = e & (kBlockCols - 1), kw = e >> LOGB;
            const int idx = (pad16(kw) << LOGB) + c;
            const float2 hv = h[c * N + kw], v = z[idx];
            float2 a = sm.acc[idx];
            a.x += hv.x * v.x - hv.y * v.y;
            a.y += hv.x * v.y + hv.y * v.x;
            sm.acc[idx] = a;
        }
        __syncthreads();                         // stage s is free again
        if (tid == 0 && i + 2 < n_items) {
            fence_proxy_async_smem();
            issue(i + 2);
        }
        if (j == d.n_imp - 1) {
            const float2* m = run_plan<true, LOGB>(p, SmemLd<LOGB>{sm.acc}, sm.X, sm.Y);
            float2* out = mt + (int64_t)kb * d.n_w * kBlockCols;
            for (int e = tid; e < d.n_w * kBlockCols; e += blockDim.x)
                out[e] = m[(pad16(e >> LOGB) << LOGB) + (e & (kBlockCols - 1))];
            for (int e = tid; e < plen; e += blockDim.x) sm.acc[e] = make_float2(0.f, 0.f);
            __syncthreads();
        }
    }
    if (i < n_items && tid == 0) {
        // a copy never landed: flag it, let what is still in flight finish, and leave
        atomicOr(flags, kErrTimeout);
        for (int k = i; k < n_items && k < i + 2; ++k) mbar_wait(&sm.bar[k & 1], (k >> 1) & 1);
    }
}

// Direct variant for planes too wide for the staged kernel's shared memory: one CTA per
// group of 2^LG time frequencies, the first wire pass reads global memory directly.
template <int LG>
struct BlockedColLd {
    const float2* src;   // Shat_j, blocked [nkb][n_w][4]
    int n_w, kt0;
    __device__ __forceinline__ float2 operator()(int c, int w) const
    {
        return (w < n_w) ? __ldg(src + blk_index(kt0 + c, w, n_w)) : make_float2(0.f, 0.f);
    }
};

template <int LG>
__global__ void __launch_bounds__(256, 1)
k_wire_direct(ConvDims d, FftPlan p, const float2* __restrict__ shat, const float2* __restrict__ H,
              float2* __restrict__ mt)
{
    constexpr int B = 1 << LG;
    extern __shared__ __align__(128) unsigned char smraw[];
    const int N = p.n;
    const int plen = padded_len(N) << LG;
    float2* X = reinterpret_cast<float2*>(smraw);
    float2* Y = X + plen;
    float2* acc = Y + plen;
    const int kt0 = blockIdx.x * B;        // B divides 4: a group never straddles blocks
    for (int e = threadIdx.x; e < plen; e += blockDim.x) acc[e] = make_float2(0.f, 0.f);
    for (int j = 0; j < d.n_imp; ++j) {
        const float2* sj = shat + (int64_t)j * d.nkb * d.n_w * kBlockCols;
        const float2* z = run_plan<false, LG>(p, BlockedColLd<LG>{sj, d.n_w, kt0}, X, Y);
        const float2* hj = H + (int64_t)j * d.nkb * N * kBlockCols;   // [4 nkb][N]
        for (int e = threadIdx.x; e < (N << LG); e += blockDim.x) {
            const int c = e & (B - 1), kw = e >> LG;
            const int idx = (pad16(kw) << LG) + c;
            const float2 hv = __ldg(hj + (int64_t)(kt0 + c) * N + kw), v = z[idx];
            float2 a = acc[idx];
            a.x += hv.x * v.x - hv.y * v.y;
            a.y += hv.x * v.y + hv.y * v.x;
            acc[idx] = a;
        }
        __syncthreads();
    }
    const float2* m = run_plan<true, LG>(p, SmemLd<LG>{acc}, X, Y);
    for (int e = threadIdx.x; e < (d.n_w << LG); e += blockDim.x) {
        const int c = e & (B - 1), w = e >> LG;
        mt[blk_index(kt0 + c, w, d.n_w)] = m[(pad16(w) << LG) + c];
    }
}

// First-pass source of the inverse wire FFT of the adjoint: conj(H_j(kt0 + c, kw)) G^(kw)
// for column c, G^ held in shared memory in the padded layout of a plan's output.
template <int LG>
struct ConjHGLd {
    const float2* hj;    // H_j's rows kt0 .. kt0 + 2^LG - 1 (time-frequency major, n_fw each)
    const float2* gh;
    int n_fw;
    __device__ __forceinline__ float2 operator()(int c, int kw) const
    {
        const float2 h = __ldg(hj + (int64_t)c * n_fw + kw);
        const float2 g = gh[(pad16(kw) << LG) + c];
        return make_float2(h.x * g.x + h.y * g.y, h.x * g.y - h.y * g.x);
    }
};

// Adjoint of the wire pass for any wire FFT size (the one-warp-per-column kernels of
// adjoint.cu take n_fw = 32 M): one CTA per group of 2^LG time frequencies.  G^ = the wire
// FFT of G's time-axis spectrum stays in shared memory; for every j the CTA transforms S_j's
// columns and writes dL/dR_j = conj(S^_j) G^ / (n_fw n_ft) at (kw, kt) and its mirror
// (-kw, -kt) (when dR is not null), then transforms conj(H_j) G^ back along the wires and
// writes it over S_j's columns (the time-axis spectrum of dL/dS_j).
template <int LG>
__global__ void __launch_bounds__(256, 1)
k_wire_adjoint_block(ConvDims d, FftPlan p, const float2* __restrict__ gt,
                     float2* __restrict__ shat, const float2* __restrict__ H,
                     float2* __restrict__ dR, float inv_n)
{
    constexpr int B = 1 << LG;
    extern __shared__ __align__(128) unsigned char smraw[];
    const int N = p.n;
    const int plen = padded_len(N) << LG;
    float2* X = reinterpret_cast<float2*>(smraw);
    float2* Y = X + plen;
    float2* gh = Y + plen;
    const int kt0 = blockIdx.x * B;        // B divides 4: a group never straddles blocks
    {
        const float2* z = run_plan<false, LG>(p, BlockedColLd<LG>{gt, d.n_w, kt0}, X, Y);
        for (int e = threadIdx.x; e < plen; e += blockDim.x) gh[e] = z[e];
        __syncthreads();
    }
    for (int j = 0; j < d.n_imp; ++j) {
        float2* sj = shat + (int64_t)j * d.nkb * d.n_w * kBlockCols;
        if (dR) {
            const float2* z = run_plan<false, LG>(p, BlockedColLd<LG>{sj, d.n_w, kt0}, X, Y);
            float2* dRj = dR + (int64_t)j * N * d.n_ft;
            for (int e = threadIdx.x; e < (N << LG); e += blockDim.x) {
                const int c = e & (B - 1), kw = e >> LG, kt = kt0 + c;
                if (kt >= d.nh) continue;
                const int idx = (pad16(kw) << LG) + c;
                const float2 u = z[idx], g = gh[idx];
                const float2 v = make_float2(inv_n * (u.x * g.x + u.y * g.y),
                                             inv_n * (u.x * g.y - u.y * g.x));
                dRj[(int64_t)kw * d.n_ft + kt] = v;
                if (kt >= 1 && d.n_ft - kt >= d.nh)
                    dRj[(int64_t)((N - kw) % N) * d.n_ft + (d.n_ft - kt)] = make_float2(v.x, -v.y);
            }
            __syncthreads();
        }
        const float2* hj = H + ((int64_t)j * d.nkb * kBlockCols + kt0) * N;
        const float2* m = run_plan<true, LG>(p, ConjHGLd<LG>{hj, gh, N}, X, Y);
        for (int e = threadIdx.x; e < (d.n_w << LG); e += blockDim.x) {
            const int c = e & (B - 1), w = e >> LG;
            sj[blk_index(kt0 + c, w, d.n_w)] = m[(pad16(w) << LG) + c];
        }
        __syncthreads();
    }
}

// H[j][kt][kw] = scale (R_j[kw][kt] + conj R_j[-kw][-kt]) / 2 for kt < nh, zero for the
// padding rows nh <= kt < 4 nkb.  A 32 x 32 tile of (kw, kt) per CTA, transposed through
// shared memory so that both the reads of R (along kt) and the writes of H (along kw) are
// coalesced.  grid (ceil(4 nkb / 32), ceil(n_fw / 32), n_imp), block (32, 8).
__global__ void k_make_hermitian(ConvDims d, const float2* __restrict__ R, float2* __restrict__ H,
                                 float scale)
{
    __shared__ float2 tile[32][33];
    const int j = blockIdx.z, kt0 = blockIdx.x * 32, kw0 = blockIdx.y * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int n_kt = d.nkb * kBlockCols;
    const float f = 0.5f * scale;
    const float2* Rj = R + (int64_t)j * d.n_fw * d.n_ft;
    for (int i = ty; i < 32; i += blockDim.y) {
        const int kw = kw0 + i, kt = kt0 + tx;
        float2 h = make_float2(0.f, 0.f);
        if (kw < d.n_fw && kt < d.nh) {
            const float2 a = Rj[(int64_t)kw * d.n_ft + kt];
            const int kwm = (d.n_fw - kw) % d.n_fw, ktm = (d.n_ft - kt) % d.n_ft;
            const float2 b = Rj[(int64_t)kwm * d.n_ft + ktm];
            h = make_float2(f * (a.x + b.x), f * (a.y - b.y));
        }
        tile[i][tx] = h;
    }
    __syncthreads();
    float2* Hj = H + (int64_t)j * n_kt * d.n_fw;
    for (int i = ty; i < 32; i += blockDim.y) {
        const int kt = kt0 + i, kw = kw0 + tx;
        if (kt < n_kt && kw < d.n_fw) Hj[(int64_t)kt * d.n_fw + kw] = tile[tx][i];
    }
}

DeviceOnce g_attr;

}  // namespace

int sm_count()
{
    static int n[64] = {};                 // per device ordinal
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 1;
    if (n[dev] == 0) {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0)
            v = 1;
        n[dev] = v;
    }
    return n[dev];
}

cudaError_t launch_make_hermitian(const ConvDims& d, const float2* resp, float2* H, float scale,
                                  cudaStream_t s)
{
    const dim3 grid((unsigned)((d.nkb * kBlockCols + 31) / 32), (unsigned)((d.n_fw + 31) / 32),
                    (unsigned)d.n_imp);
    k_make_hermitian<<<grid, dim3(32, 8), 0, s>>>(d, resp, H, scale);
    return cudaGetLastError();
}

constexpr size_t kMaxSmem = 227 * 1024;

cudaError_t launch_wire_pass(const ConvDims& d, const FftPlan& pw, const float2* shat,
                             const float2* H, float2* mt, int* flags, cudaStream_t s)
{
    if (g_attr.pending()) {
        cudaError_t e = cudaFuncSetAttribute(k_wire_pass, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMaxSmem);
        if (!e) e = cudaFuncSetAttribute(k_wire_direct<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMaxSmem);
        if (!e) e = cudaFuncSetAttribute(k_wire_direct<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMaxSmem);
        if (e) return e;
        g_attr.mark();
    }
    const size_t staged = wire_smem_bytes(d.n_w, pw.n);
    if (staged <= kMaxSmem) {
        const int grid = d.nkb < sm_count() ? d.nkb : sm_count();
        k_wire_pass<<<grid, kThreads, staged, s>>>(d, pw, shat, H, mt, flags);
    } else if (3 * (size_t)(padded_len(pw.n) << 2) * sizeof(float2) <= kMaxSmem) {
        k_wire_direct<2><<<d.nkb, 256, 3 * (size_t)(padded_len(pw.n) << 2) * sizeof(float2), s>>>(
            d, pw, shat, H, mt);
    } else {
        k_wire_direct<0><<<d.nkb * kBlockCols, 256, 3 * (size_t)padded_len(pw.n) * sizeof(float2), s>>>(
            d, pw, shat, H, mt);
    }
    return cudaGetLastError();
}

cudaError_t launch_wire_adjoint_block(const ConvDims& d, const FftPlan& pw, const float2* gt,
                                      float2* shat, const float2* H, float2* dR, float inv_n,
                                      cudaStream_t s)
{
    static DeviceOnce attr;
    if (attr.pending()) {
        cudaError_t e = cudaFuncSetAttribute(k_wire_adjoint_block<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMaxSmem);
        if (!e) e = cudaFuncSetAttribute(k_wire_adjoint_block<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMaxSmem);
        if (e) return e;
        attr.mark();
    }
    const size_t four = 3 * (size_t)(padded_len(pw.n) << 2) * sizeof(float2);
    const size_t one = 3 * (size_t)padded_len(pw.n) * sizeof(float2);
    if (four <= kMaxSmem)
        k_wire_adjoint_block<2><<<d.nkb, 256, four, s>>>(d, pw, gt, shat, H, dR, inv_n);
    else if (one <= kMaxSmem)
        k_wire_adjoint_block<0><<<d.nkb * kBlockCols, 256, one, s>>>(d, pw, gt, shat, H, dR, inv_n);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

}  // namespace wcsim
