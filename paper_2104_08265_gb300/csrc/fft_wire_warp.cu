// Wire-axis part of Eq. 2 with one warp per time frequency.
//
// n_fw = 32 M.  A warp owns column kt of the blocked spectra; lane l holds the M wires
// w = l + 32 m.  Forward: X[k2 + M k1] = sum_l W32^(l k1) W^(l k2) sum_m x[l + 32 m] WM^(m k2):
// an M-point DFT in each lane's registers, the twiddle W^(l k2), a transpose through a
// padded per-warp shared tile, and a 32-point DFT in the registers of lanes k2 < M.  Lane k2
// then holds X[k2 + M k1] for all 32 k1, multiplies by H_j and accumulates over j in
// registers.  The inverse runs the same steps backwards (32-point DFT per lane, twiddle,
// transpose, M-point DFT per lane) and leaves wire w = l + 32 n1 in lane l.
//
// Data movement.  S_j's column is loaded by each lane straight into registers (all M loads
// in flight).  H_j's tile (the CTA's 4 columns, one contiguous 30 KB block for n_fw = 960)
// is brought into shared memory by one bulk asynchronous copy on an mbarrier: the copy of
// H_{j+1} is issued as soon as every warp has used H_j, so it lands while the warps load and
// transform S_{j+1}.  Every wait is bounded in time; a wait that runs out raises the timeout
// flag and the CTA leaves.  The result leaves through shared memory as 16-byte stores.  In
// the S2D instance (fit steps) each warp also stores its S_j column's wire spectrum.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <vector>

#include "async_copy.cuh"
#include "fft_engine.cuh"
#include "warp_fft.cuh"
#include "wcsim_internal.cuh"

namespace wcsim {
namespace {

// A CTA takes CW of the 4 columns of a block, one warp per column (CW = 2: the 751 blocks of
// a 6000-tick plane become 1502 CTAs, which fill whole waves of the 5 CTAs that fit an SM).
constexpr int kCols = 2;

template <int M, int CW>
constexpr size_t warp_smem() { return (size_t)32 * M * CW * sizeof(float2) + 16; }

// S2D: the 2D spectra of S (the wire FFT of every Shat_j column, before the product with H_j)
// are also written to s2d, time-frequency major [n_imp][4 nkb][n_fw] (the layout of H): each
// warp stores its column from registers, consecutive lanes on consecutive wire frequencies,
// for an adjoint that takes dL/dR from them (wcsim_plane_set_reuse_forward mode 2).
template <int M, int CW, bool S2D>
__global__ void __launch_bounds__(CW * 32, CW == 4 ? 3 : 5)
k_wire_warp(ConvDims d, const float2* __restrict__ tw2, const float2* __restrict__ shat,
            const float2* __restrict__ H, float2* __restrict__ mt, int* flags,
            float2* __restrict__ s2d)
{
    static_assert(CW == 2 || CW == 4, "columns per CTA");
    constexpr int N = 32 * M;
    constexpr int TR = (33 * M > 32 * (M + 1)) ? 33 * M : 32 * (M + 1);
    constexpr uint32_t kTileBytes = N * CW * sizeof(float2);
    __shared__ float2 s_twf[N];          // W^(l k2) at k2 * 32 + l
    __shared__ float2 s_tr[CW][TR];
    // dynamic: H_j's tile [CW][n] (one column per warp, read without bank conflicts); after
    // the j loop the inverse twiddles, then the output columns [CW][n]; an mbarrier behind it
    extern __shared__ __align__(128) unsigned char smraw[];
    float2* s_h = reinterpret_cast<float2*>(smraw);
    uint64_t* bar = reinterpret_cast<uint64_t*>(s_h + N * CW);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // grid (events, blocks x parts): the events of one block run side by side and share H's
    // tiles; columns c0 .. c0 + CW - 1 of block kb
    constexpr int kParts = kBlockCols / CW;
    const int kb = blockIdx.y / kParts, c0 = (blockIdx.y % kParts) * CW, c = c0 + warp;
    shat += blockIdx.x * d.ev_shat;
    mt += blockIdx.x * d.ev_mt;
    // rows 4 kb + c0 .. of H_j (time-frequency major): one contiguous tile
    auto h_tile = [&](int64_t blk) { return H + (blk * kBlockCols + c0) * N; };
    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
        mbar_arrive_expect_tx(bar, kTileBytes);
        bulk_g2s(s_h, h_tile(kb), kTileBytes, bar);
    }
    for (int e = threadIdx.x; e < N; e += blockDim.x) s_twf[e] = tw2[e];
    __syncthreads();
    float2* tr = s_tr[warp];
    float2 acc[32];
#pragma unroll
    for (int k1 = 0; k1 < 32; ++k1) acc[k1] = make_float2(0.f, 0.f);

    for (int j = 0; j < d.n_imp; ++j) {
        const int64_t blk = (int64_t)j * d.nkb + kb;
        float2 u[32];
        bool landed;
        {
            float2 v[M];
            load_col<M>(shat + blk * d.n_w * kBlockCols, c, d.n_w, lane, v);
            landed = mbar_wait(bar, j & 1, d.wait_ns);   // H_j's tile, copied while S_j loads
            warp_fft_fwd<M>(v, s_twf, tr, lane, u);
        }
        if (lane < M) {
            if (landed) {
#pragma unroll
                for (int k1 = 0; k1 < 32; ++k1) {
                    const float2 h = s_h[warp * N + lane + M * k1];
                    acc[k1].x += h.x * u[k1].x - h.y * u[k1].y;
                    acc[k1].y += h.x * u[k1].y + h.y * u[k1].x;
                }
            }
            if constexpr (S2D) {
                // S_j's 2D spectrum in column 4 kb + c: lane k2 < M holds kw = k2 + M k1
                float2* col = s2d + ((int64_t)j * kBlockCols * d.nkb + kb * kBlockCols + c) * N;
#pragma unroll
                for (int k1 = 0; k1 < 32; ++k1) __stcs(col + lane + M * k1, u[k1]);
            }
        }
        // every warp is done with s_h (and its transpose tile)
        if (__syncthreads_or(!landed)) {
            if (threadIdx.x == 0) {
                atomicOr(flags, kErrTimeout);
                mbar_wait(bar, j & 1);           // the copy still in flight, bounded
            }
            return;
        }
        if (threadIdx.x == 0 && j + 1 < d.n_imp) {
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(bar, kTileBytes);
            bulk_g2s(s_h, h_tile(blk + d.nkb), kTileBytes, bar);
        }
    }

    // inverse along the wire axis: lane k2 holds X[k2 + M k1]
    float2* s_twi = s_h;                         // W^(k2 n2) at n2 * M + k2
    for (int e = threadIdx.x; e < N; e += blockDim.x) s_twi[e] = tw2[N + e];
    __syncthreads();
    float2 v[M];
    warp_fft_inv<M>(acc, s_twi, tr, lane, v);
    __syncthreads();                             // s_twi is read out
#pragma unroll
    for (int n1 = 0; n1 < M; ++n1) {
        const int w = lane + 32 * n1;
        if (w < d.n_w) s_h[warp * N + w] = v[n1];
    }
    __syncthreads();
    float2* out = mt + (int64_t)kb * d.n_w * kBlockCols;
    if constexpr (CW == 4) {
        store_tile_cols(s_h, d.n_w, N, out);
    } else {
        for (int w = threadIdx.x; w < d.n_w; w += blockDim.x) {
            const float2 a = s_h[w], b = s_h[N + w];
            *reinterpret_cast<float4*>(out + (int64_t)w * kBlockCols + c0) = make_float4(a.x, a.y, b.x, b.y);
        }
    }
}

#define WCSIM_WARP_M(X) X(4) X(8) X(15) X(16) X(20) X(24) X(25) X(30)

}  // namespace

bool wire_warp_supported(int n_fw)
{
    if (n_fw % 32) return false;
    switch (n_fw / 32) {
#define WCSIM_CASE(MM) case MM:
        WCSIM_WARP_M(WCSIM_CASE)
#undef WCSIM_CASE
        return true;
        default: return false;
    }
}

cudaError_t wire_warp_twiddles(int n_fw, float2** dev)
{
    const int M = n_fw / 32;
    std::vector<float2> t(2 * (size_t)n_fw);
    for (int a = 0; a < M; ++a)
        for (int b = 0; b < 32; ++b) {
            const double ang = -2.0 * M_PI * (double)((int64_t)a * b % n_fw) / n_fw;
            const float2 w = make_float2((float)cos(ang), (float)sin(ang));
            t[(size_t)a * 32 + b] = w;
            t[n_fw + (size_t)b * M + a] = w;
        }
    cudaError_t e = cudaMalloc(dev, t.size() * sizeof(float2));
    if (e) return e;
    e = cudaMemcpy(*dev, t.data(), t.size() * sizeof(float2), cudaMemcpyHostToDevice);
    if (e) { cudaFree(*dev); *dev = nullptr; }
    return e;
}

cudaError_t launch_wire_warp(const ConvDims& d, const float2* tw2, const float2* shat,
                             const float2* H, float2* mt, int* flags, cudaStream_t s, int n_ev,
                             float2* s2d)
{
    const dim3 grid((unsigned)n_ev, (unsigned)(d.nkb * (kBlockCols / kCols)));
    if (s2d && n_ev != 1) return cudaErrorInvalidValue;
    switch (d.n_fw / 32) {
#define WCSIM_CASE(MM)                                                                         \
    case MM: {                                                                                 \
        static DeviceOnce attr_set;                                                            \
        if (attr_set.pending()) {                                                              \
            cudaError_t e = cudaFuncSetAttribute(k_wire_warp<MM, kCols, false>,                \
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize,  \
                                                 (int)warp_smem<MM, kCols>());                 \
            if (!e) e = cudaFuncSetAttribute(k_wire_warp<MM, kCols, true>,                     \
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,      \
                                             (int)warp_smem<MM, kCols>());                 \
            if (e) return e;                                                                   \
            attr_set.mark();                                                                   \
        }                                                                                      \
        if (s2d)                                                                               \
            k_wire_warp<MM, kCols, true><<<grid, kCols * 32, warp_smem<MM, kCols>(), s>>>(     \
                d, tw2, shat, H, mt, flags, s2d);                                              \
        else                                                                                   \
            k_wire_warp<MM, kCols, false><<<grid, kCols * 32, warp_smem<MM, kCols>(), s>>>(    \
                d, tw2, shat, H, mt, flags, nullptr);                                          \
        break;                                                                                 \
    }
        WCSIM_WARP_M(WCSIM_CASE)
#undef WCSIM_CASE
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace wcsim
