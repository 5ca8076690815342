// Wire-axis part of Eq. 2 with one warp per time frequency.
//
// n_fw = 32 M.  A warp owns column kt of the blocked spectra; lane l holds the M wires
// w = l + 32 m.  Forward: X[k2 + M k1] = sum_l W32^(l k1) W^(l k2) sum_m x[l + 32 m] WM^(m k2):
// an M-point DFT in each lane's registers, the twiddle W^(l k2), a transpose through a
// padded per-warp shared tile, and a 32-point DFT in the registers of lanes k2 < M.  Lane k2
// then holds X[k2 + M k1] for all 32 k1, multiplies by H_j and accumulates over j in
// registers.  The inverse runs the same steps backwards (32-point DFT per lane, twiddle,
// transpose, M-point DFT per lane) and leaves wire w = l + 32 n1 in lane l.  The only
// synchronisation is __syncwarp around the transposes.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <vector>

#include "fft_engine.cuh"
#include "wcsim_internal.cuh"

namespace wcsim {
namespace {

constexpr int kWarps = 4;            // = kBlockCols: warp c takes column c of a block

template <int M>
__global__ void __launch_bounds__(kWarps * 32, 3)
k_wire_warp(ConvDims d, const float2* __restrict__ tw2, const float2* __restrict__ shat,
            const float2* __restrict__ H, float2* __restrict__ mt)
{
    constexpr int N = 32 * M;
    constexpr int TR = (33 * M > 32 * (M + 1)) ? 33 * M : 32 * (M + 1);
    __shared__ float2 s_twf[N];          // W^(l k2) at k2 * 32 + l
    __shared__ float2 s_twi[N];          // W^(k2 n2) at n2 * M + k2
    __shared__ float2 s_tr[kWarps][TR];
    for (int e = threadIdx.x; e < N; e += blockDim.x) {
        s_twf[e] = tw2[e];
        s_twi[e] = tw2[N + e];
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // grid (events, blocks): the events of one block run side by side and share H's tiles
    const int kb = blockIdx.y, c = warp;
    shat += blockIdx.x * d.ev_shat;
    mt += blockIdx.x * d.ev_mt;
    float2* tr = s_tr[warp];
    float2 acc[32];
#pragma unroll
    for (int k1 = 0; k1 < 32; ++k1) acc[k1] = make_float2(0.f, 0.f);

    for (int j = 0; j < d.n_imp; ++j) {
        const int64_t blk = (int64_t)j * d.nkb + kb;
        const float2* src = shat + blk * d.n_w * kBlockCols + c;
        float2 v[M];
#pragma unroll
        for (int m = 0; m < M; ++m) {
            const int w = lane + 32 * m;
            v[m] = (w < d.n_w) ? __ldg(src + (int64_t)w * kBlockCols) : make_float2(0.f, 0.f);
        }
        dft<M, false>(v);
#pragma unroll
        for (int k2 = 1; k2 < M; ++k2) v[k2] = cmul(v[k2], s_twf[k2 * 32 + lane]);
#pragma unroll
        for (int k2 = 0; k2 < M; ++k2) tr[k2 * 33 + lane] = v[k2];
        __syncwarp();
        if (lane < M) {
            float2 u[32];
#pragma unroll
            for (int l = 0; l < 32; ++l) u[l] = tr[lane * 33 + l];
            dft<32, false>(u);
            const float2* hj = H + blk * N * kBlockCols + c;
#pragma unroll
            for (int k1 = 0; k1 < 32; ++k1) {
                const float2 h = __ldg(hj + (int64_t)(lane + M * k1) * kBlockCols);
                acc[k1].x += h.x * u[k1].x - h.y * u[k1].y;
                acc[k1].y += h.x * u[k1].y + h.y * u[k1].x;
            }
        }
        __syncwarp();
    }

    // inverse along the wire axis: lane k2 holds X[k2 + M k1]
    if (lane < M) {
        dft<32, true>(acc);
#pragma unroll
        for (int n2 = 1; n2 < 32; ++n2) acc[n2] = twiddle<true>(acc[n2], s_twi[n2 * M + lane]);
#pragma unroll
        for (int n2 = 0; n2 < 32; ++n2) tr[n2 * (M + 1) + lane] = acc[n2];
    }
    __syncwarp();
    float2 v[M];
#pragma unroll
    for (int k2 = 0; k2 < M; ++k2) v[k2] = tr[lane * (M + 1) + k2];
    dft<M, true>(v);
    float2* out = mt + (int64_t)kb * d.n_w * kBlockCols + c;
#pragma unroll
    for (int n1 = 0; n1 < M; ++n1) {
        const int w = lane + 32 * n1;
        if (w < d.n_w) out[(int64_t)w * kBlockCols] = v[n1];
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
                             const float2* H, float2* mt, cudaStream_t s, int n_ev)
{
    const dim3 grid((unsigned)n_ev, (unsigned)d.nkb);
    switch (d.n_fw / 32) {
#define WCSIM_CASE(MM) \
    case MM: k_wire_warp<MM><<<grid, kWarps * 32, 0, s>>>(d, tw2, shat, H, mt); break;
        WCSIM_WARP_M(WCSIM_CASE)
#undef WCSIM_CASE
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace wcsim
