// Adjoint of the Eq. 2 convolution.
//
// The forward computes M = IFFT2(sum_j H_j FFT2(S_j)) with H_j the Hermitian part of R_j
// (scaled by 1/(n_fw n_ft)).  For a loss L with G = dL/dM:
//   dL/dS_j = IFFT2(conj(H_j) FFT2(G))                (same unnormalised inverse, same scale)
//   dL/dR_j = conj(FFT2(S_j)) FFT2(G) / (n_fw n_ft)    (complex-gradient convention dRe + i dIm)
// wire_adjoint_warp: one warp per time frequency kt (n_fw = 32 M, the layout of the forward
// warp kernel).  It transforms the column of G's time-axis spectrum along the wires once,
// then for every j transforms S_j's column, writes dL/dR_j at (kw, kt) and its Hermitian
// mirror (-kw, -kt), forms conj(H_j) G^ and transforms it back along the wires, overwriting
// S_j's column with the time-axis spectrum of dL/dS_j.
// rows_c2r_grid: the inverse time-axis FFT of those spectra for every grid row.
#include <cuda_runtime.h>
#include <stdint.h>

#include "fft_engine.cuh"
#include "wcsim_internal.cuh"

namespace wcsim {
namespace {

constexpr int kWarps = 4;

// Forward wire FFT of one column of a blocked spectrum: lane l loads wires l + 32 m; after
// the call lanes k2 < M hold X[k2 + M k1] in u[k1].
template <int M>
__device__ __forceinline__ void warp_wire_fft(const float2* __restrict__ col, int n_w,
                                              const float2* s_twf, float2* tr, int lane,
                                              float2 (&u)[32])
{
    float2 v[M];
#pragma unroll
    for (int m = 0; m < M; ++m) {
        const int w = lane + 32 * m;
        v[m] = (w < n_w) ? __ldg(col + (int64_t)w * kBlockCols) : make_float2(0.f, 0.f);
    }
    dft<M, false>(v);
#pragma unroll
    for (int k2 = 1; k2 < M; ++k2) v[k2] = cmul(v[k2], s_twf[k2 * 32 + lane]);
    __syncwarp();
#pragma unroll
    for (int k2 = 0; k2 < M; ++k2) tr[k2 * 33 + lane] = v[k2];
    __syncwarp();
    if (lane < M) {
#pragma unroll
        for (int l = 0; l < 32; ++l) u[l] = tr[lane * 33 + l];
        dft<32, false>(u);
    }
}

template <int M>
__global__ void __launch_bounds__(kWarps * 32, 2)
k_wire_adjoint_warp(ConvDims d, const float2* __restrict__ tw2, const float2* __restrict__ gt,
                    float2* __restrict__ shat, const float2* __restrict__ H, float2* __restrict__ dR,
                    float inv_n)
{
    constexpr int N = 32 * M;
    constexpr int TR = (33 * M > 32 * (M + 1)) ? 33 * M : 32 * (M + 1);
    __shared__ float2 s_twf[N];
    __shared__ float2 s_twi[N];
    __shared__ float2 s_tr[kWarps][TR];
    for (int e = threadIdx.x; e < N; e += blockDim.x) {
        s_twf[e] = tw2[e];
        s_twi[e] = tw2[N + e];
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int kb = blockIdx.x, c = warp, kt = kb * kBlockCols + c;
    float2* tr = s_tr[warp];

    float2 g[32];                           // G^(kw = lane + M k1, kt), lanes < M
    warp_wire_fft<M>(gt + (int64_t)kb * d.n_w * kBlockCols + c, d.n_w, s_twf, tr, lane, g);
    const bool dr_here = (dR != nullptr) && (kt < d.nh);
    const bool mirror = dr_here && kt >= 1 && (d.n_ft - kt) >= d.nh;

    for (int j = 0; j < d.n_imp; ++j) {
        const int64_t blk = (int64_t)j * d.nkb + kb;
        float2* col = shat + blk * d.n_w * kBlockCols + c;
        float2 u[32];
        warp_wire_fft<M>(col, d.n_w, s_twf, tr, lane, u);
        if (lane < M) {
            const float2* hj = H + blk * N * kBlockCols + c;
#pragma unroll
            for (int k1 = 0; k1 < 32; ++k1) {
                const int kw = lane + M * k1;
                if (dr_here) {
                    // conj(S^) G^ / n
                    const float2 val = make_float2(inv_n * (u[k1].x * g[k1].x + u[k1].y * g[k1].y),
                                                   inv_n * (u[k1].x * g[k1].y - u[k1].y * g[k1].x));
                    float2* dRj = dR + (int64_t)j * N * d.n_ft;
                    dRj[(int64_t)kw * d.n_ft + kt] = val;
                    if (mirror)
                        dRj[(int64_t)((N - kw) % N) * d.n_ft + (d.n_ft - kt)] = make_float2(val.x, -val.y);
                }
                // conj(H_j) G^
                const float2 h = __ldg(hj + (int64_t)kw * kBlockCols);
                u[k1] = make_float2(h.x * g[k1].x + h.y * g[k1].y, h.x * g[k1].y - h.y * g[k1].x);
            }
            dft<32, true>(u);
#pragma unroll
            for (int n2 = 1; n2 < 32; ++n2) u[n2] = twiddle<true>(u[n2], s_twi[n2 * M + lane]);
        }
        __syncwarp();
        if (lane < M) {
#pragma unroll
            for (int n2 = 0; n2 < 32; ++n2) tr[n2 * (M + 1) + lane] = u[n2];
        }
        __syncwarp();
        float2 v[M];
#pragma unroll
        for (int k2 = 0; k2 < M; ++k2) v[k2] = tr[lane * (M + 1) + k2];
        dft<M, true>(v);
#pragma unroll
        for (int n1 = 0; n1 < M; ++n1) {
            const int w = lane + 32 * n1;
            if (w < d.n_w) col[(int64_t)w * kBlockCols] = v[n1];
        }
    }
}

// First-pass source of the inverse time FFT of grid rows r0, r1 (wire w, impact j each):
// z[k] = X0[k] + i X1[k] from the blocked half spectra.
struct GridHermPairLd {
    const float2* s0;     // blocked slab of row r0's impact position
    const float2* s1;
    int w0, w1, n_w, nh, n;
    bool has1;
    __device__ __forceinline__ float2 operator()(int, int k) const
    {
        const bool lo = k < nh;
        const int kk = lo ? k : n - k;
        float2 a = __ldg(s0 + blk_index(kk, w0, n_w));
        float2 b = has1 ? __ldg(s1 + blk_index(kk, w1, n_w)) : make_float2(0.f, 0.f);
        if (!lo) {
            a.y = -a.y;
            b.y = -b.y;
        }
        return make_float2(a.x - b.y, a.y + b.x);
    }
};

__global__ void __launch_bounds__(256, 2)
k_rows_c2r_grid(ConvDims d, FftPlan p, const float2* __restrict__ shat, float* __restrict__ grid)
{
    extern __shared__ __align__(128) unsigned char smraw[];
    const int N = p.n;
    float2* X = reinterpret_cast<float2*>(smraw);
    float2* Y = X + padded_len(N);
    const int64_t n_rows = (int64_t)d.n_w * d.n_imp;
    const int64_t r0 = 2 * (int64_t)blockIdx.x, r1 = r0 + 1;
    const bool has1 = r1 < n_rows;
    const int w0 = (int)(r0 / d.n_imp), j0 = (int)(r0 % d.n_imp);
    const int w1 = has1 ? (int)(r1 / d.n_imp) : w0, j1 = has1 ? (int)(r1 % d.n_imp) : j0;
    const int64_t slab = (int64_t)d.nkb * d.n_w * kBlockCols;
    const GridHermPairLd src{shat + j0 * slab, shat + j1 * slab, w0, w1, d.n_w, d.nh, N, has1};
    const float2* z = run_plan<true, 0>(p, src, X, Y);
    float* o0 = grid + r0 * d.n_t;
    float* o1 = grid + r1 * d.n_t;
    for (int t = threadIdx.x; t < d.n_t; t += blockDim.x) {
        const float2 v = z[pad16(t)];
        o0[t] = v.x;
        if (has1) o1[t] = v.y;
    }
}

#define WCSIM_ADJ_M(X) X(4) X(8) X(15) X(16) X(20) X(24) X(25) X(30)

bool g_attr = false;

}  // namespace

cudaError_t launch_wire_adjoint_warp(const ConvDims& d, const float2* tw2, const float2* gt,
                                     float2* shat, const float2* H, float2* dR, float inv_n,
                                     cudaStream_t s)
{
    switch (d.n_fw / 32) {
#define WCSIM_CASE(MM)                                                                       \
    case MM:                                                                                 \
        k_wire_adjoint_warp<MM><<<d.nkb, kWarps * 32, 0, s>>>(d, tw2, gt, shat, H, dR, inv_n); \
        break;
        WCSIM_ADJ_M(WCSIM_CASE)
#undef WCSIM_CASE
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_rows_c2r_grid(const ConvDims& d, const FftPlan& pt, const float2* shat,
                                 float* grid, cudaStream_t s)
{
    if (!g_attr) {
        cudaError_t e = cudaFuncSetAttribute(k_rows_c2r_grid, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             227 * 1024);
        if (e) return e;
        g_attr = true;
    }
    const int64_t n_rows = (int64_t)d.n_w * d.n_imp;
    k_rows_c2r_grid<<<(unsigned)((n_rows + 1) / 2), 256, 2 * (size_t)padded_len(pt.n) * sizeof(float2), s>>>(
        d, pt, shat, grid);
    return cudaGetLastError();
}

}  // namespace wcsim
