// Time-axis transforms of Eq. 2: forward real-to-complex FFT of every grid row and inverse
// complex-to-real FFT of every wire's spectrum.  Two real rows ride in one complex FFT
// (z = x0 + i x1); their spectra are separated with X0 = (Z[k] + conj Z[-k]) / 2,
// X1 = (Z[k] - conj Z[-k]) / 2i.  One CTA per pair of rows, two padded N-point buffers in
// shared memory, the first pass reads global memory directly.
#include <cuda_runtime.h>
#include <stdint.h>

#include "fft_engine.cuh"
#include "wcsim_internal.cuh"

namespace wcsim {
namespace {

constexpr int kThreads = 256;

// First-pass source: element i of z = x0 + i x1 (zero beyond the frame).
struct RealPairLd {
    const float* g0;
    const float* g1;      // nullptr: second row absent
    int n_t;
    __device__ __forceinline__ float2 operator()(int, int i) const
    {
        if (i >= n_t) return make_float2(0.f, 0.f);
        return make_float2(__ldg(g0 + i), g1 ? __ldg(g1 + i) : 0.f);
    }
};

// First-pass source of the inverse: z[i] = X0[i] + i X1[i], both Hermitian, from the
// stored half spectra m0, m1 (k < nh), conj(m[N - k]) above.
struct HermPairLd {
    const float2* m0;
    const float2* m1;     // nullptr: second wire absent
    int nh, n;
    __device__ __forceinline__ float2 operator()(int, int k) const
    {
        float2 a, b = make_float2(0.f, 0.f);
        if (k < nh) {
            a = __ldg(m0 + k);
            if (m1) b = __ldg(m1 + k);
        } else {
            const float2 ac = __ldg(m0 + (n - k));
            a = make_float2(ac.x, -ac.y);
            if (m1) {
                const float2 bc = __ldg(m1 + (n - k));
                b = make_float2(bc.x, -bc.y);
            }
        }
        return make_float2(a.x - b.y, a.y + b.x);
    }
};

__global__ void __launch_bounds__(kThreads, 2)
k_rows_r2c(ConvDims d, FftPlan p, const float* __restrict__ grid, float2* __restrict__ shat)
{
    extern __shared__ float2 sm[];
    const int N = p.n;
    float2* X = sm;
    float2* Y = sm + padded_len(N);
    const int64_t n_rows = (int64_t)d.n_w * d.n_imp;
    const int64_t r0 = 2 * (int64_t)blockIdx.x, r1 = r0 + 1;
    const bool has1 = r1 < n_rows;
    const RealPairLd src{grid + r0 * d.n_t, has1 ? grid + r1 * d.n_t : nullptr, d.n_t};
    const float2* z = run_plan<false, 0>(p, src, X, Y);
    const int w0 = (int)(r0 / d.n_imp), j0 = (int)(r0 % d.n_imp);
    const int w1 = (int)(r1 / d.n_imp), j1 = (int)(r1 % d.n_imp);
    float2* o0 = shat + ((int64_t)j0 * d.n_w + w0) * d.nh;
    float2* o1 = shat + ((int64_t)j1 * d.n_w + w1) * d.nh;
    for (int k = threadIdx.x; k < d.nh; k += blockDim.x) {
        const float2 a = z[pad16(k)];
        const float2 b = z[pad16(k == 0 ? 0 : N - k)];
        o0[k] = make_float2(0.5f * (a.x + b.x), 0.5f * (a.y - b.y));
        if (has1) o1[k] = make_float2(0.5f * (a.y + b.y), 0.5f * (b.x - a.x));
    }
}

__global__ void __launch_bounds__(kThreads, 2)
k_rows_c2r(ConvDims d, FftPlan p, const float2* __restrict__ mt, float* __restrict__ wave)
{
    extern __shared__ float2 sm[];
    const int N = p.n;
    float2* X = sm;
    float2* Y = sm + padded_len(N);
    const int w0 = 2 * blockIdx.x, w1 = w0 + 1;
    const bool has1 = w1 < d.n_w;
    const HermPairLd src{mt + (int64_t)w0 * d.nh, has1 ? mt + (int64_t)w1 * d.nh : nullptr,
                         d.nh, N};
    const float2* z = run_plan<true, 0>(p, src, X, Y);
    float* o0 = wave + (int64_t)w0 * d.n_t;
    float* o1 = wave + (int64_t)w1 * d.n_t;
    for (int t = threadIdx.x; t < d.n_t; t += blockDim.x) {
        const float2 v = z[pad16(t)];
        o0[t] = v.x;
        if (has1) o1[t] = v.y;
    }
}

size_t rows_smem(int n) { return 2 * (size_t)padded_len(n) * sizeof(float2); }

bool g_attr = false;
cudaError_t attrs()
{
    if (g_attr) return cudaSuccess;
    const int mx = 227 * 1024;
    cudaError_t e = cudaFuncSetAttribute(k_rows_r2c, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    if (!e) e = cudaFuncSetAttribute(k_rows_c2r, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    if (!e) g_attr = true;
    return e;
}

}  // namespace

cudaError_t launch_rows_r2c(const ConvDims& d, const FftPlan& pt, const float* grid,
                            float2* shat, cudaStream_t s)
{
    cudaError_t e = attrs();
    if (e) return e;
    const int64_t n_rows = (int64_t)d.n_w * d.n_imp;
    k_rows_r2c<<<(unsigned)((n_rows + 1) / 2), kThreads, rows_smem(pt.n), s>>>(d, pt, grid, shat);
    return cudaGetLastError();
}

cudaError_t launch_rows_c2r(const ConvDims& d, const FftPlan& pt, const float2* mt,
                            float* wave, cudaStream_t s)
{
    cudaError_t e = attrs();
    if (e) return e;
    k_rows_c2r<<<(unsigned)((d.n_w + 1) / 2), kThreads, rows_smem(pt.n), s>>>(d, pt, mt, wave);
    return cudaGetLastError();
}

}  // namespace wcsim
