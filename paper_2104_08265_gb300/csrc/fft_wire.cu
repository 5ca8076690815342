// Wire-axis part of Eq. 2 and the response preparation.
//
// wire_pass: a CTA owns B = 2^LOGB adjacent time frequencies.  For each impact position j
// it transforms the B columns Shat_j[.][kt] along the wire axis (first pass straight from
// global memory), multiplies them by H_j and accumulates over j in shared memory; the sum is
// transformed back along the wire axis and written as Mt[w][kt].
#include <cuda_runtime.h>
#include <stdint.h>

#include "fft_engine.cuh"
#include "wcsim_internal.cuh"

namespace wcsim {
namespace {

constexpr int kThreads = 256;

// First-pass source: column kt0 + c of Shat_j, zero beyond the frame's wires or the
// half spectrum.
struct TileLd {
    const float2* src;    // Shat_j, [n_w][nh]
    int nh, kt0, n_w;
    __device__ __forceinline__ float2 operator()(int c, int w) const
    {
        const int kt = kt0 + c;
        return (w < n_w && kt < nh) ? __ldg(src + (int64_t)w * nh + kt) : make_float2(0.f, 0.f);
    }
};

template <int LOGB>
__global__ void __launch_bounds__(kThreads, 2)
k_wire_pass(ConvDims d, FftPlan p, const float2* __restrict__ shat, const float2* __restrict__ H,
            float2* __restrict__ mt)
{
    constexpr int B = 1 << LOGB;
    extern __shared__ float2 sm[];
    const int N = p.n;          // n_fw
    const int plen = padded_len(N) << LOGB;
    float2* X = sm;
    float2* Y = sm + plen;
    float2* acc = sm + 2 * plen;
    const int kt0 = blockIdx.x * B;
    for (int e = threadIdx.x; e < plen; e += blockDim.x) acc[e] = make_float2(0.f, 0.f);
    for (int j = 0; j < d.n_imp; ++j) {
        const TileLd src{shat + (int64_t)j * d.n_w * d.nh, d.nh, kt0, d.n_w};
        const float2* z = run_plan<false, LOGB>(p, src, X, Y);
        const float2* hj = H + (int64_t)j * d.n_fw * d.nh;
        for (int e = threadIdx.x; e < (N << LOGB); e += blockDim.x) {
            const int c = e & (B - 1), kw = e >> LOGB, kt = kt0 + c;
            if (kt < d.nh) {
                const int s = (pad16(kw) << LOGB) + c;
                const float2 h = __ldg(hj + (int64_t)kw * d.nh + kt);
                const float2 v = z[s];
                float2 a = acc[s];
                a.x += h.x * v.x - h.y * v.y;
                a.y += h.x * v.y + h.y * v.x;
                acc[s] = a;
            }
        }
        __syncthreads();
    }
    const float2* m = run_plan<true, LOGB>(p, SmemLd<LOGB>{acc}, X, Y);
    for (int e = threadIdx.x; e < (d.n_w << LOGB); e += blockDim.x) {
        const int c = e & (B - 1), w = e >> LOGB, kt = kt0 + c;
        if (kt < d.nh) mt[(int64_t)w * d.nh + kt] = m[(pad16(w) << LOGB) + c];
    }
}

__global__ void k_make_hermitian(ConvDims d, const float2* __restrict__ R, float2* __restrict__ H,
                                 float scale)
{
    const int64_t total = (int64_t)d.n_imp * d.n_fw * d.nh;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int kt = (int)(i % d.nh);
        const int64_t rest = i / d.nh;
        const int kw = (int)(rest % d.n_fw);
        const int j = (int)(rest / d.n_fw);
        const float2 a = R[((int64_t)j * d.n_fw + kw) * d.n_ft + kt];
        const int kwm = (d.n_fw - kw) % d.n_fw, ktm = (d.n_ft - kt) % d.n_ft;
        const float2 b = R[((int64_t)j * d.n_fw + kwm) * d.n_ft + ktm];
        const float h = 0.5f * scale;
        H[i] = make_float2(h * (a.x + b.x), h * (a.y - b.y));
    }
}

// Columns per CTA: 4 (full 32-byte sectors per wire row) when three padded 4-column
// buffers fit two CTAs per SM, else 1.
int wire_logb(int n_fw) { return (3 * (size_t)(padded_len(n_fw) << 2) * sizeof(float2) <= 110 * 1024) ? 2 : 0; }

bool g_attr = false;
cudaError_t attrs()
{
    if (g_attr) return cudaSuccess;
    const int mx = 227 * 1024;
    cudaError_t e = cudaFuncSetAttribute(k_wire_pass<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    if (!e) e = cudaFuncSetAttribute(k_wire_pass<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    if (!e) g_attr = true;
    return e;
}

}  // namespace

cudaError_t launch_make_hermitian(const ConvDims& d, const float2* resp, float2* H, float scale,
                                  cudaStream_t s)
{
    const int64_t total = (int64_t)d.n_imp * d.n_fw * d.nh;
    int64_t blocks = (total + 255) / 256;
    if (blocks > 65535 * 16) blocks = 65535 * 16;
    k_make_hermitian<<<(unsigned)blocks, 256, 0, s>>>(d, resp, H, scale);
    return cudaGetLastError();
}

cudaError_t launch_wire_pass(const ConvDims& d, const FftPlan& pw, const float2* shat,
                             const float2* H, float2* mt, cudaStream_t s)
{
    cudaError_t e = attrs();
    if (e) return e;
    const int logb = wire_logb(pw.n);
    const int B = 1 << logb;
    const unsigned blocks = (unsigned)((d.nh + B - 1) / B);
    const size_t smem = 3 * (size_t)(padded_len(pw.n) << logb) * sizeof(float2);
    if (logb == 2)
        k_wire_pass<2><<<blocks, kThreads, smem, s>>>(d, pw, shat, H, mt);
    else
        k_wire_pass<0><<<blocks, kThreads, smem, s>>>(d, pw, shat, H, mt);
    return cudaGetLastError();
}

}  // namespace wcsim
