// wcsim_convolve_noalloc: the Eq. 2 convolution of wcsim_convolve for callers that may not
// allocate device memory: code that runs under an allocator it does not own (a framework's
// caching allocator or a memory pool with a fixed budget), or a host process that forbids
// allocation once it has started.  Every intermediate array lives in one file-scope static
// device array of fixed size (WCSIM_NOALLOC_SCRATCH_BYTES); the caller passes only the
// response spectrum, the grid and the output.
//
// The array exists once per device that loads this library and stays until the process
// exits.  In host code its name is only a host-side stand-in, not a device address, so the
// first call on each device looks the address up with cudaGetSymbolAddress (with that
// device current) and caches it; that first call should therefore come before any stream
// capture.  All calls share the array and it keeps the last call's contents: calls whose GPU
// work overlaps (on different streams, or from different threads) race on it and must be
// serialised by the caller.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>

#include "async_copy.cuh"
#include "wcsim_internal.cuh"

// The scratch of every wcsim_convolve_noalloc call on this device.
static __device__ __align__(256) unsigned char g_scratch[WCSIM_NOALLOC_SCRATCH_BYTES];

namespace wcsim {
namespace {

constexpr size_t kScratchBytes = WCSIM_NOALLOC_SCRATCH_BYTES;
constexpr int kMaxDevices = 64;

void* g_scratch_addr[kMaxDevices];   // device address of g_scratch per device ordinal

size_t up256(size_t b) { return (b + 255) & ~(size_t)255; }

// The flag word sits at the start of the scratch (offset 0 in every call's carving).
constexpr size_t kFlagsOffset = 0;

// The device address of g_scratch on the current device, looked up once per device (with
// that device current).  Returns a CUDA error code or cudaSuccess.
cudaError_t scratch_base(unsigned char** out, char* msg, size_t msg_len)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        snprintf(msg, msg_len, "cudaGetDevice: %s", cudaGetErrorString(e));
        return e;
    }
    if (dev < 0 || dev >= kMaxDevices) {
        snprintf(msg, msg_len, "device ordinal %d out of range", dev);
        return cudaErrorInvalidDevice;
    }
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p) {
            snprintf(msg, msg_len, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
            return e != cudaSuccess ? e : cudaErrorInvalidSymbol;
        }
        g_scratch_addr[dev] = p;
    }
    *out = static_cast<unsigned char*>(g_scratch_addr[dev]);
    return cudaSuccess;
}

// Twiddle table of a plan: entry (r - 1) ns + k of pass p = exp(-2 pi i r k / (ns R)),
// FP64 sincospi rounded to FP32.
__global__ void k_fill_plan_twiddles(FftPlan p, float2* tw)
{
    const int stride = gridDim.x * blockDim.x;
    for (int i = 0; i < p.npass; ++i) {
        const int R = p.radix[i], ns = p.ns[i], cnt = (R - 1) * ns;
        for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < cnt; e += stride) {
            const int r = e / ns + 1, k = e % ns;
            double s, c;
            sincospi(-2.0 * (double)(r * k) / ((double)ns * R), &s, &c);
            tw[p.tw_off[i] + e] = make_float2((float)c, (float)s);
        }
    }
}

// Twiddles of the one-warp-per-column wire pass: [2][n], exp(-2 pi i a b / n) at a * 32 + b
// and at b * M + a (a < M = n / 32, b < 32).
__global__ void k_fill_warp_twiddles(int n, float2* tw)
{
    const int M = n / 32;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
        const int a = e / 32, b = e % 32;
        double s, c;
        sincospi(-2.0 * (double)((a * b) % n) / (double)n, &s, &c);
        const float2 w = make_float2((float)c, (float)s);
        tw[e] = w;
        tw[n + b * M + a] = w;
    }
}

}  // namespace
}  // namespace wcsim

using namespace wcsim;

extern "C" wcsim_status wcsim_convolve_noalloc(const wcsim_geometry* geom, const void* resp_c64,
                                               int32_t n_fw, int32_t n_ft, const float* grid,
                                               float* wave, void* stream)
{
    char msg[256];
    if (!geom || !resp_c64 || !grid || !wave)
        return report_error(WCSIM_EINVAL, "geometry, response, grid or wave is NULL");
    if (geom->n_wires < 1 || geom->n_imp < 1 || geom->n_ticks < 1 || geom->reserved != 0)
        return report_error(WCSIM_ESHAPE, "n_wires, n_imp, n_ticks must be >= 1 and reserved 0");
    if (n_fw == 0) n_fw = geom->n_wires;
    if (n_ft == 0) n_ft = geom->n_ticks;
    if (n_fw < geom->n_wires || n_ft < geom->n_ticks || n_ft > kMaxFftN || n_fw > kMaxWireN)
        return report_error(WCSIM_ESHAPE, "spectrum size smaller than the frame or too large");

    ConvDims d{};
    d.n_w = geom->n_wires;
    d.n_imp = geom->n_imp;
    d.n_t = geom->n_ticks;
    d.n_fw = n_fw;
    d.n_ft = n_ft;
    d.nh = n_ft / 2 + 1;
    d.nkb = (d.nh + kBlockCols - 1) / kBlockCols;
    d.rows_variant = 0;
    FftPlan pt, pw;
    const int len_t = fft_plan_describe(n_ft, &pt);
    const int len_w = fft_plan_describe(n_fw, &pw);
    if (len_t < 0 || len_w < 0)
        return report_error(WCSIM_ESHAPE, "FFT sizes must factor into 2, 3, 5 and 7");
    const bool warp = wire_warp_supported(n_fw);

    // carve the static scratch: flag word, twiddles, H, Shat, Mt
    const size_t cols = (size_t)d.nkb * kBlockCols;
    size_t off = 0;
    const size_t o_flags = kFlagsOffset;  off += 256;
    const size_t o_twt = off;    off += up256((size_t)len_t * sizeof(float2));
    const size_t o_tww = off;    off += up256((size_t)len_w * sizeof(float2));
    const size_t o_twarp = off;  off += warp ? up256(2 * (size_t)n_fw * sizeof(float2)) : 0;
    const size_t o_h = off;      off += up256((size_t)d.n_imp * n_fw * cols * sizeof(float2));
    const size_t o_shat = off;   off += up256((size_t)d.n_imp * d.n_w * cols * sizeof(float2));
    const size_t o_mt = off;     off += up256((size_t)d.n_w * cols * sizeof(float2));
    if (off > kScratchBytes) {
        snprintf(msg, sizeof(msg),
                 "frame needs %zu bytes of scratch; the static scratch holds %zu bytes "
                 "(use wcsim_plane_create / wcsim_convolve for larger planes)",
                 off, kScratchBytes);
        return report_error(WCSIM_ESHAPE, msg);
    }

    // set-up, once per device: the device address of the static array
    unsigned char* base = nullptr;
    cudaError_t e = scratch_base(&base, msg, sizeof(msg));
    if (e != cudaSuccess) return report_error(WCSIM_ECUDA, msg);
    int* flags = reinterpret_cast<int*>(base + o_flags);
    float2* tw_t = reinterpret_cast<float2*>(base + o_twt);
    float2* tw_w = reinterpret_cast<float2*>(base + o_tww);
    float2* tw_warp = reinterpret_cast<float2*>(base + o_twarp);
    float2* H = reinterpret_cast<float2*>(base + o_h);
    float2* shat = reinterpret_cast<float2*>(base + o_shat);
    float2* mt = reinterpret_cast<float2*>(base + o_mt);
    pt.tw = tw_t;
    pw.tw = tw_w;

    cudaStream_t s = (cudaStream_t)stream;
    // the flag word is the only scratch read before it is written
    if ((e = cudaMemsetAsync(flags, 0, sizeof(int), s))) return report_error(WCSIM_ECUDA, cudaGetErrorString(e));
    k_fill_plan_twiddles<<<8, 256, 0, s>>>(pt, tw_t);
    k_fill_plan_twiddles<<<4, 256, 0, s>>>(pw, tw_w);
    if (warp) k_fill_warp_twiddles<<<4, 256, 0, s>>>(n_fw, tw_warp);
    if ((e = cudaGetLastError())) return report_error(WCSIM_ECUDA, cudaGetErrorString(e));
    if ((e = launch_make_hermitian(d, (const float2*)resp_c64, H,
                                   (float)(1.0 / ((double)n_fw * (double)n_ft)), s)) ||
        (e = launch_rows_r2c(d, pt, grid, shat, flags, s)) ||
        (e = warp ? launch_wire_warp(d, tw_warp, shat, H, mt, flags, s)
                  : launch_wire_pass(d, pw, shat, H, mt, flags, s)) ||
        (e = launch_rows_c2r(d, pt, mt, wave, s)))
        return report_error(WCSIM_ECUDA, cudaGetErrorString(e));
    return WCSIM_OK;
}

extern "C" wcsim_status wcsim_convolve_noalloc_check(void* stream, int32_t* flags)
{
    char msg[256];
    unsigned char* base = nullptr;
    cudaError_t e = scratch_base(&base, msg, sizeof(msg));
    if (e != cudaSuccess) return report_error(WCSIM_ECUDA, msg);
    cudaStream_t s = (cudaStream_t)stream;
    int32_t h = 0;
    // a copy into pageable host memory: the runtime stages it itself, nothing is allocated here
    e = cudaMemcpyAsync(&h, base + kFlagsOffset, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        snprintf(msg, sizeof(msg), "flag read: %s", cudaGetErrorString(e));
        return report_error(WCSIM_ECUDA, msg);
    }
    if (flags) *flags = h;
    if (h & kErrTimeout) {
        snprintf(msg, sizeof(msg),
                 "a device-side wait for an asynchronous copy gave up in the last "
                 "wcsim_convolve_noalloc call (flags 0x%x); its output is incomplete", h);
        return report_error(WCSIM_ETIMEOUT, msg);
    }
    return WCSIM_OK;
}
