// Frequency-domain convolution of Eq. 2 with hand-written mixed-radix Stockham FFTs.
//
//   1. rows_r2c:  every grid row (one impact position j of one wire w) is transformed along
//                 the time axis.  Two real rows ride in one complex FFT (z = x0 + i x1) and
//                 are separated afterwards; the Hermitian half (n_ft/2 + 1 bins) is stored
//                 as Shat[j][w][kt].
//   2. wire_pass: for a block of F time frequencies, each S_j is transformed along the wire
//                 axis, multiplied by its response H_j and accumulated over j in shared
//                 memory; the sum is transformed back along the wire axis.  Mt[w][kt].
//   3. rows_c2r:  the Hermitian half rows of Mt are transformed back along the time axis
//                 (two real outputs per complex FFT) and cropped to the frame.
// H_j is the Hermitian part of the supplied R_j with 1/(n_fw n_ft) folded in, so that the
// real part of Re IFFT2(sum_j R_j FFT2(S_j)) comes out directly.
//
// A Stockham pass of radix R over length N (Ns = product of the radices already applied)
// reads x[j + r N/R], multiplies by exp(-+2 pi i r (j mod Ns) / (Ns R)), applies an R-point
// DFT and writes y[(j / Ns) Ns R + (j mod Ns) + r Ns]; the output is in natural order.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

#include <vector>

#include "wcsim_internal.cuh"

namespace wcsim {

// ------------------------------------------------------------------ host: plans
bool fft_factor(int n, int32_t* radix, int32_t* npass)
{
    int m = n, np = 0;
    int twos = 0;
    while (m % 2 == 0) { m /= 2; ++twos; }
    while (twos >= 4) { radix[np++] = 16; twos -= 4; if (np >= kMaxPasses) return false; }
    if (twos == 3) radix[np++] = 8;
    if (twos == 2) radix[np++] = 4;
    if (twos == 1) radix[np++] = 2;
    const int odd[3] = {5, 3, 7};
    for (int f : odd) {
        while (m % f == 0) {
            if (np >= kMaxPasses) return false;
            radix[np++] = f;
            m /= f;
        }
    }
    if (m != 1) return false;
    if (np == 0) radix[np++] = 1;   // n == 1: a single identity pass
    *npass = np;
    return true;
}

static uint32_t magic_for(int d) { return d <= 1 ? 0u : (uint32_t)((0x100000000ull + d - 1) / (uint64_t)d); }

cudaError_t fft_plan_create(int n, FftPlan* plan, float2** dev_tw)
{
    FftPlan p{};
    p.n = n;
    if (!fft_factor(n, p.radix, &p.npass)) return cudaErrorInvalidValue;
    std::vector<float2> tw;
    int ns = 1;
    for (int i = 0; i < p.npass; ++i) {
        const int R = p.radix[i];
        p.ns[i] = ns;
        p.tw_off[i] = (int32_t)tw.size();
        p.ns_magic[i] = magic_for(ns);
        p.nb_magic[i] = magic_for(n / (R > 0 ? R : 1));
        for (int k = 0; k < ns; ++k)
            for (int r = 1; r < R; ++r) {
                const double a = -2.0 * M_PI * (double)r * (double)k / ((double)ns * R);
                tw.push_back(make_float2((float)cos(a), (float)sin(a)));
            }
        ns *= R;
    }
    if (tw.empty()) tw.push_back(make_float2(1.f, 0.f));
    float2* d = nullptr;
    cudaError_t e = cudaMalloc(&d, tw.size() * sizeof(float2));
    if (e != cudaSuccess) return e;
    e = cudaMemcpy(d, tw.data(), tw.size() * sizeof(float2), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) { cudaFree(d); return e; }
    p.tw = d;
    *plan = p;
    *dev_tw = d;
    return cudaSuccess;
}

namespace {

// ------------------------------------------------------------------ device: butterflies
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b)
{
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a * w (forward) or a * conj(w) (inverse)
template <bool INV>
__device__ __forceinline__ float2 twiddle(float2 a, float2 w)
{
    return INV ? make_float2(a.x * w.x + a.y * w.y, a.y * w.x - a.x * w.y) : cmul(a, w);
}
// -i a (forward) or +i a (inverse)
template <bool INV>
__device__ __forceinline__ float2 rot(float2 a)
{
    return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

template <bool INV>
__device__ __forceinline__ void dft2(float2* v)
{
    const float2 a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
}

template <bool INV>
__device__ __forceinline__ void dft4(float2& v0, float2& v1, float2& v2, float2& v3)
{
    const float2 s02 = cadd(v0, v2), d02 = csub(v0, v2);
    const float2 s13 = cadd(v1, v3), d13 = rot<INV>(csub(v1, v3));
    v0 = cadd(s02, s13);
    v2 = csub(s02, s13);
    v1 = cadd(d02, d13);
    v3 = csub(d02, d13);
}

template <bool INV>
__device__ __forceinline__ void dft3(float2* v)
{
    const float s3 = 0.866025403784438647f;
    const float2 t = cadd(v[1], v[2]);
    const float2 d = rot<INV>(cscale(csub(v[1], v[2]), s3));
    const float2 m = make_float2(v[0].x - 0.5f * t.x, v[0].y - 0.5f * t.y);
    v[0] = cadd(v[0], t);
    v[1] = cadd(m, d);
    v[2] = csub(m, d);
}

template <bool INV>
__device__ __forceinline__ void dft5(float2* v)
{
    const float c1 = 0.309016994374947424f, c2 = -0.809016994374947424f;
    const float s1 = 0.951056516295153572f, s2 = 0.587785252292473129f;
    const float2 t1 = cadd(v[1], v[4]), t2 = cadd(v[2], v[3]);
    const float2 d1 = csub(v[1], v[4]), d2 = csub(v[2], v[3]);
    const float2 v0 = v[0];
    const float2 a1 = make_float2(v0.x + c1 * t1.x + c2 * t2.x, v0.y + c1 * t1.y + c2 * t2.y);
    const float2 a2 = make_float2(v0.x + c2 * t1.x + c1 * t2.x, v0.y + c2 * t1.y + c1 * t2.y);
    const float2 b1 = rot<INV>(make_float2(s1 * d1.x + s2 * d2.x, s1 * d1.y + s2 * d2.y));
    const float2 b2 = rot<INV>(make_float2(s2 * d1.x - s1 * d2.x, s2 * d1.y - s1 * d2.y));
    v[0] = cadd(v0, cadd(t1, t2));
    v[1] = cadd(a1, b1);
    v[4] = csub(a1, b1);
    v[2] = cadd(a2, b2);
    v[3] = csub(a2, b2);
}

template <bool INV>
__device__ __forceinline__ void dft7(float2* v)
{
    // cos / sin (2 pi m / 7), m = 1, 2, 3
    const float c[3] = {0.623489801858733530f, -0.222520933956314404f, -0.900968867902419126f};
    const float s[3] = {0.781831482468029809f, 0.974927912181823607f, 0.433883739117558120f};
    float2 t[3], d[3];
#pragma unroll
    for (int p = 0; p < 3; ++p) {
        t[p] = cadd(v[p + 1], v[6 - p]);
        d[p] = csub(v[p + 1], v[6 - p]);
    }
    const float2 v0 = v[0];
    v[0] = cadd(v0, cadd(t[0], cadd(t[1], t[2])));
#pragma unroll
    for (int k = 1; k <= 3; ++k) {
        float2 a = v0, b = make_float2(0.f, 0.f);
#pragma unroll
        for (int p = 1; p <= 3; ++p) {
            const int m = (p * k) % 7;                 // angle index 2 pi m / 7
            const float cm = (m <= 3) ? c[m - 1] : c[7 - m - 1];
            const float sm = (m <= 3) ? s[m - 1] : -s[7 - m - 1];
            a.x += cm * t[p - 1].x; a.y += cm * t[p - 1].y;
            b.x += sm * d[p - 1].x; b.y += sm * d[p - 1].y;
        }
        const float2 rb = rot<INV>(b);
        v[k] = cadd(a, rb);
        v[7 - k] = csub(a, rb);
    }
}

template <bool INV>
__device__ __forceinline__ void dft8(float2* v)
{
    const float h = 0.707106781186547524f;
    dft4<INV>(v[0], v[2], v[4], v[6]);
    dft4<INV>(v[1], v[3], v[5], v[7]);
    // odd part times w8^k, k = 0..3
    float2 o1 = v[3], o2 = v[5], o3 = v[7];
    // w8 = (h, -h) forward; conj for inverse
    o1 = INV ? make_float2(h * (o1.x - o1.y), h * (o1.x + o1.y))
             : make_float2(h * (o1.x + o1.y), h * (o1.y - o1.x));
    o2 = rot<INV>(o2);
    o3 = INV ? make_float2(-h * (o3.x + o3.y), h * (o3.x - o3.y))
             : make_float2(h * (o3.y - o3.x), -h * (o3.x + o3.y));
    const float2 e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6], o0 = v[1];
    v[0] = cadd(e0, o0); v[4] = csub(e0, o0);
    v[1] = cadd(e1, o1); v[5] = csub(e1, o1);
    v[2] = cadd(e2, o2); v[6] = csub(e2, o2);
    v[3] = cadd(e3, o3); v[7] = csub(e3, o3);
}

template <bool INV>
__device__ __forceinline__ void dft16(float2* v)
{
    // X[k1 + 4 k2] = sum_b w16^(b k1) w4^(b k2) Y_b[k1],  Y_b = DFT4 of v[b + 4 a] over a
#pragma unroll
    for (int b = 0; b < 4; ++b) dft4<INV>(v[b], v[b + 4], v[b + 8], v[b + 12]);
    // after this, v[b + 4 k1] holds Y_b[k1]
    const float cs[4] = {1.0f, 0.923879532511286756f, 0.707106781186547524f, 0.382683432365089772f};
#pragma unroll
    for (int b = 1; b < 4; ++b)
#pragma unroll
        for (int k1 = 1; k1 < 4; ++k1) {
            const int m = b * k1;                      // angle 2 pi m / 16, m in 1..9
            // cos(2 pi m/16) and sin(2 pi m/16) from the first quadrant table
            float cm, sm;
            const int q = m / 4, rr = m % 4;
            const float cr = cs[rr], sr = cs[(4 - rr) & 3] * (rr == 0 ? 0.0f : 1.0f);
            if (q == 0) { cm = cr; sm = sr; }
            else if (q == 1) { cm = -sr; sm = cr; }
            else { cm = -cr; sm = -sr; }
            // forward multiplies by exp(-i a) = (cm, -sm); inverse by (cm, sm)
            const float2 w = make_float2(cm, INV ? sm : -sm);
            v[b + 4 * k1] = cmul(v[b + 4 * k1], w);
        }
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) dft4<INV>(v[4 * k1], v[4 * k1 + 1], v[4 * k1 + 2], v[4 * k1 + 3]);
    // v[4 k1 + k2] now holds X[k1 + 4 k2]: transpose the 4x4 index in registers
    float2 o[16];
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1)
#pragma unroll
        for (int k2 = 0; k2 < 4; ++k2) o[k1 + 4 * k2] = v[4 * k1 + k2];
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = o[i];
}

template <int R, bool INV>
__device__ __forceinline__ void dft(float2* v)
{
    if constexpr (R == 2) dft2<INV>(v);
    else if constexpr (R == 3) dft3<INV>(v);
    else if constexpr (R == 4) dft4<INV>(v[0], v[1], v[2], v[3]);
    else if constexpr (R == 5) dft5<INV>(v);
    else if constexpr (R == 7) dft7<INV>(v);
    else if constexpr (R == 8) dft8<INV>(v);
    else if constexpr (R == 16) dft16<INV>(v);
}

// One Stockham pass over `batch` sequences of length n stored back to back (stride n).
template <int R, bool INV>
__device__ __forceinline__ void pass_body(const float2* __restrict__ x, float2* __restrict__ y,
                                          int n, int batch, int ns, uint32_t ns_magic,
                                          uint32_t nb_magic, const float2* __restrict__ tw)
{
    const int nb = n / R;
    const int total = nb * batch;
    for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
        const int b = (nb == 1) ? idx : (int)__umulhi((uint32_t)idx, nb_magic);
        const int j = idx - b * nb;
        const int q = (ns == 1) ? j : (int)__umulhi((uint32_t)j, ns_magic);
        const int k = j - q * ns;
        const float2* xb = x + b * n;
        float2* yb = y + b * n;
        float2 v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = xb[j + r * nb];
        if (k > 0) {
            const float2* t = tw + k * (R - 1);
#pragma unroll
            for (int r = 1; r < R; ++r) v[r] = twiddle<INV>(v[r], __ldg(t + r - 1));
        }
        dft<R, INV>(v);
        const int o = q * ns * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) yb[o + r * ns] = v[r];
    }
}

// All passes of a plan; returns the buffer holding the result (x or y).
template <bool INV>
__device__ float2* run_fft(float2* x, float2* y, int batch, const FftPlan& p)
{
    for (int i = 0; i < p.npass; ++i) {
        const float2* tw = p.tw + p.tw_off[i];
        switch (p.radix[i]) {
            case 16: pass_body<16, INV>(x, y, p.n, batch, p.ns[i], p.ns_magic[i], p.nb_magic[i], tw); break;
            case 8: pass_body<8, INV>(x, y, p.n, batch, p.ns[i], p.ns_magic[i], p.nb_magic[i], tw); break;
            case 4: pass_body<4, INV>(x, y, p.n, batch, p.ns[i], p.ns_magic[i], p.nb_magic[i], tw); break;
            case 2: pass_body<2, INV>(x, y, p.n, batch, p.ns[i], p.ns_magic[i], p.nb_magic[i], tw); break;
            case 5: pass_body<5, INV>(x, y, p.n, batch, p.ns[i], p.ns_magic[i], p.nb_magic[i], tw); break;
            case 3: pass_body<3, INV>(x, y, p.n, batch, p.ns[i], p.ns_magic[i], p.nb_magic[i], tw); break;
            case 7: pass_body<7, INV>(x, y, p.n, batch, p.ns[i], p.ns_magic[i], p.nb_magic[i], tw); break;
            default: {   // radix 1 (n == 1): copy
                for (int e = threadIdx.x; e < p.n * batch; e += blockDim.x) y[e] = x[e];
            }
        }
        __syncthreads();
        float2* t = x; x = y; y = t;
    }
    return x;
}

// ------------------------------------------------------------------ kernels
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

__global__ void __launch_bounds__(512)
k_rows_r2c(ConvDims d, FftPlan p, const float* __restrict__ grid, float2* __restrict__ shat)
{
    extern __shared__ float2 sm[];
    const int N = p.n;
    float2* x = sm;
    float2* y = sm + N;
    const int64_t n_rows = (int64_t)d.n_w * d.n_imp;
    const int64_t r0 = 2 * (int64_t)blockIdx.x, r1 = r0 + 1;
    const bool has1 = r1 < n_rows;
    const float* g0 = grid + r0 * d.n_t;
    const float* g1 = grid + (has1 ? r1 : r0) * d.n_t;
    for (int n = threadIdx.x; n < N; n += blockDim.x) {
        float a = 0.f, b = 0.f;
        if (n < d.n_t) {
            a = g0[n];
            b = has1 ? g1[n] : 0.f;
        }
        x[n] = make_float2(a, b);
    }
    __syncthreads();
    const float2* z = run_fft<false>(x, y, 1, p);
    const int w0 = (int)(r0 / d.n_imp), j0 = (int)(r0 % d.n_imp);
    const int w1 = (int)(r1 / d.n_imp), j1 = (int)(r1 % d.n_imp);
    float2* o0 = shat + ((int64_t)j0 * d.n_w + w0) * d.nh;
    float2* o1 = shat + ((int64_t)j1 * d.n_w + w1) * d.nh;
    for (int k = threadIdx.x; k < d.nh; k += blockDim.x) {
        const float2 a = z[k];
        const float2 b = z[k == 0 ? 0 : N - k];
        // x0 -> (Z[k] + conj Z[-k]) / 2,  x1 -> (Z[k] - conj Z[-k]) / (2 i)
        o0[k] = make_float2(0.5f * (a.x + b.x), 0.5f * (a.y - b.y));
        if (has1) o1[k] = make_float2(0.5f * (a.y + b.y), 0.5f * (b.x - a.x));
    }
}

template <int LOGF>
__global__ void __launch_bounds__(256)
k_wire_pass(ConvDims d, FftPlan p, const float2* __restrict__ shat, const float2* __restrict__ H,
            float2* __restrict__ mt)
{
    constexpr int F = 1 << LOGF;
    extern __shared__ float2 sm[];
    const int N = p.n;                 // n_fw
    float2* xa = sm;
    float2* xb = sm + F * N;
    float2* acc = sm + 2 * F * N;
    const int kt0 = blockIdx.x * F;
    for (int e = threadIdx.x; e < F * N; e += blockDim.x) acc[e] = make_float2(0.f, 0.f);
    for (int j = 0; j < d.n_imp; ++j) {
        const float2* src = shat + (int64_t)j * d.n_w * d.nh;
        for (int e = threadIdx.x; e < F * N; e += blockDim.x) {
            const int w = e >> LOGF, c = e & (F - 1), kt = kt0 + c;
            xa[c * N + w] = (w < d.n_w && kt < d.nh) ? src[(int64_t)w * d.nh + kt]
                                                      : make_float2(0.f, 0.f);
        }
        __syncthreads();
        const float2* z = run_fft<false>(xa, xb, F, p);
        const float2* hj = H + (int64_t)j * d.n_fw * d.nh;
        for (int e = threadIdx.x; e < F * N; e += blockDim.x) {
            const int kw = e >> LOGF, c = e & (F - 1), kt = kt0 + c;
            if (kt < d.nh) {
                const float2 h = hj[(int64_t)kw * d.nh + kt];
                const float2 s = z[c * N + kw];
                float2 a = acc[c * N + kw];
                a.x += h.x * s.x - h.y * s.y;
                a.y += h.x * s.y + h.y * s.x;
                acc[c * N + kw] = a;
            }
        }
        __syncthreads();
    }
    const float2* m = run_fft<true>(acc, xa, F, p);
    for (int e = threadIdx.x; e < F * N; e += blockDim.x) {
        const int w = e >> LOGF, c = e & (F - 1), kt = kt0 + c;
        if (w < d.n_w && kt < d.nh) mt[(int64_t)w * d.nh + kt] = m[c * N + w];
    }
}

__global__ void __launch_bounds__(512)
k_rows_c2r(ConvDims d, FftPlan p, const float2* __restrict__ mt, float* __restrict__ wave)
{
    extern __shared__ float2 sm[];
    const int N = p.n;
    float2* x = sm;
    float2* y = sm + N;
    const int w0 = 2 * blockIdx.x, w1 = w0 + 1;
    const bool has1 = w1 < d.n_w;
    const float2* m0 = mt + (int64_t)w0 * d.nh;
    const float2* m1 = mt + (int64_t)(has1 ? w1 : w0) * d.nh;
    for (int k = threadIdx.x; k < N; k += blockDim.x) {
        float2 a, b;
        if (k < d.nh) {
            a = m0[k];
            b = has1 ? m1[k] : make_float2(0.f, 0.f);
        } else {
            const float2 ac = m0[N - k];
            const float2 bc = has1 ? m1[N - k] : make_float2(0.f, 0.f);
            a = make_float2(ac.x, -ac.y);
            b = make_float2(bc.x, -bc.y);
        }
        // z = X0 + i X1
        x[k] = make_float2(a.x - b.y, a.y + b.x);
    }
    __syncthreads();
    const float2* z = run_fft<true>(x, y, 1, p);
    float* o0 = wave + (int64_t)w0 * d.n_t;
    float* o1 = wave + (int64_t)w1 * d.n_t;
    for (int t = threadIdx.x; t < d.n_t; t += blockDim.x) {
        const float2 v = z[t];
        o0[t] = v.x;
        if (has1) o1[t] = v.y;
    }
}

int rows_threads(int n) { return n >= 4096 ? 512 : 256; }

bool g_attr_done = false;

cudaError_t set_smem_attrs()
{
    if (g_attr_done) return cudaSuccess;
    const int max_smem = 227 * 1024;
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_rows_r2c, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem))) return e;
    if ((e = cudaFuncSetAttribute(k_rows_c2r, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem))) return e;
    if ((e = cudaFuncSetAttribute(k_wire_pass<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem))) return e;
    if ((e = cudaFuncSetAttribute(k_wire_pass<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem))) return e;
    if ((e = cudaFuncSetAttribute(k_wire_pass<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem))) return e;
    if ((e = cudaFuncSetAttribute(k_wire_pass<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem))) return e;
    g_attr_done = true;
    return cudaSuccess;
}

}  // namespace

cudaError_t launch_make_hermitian(const ConvDims& d, const float2* resp, float2* H, float scale,
                                  cudaStream_t s)
{
    const int64_t total = (int64_t)d.n_imp * d.n_fw * d.nh;
    const int64_t blocks = (total + 255) / 256;
    k_make_hermitian<<<(unsigned)(blocks < 65535 * 16 ? blocks : 65535 * 16), 256, 0, s>>>(
        d, resp, H, scale);
    return cudaGetLastError();
}

cudaError_t launch_rows_r2c(const ConvDims& d, const FftPlan& pt, const float* grid,
                            float2* shat, cudaStream_t s)
{
    cudaError_t e = set_smem_attrs();
    if (e) return e;
    const int64_t n_rows = (int64_t)d.n_w * d.n_imp;
    const unsigned blocks = (unsigned)((n_rows + 1) / 2);
    const size_t smem = 2 * (size_t)pt.n * sizeof(float2);
    k_rows_r2c<<<blocks, rows_threads(pt.n), smem, s>>>(d, pt, grid, shat);
    return cudaGetLastError();
}

// Columns per wire-pass block: as many as fit three F x n_fw buffers in ~110 KB (two
// blocks per SM), at most 8.
static int wire_logf(int n_fw)
{
    int logf = 3;
    while (logf > 0 && (size_t)3 * (1 << logf) * n_fw * sizeof(float2) > 110 * 1024) --logf;
    return logf;
}

cudaError_t launch_wire_pass(const ConvDims& d, const FftPlan& pw, const float2* shat,
                             const float2* H, float2* mt, cudaStream_t s)
{
    cudaError_t e = set_smem_attrs();
    if (e) return e;
    const int logf = wire_logf(pw.n);
    const int F = 1 << logf;
    const unsigned blocks = (unsigned)((d.nh + F - 1) / F);
    const size_t smem = 3 * (size_t)F * pw.n * sizeof(float2);
    switch (logf) {
        case 3: k_wire_pass<3><<<blocks, 256, smem, s>>>(d, pw, shat, H, mt); break;
        case 2: k_wire_pass<2><<<blocks, 256, smem, s>>>(d, pw, shat, H, mt); break;
        case 1: k_wire_pass<1><<<blocks, 256, smem, s>>>(d, pw, shat, H, mt); break;
        default: k_wire_pass<0><<<blocks, 256, smem, s>>>(d, pw, shat, H, mt); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_rows_c2r(const ConvDims& d, const FftPlan& pt, const float2* mt,
                            float* wave, cudaStream_t s)
{
    cudaError_t e = set_smem_attrs();
    if (e) return e;
    const unsigned blocks = (unsigned)((d.n_w + 1) / 2);
    const size_t smem = 2 * (size_t)pt.n * sizeof(float2);
    k_rows_c2r<<<blocks, rows_threads(pt.n), smem, s>>>(d, pt, mt, wave);
    return cudaGetLastError();
}

}  // namespace wcsim
