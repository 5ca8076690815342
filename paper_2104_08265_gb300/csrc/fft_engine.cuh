// Device FFT engine: register DFTs and mixed-radix Stockham passes over shared memory.
//
// A plan factors N into a few radices R <= 25 (composite radices such as 20 or 24 are
// transformed entirely in registers), so that a 6000-point transform takes three
// shared-memory passes.  Pass p (Ns = product of the earlier radices) reads
// x[j + r N/R], r < R, multiplies by exp(-+2 pi i r (j mod Ns) / (Ns R)), applies the
// R-point DFT and writes y[(j / Ns) Ns R + (j mod Ns) + r Ns]; the result is in natural
// order.  B = 2^LOGB independent sequences are transformed together; element (c, i) of the
// batch lives at buf[pad(i) * B + c], where pad() inserts one slot every 16 elements so
// that the stride-R writes of early passes do not pile onto one shared-memory bank.
//
// Plans come in two forms: a runtime plan (FftPlan: any length that factors into radices
// <= 25, passes ping-ponging between two buffers) and compile-time plans (pass_fixed /
// pass_fixed_inplace, all strides and divisors constants; the in-place form holds each
// thread's butterfly inputs in registers across a barrier and needs one buffer).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "dft_roots.cuh"
#include "rng.cuh"
#include "wcsim_internal.cuh"

namespace wcsim {

__host__ __device__ __forceinline__ int pad16(int i) { return i + (i >> 4); }
__host__ __device__ __forceinline__ int padded_len(int n) { return n + (n >> 4) + 1; }

// ------------------------------------------------------------------ complex helpers
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

// ------------------------------------------------------------------ small DFTs
template <bool INV>
__device__ __forceinline__ void dft4v(float2& v0, float2& v1, float2& v2, float2& v3)
{
    const float2 s02 = cadd(v0, v2), d02 = csub(v0, v2);
    const float2 s13 = cadd(v1, v3), d13 = rot<INV>(csub(v1, v3));
    v0 = cadd(s02, s13);
    v2 = csub(s02, s13);
    v1 = cadd(d02, d13);
    v3 = csub(d02, d13);
}

template <bool INV>
__device__ __forceinline__ void dft3v(float2* v)
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
__device__ __forceinline__ void dft5v(float2* v)
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
__device__ __forceinline__ void dft7v(float2* v)
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
            const int m = (p * k) % 7;
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
__device__ __forceinline__ void dft8v(float2* v)
{
    const float h = 0.707106781186547524f;
    dft4v<INV>(v[0], v[2], v[4], v[6]);
    dft4v<INV>(v[1], v[3], v[5], v[7]);
    float2 o1 = v[3], o2 = v[5], o3 = v[7];
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
__device__ __forceinline__ void dft16v(float2* v)
{
    // X[k1 + 4 k2] = sum_b w16^(b k1) w4^(b k2) Y_b[k1],  Y_b = DFT4 of v[b + 4 a] over a
#pragma unroll
    for (int b = 0; b < 4; ++b) dft4v<INV>(v[b], v[b + 4], v[b + 8], v[b + 12]);
    const float cs[4] = {1.0f, 0.923879532511286756f, 0.707106781186547524f, 0.382683432365089772f};
#pragma unroll
    for (int b = 1; b < 4; ++b)
#pragma unroll
        for (int k1 = 1; k1 < 4; ++k1) {
            const int m = b * k1;
            const int q = m / 4, rr = m % 4;
            const float cr = cs[rr], sr = (rr == 0) ? 0.0f : cs[4 - rr];
            float cm, sm;
            if (q == 0) { cm = cr; sm = sr; }
            else if (q == 1) { cm = -sr; sm = cr; }
            else { cm = -cr; sm = -sr; }
            v[b + 4 * k1] = cmul(v[b + 4 * k1], make_float2(cm, INV ? sm : -sm));
        }
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) dft4v<INV>(v[4 * k1], v[4 * k1 + 1], v[4 * k1 + 2], v[4 * k1 + 3]);
    float2 o[16];
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1)
#pragma unroll
        for (int k2 = 0; k2 < 4; ++k2) o[k1 + 4 * k2] = v[4 * k1 + k2];
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = o[i];
}

// First factor of a composite radix for the Cooley-Tukey split R = A * B.
template <int R>
struct Split {
    static constexpr int A = (R % 16 == 0 && R != 16) ? 16
                           : (R % 8 == 0 && R != 8) ? 8
                           : (R % 4 == 0 && R != 4) ? 4
                           : (R % 2 == 0) ? 2
                           : (R % 3 == 0) ? 3
                           : (R % 5 == 0) ? 5 : 7;
    static constexpr int B = R / A;
};

// In-register R-point DFT, natural order in and out.  Composite R: n = B n1 + n2,
// k = k1 + A k2;  A-point DFTs over n1, twiddle exp(-+2 pi i n2 k1 / R), B-point DFTs over n2.
template <int R, bool INV>
__device__ __forceinline__ void dft(float2* v)
{
    if constexpr (R == 1) {
    } else if constexpr (R == 2) {
        const float2 a = v[0], b = v[1];
        v[0] = cadd(a, b);
        v[1] = csub(a, b);
    } else if constexpr (R == 3) {
        dft3v<INV>(v);
    } else if constexpr (R == 4) {
        dft4v<INV>(v[0], v[1], v[2], v[3]);
    } else if constexpr (R == 5) {
        dft5v<INV>(v);
    } else if constexpr (R == 7) {
        dft7v<INV>(v);
    } else if constexpr (R == 8) {
        dft8v<INV>(v);
    } else if constexpr (R == 16) {
        dft16v<INV>(v);
    } else {
        constexpr int A = Split<R>::A, B = Split<R>::B;
        float2 y[R];
#pragma unroll
        for (int n2 = 0; n2 < B; ++n2) {
            float2 t[A];
#pragma unroll
            for (int n1 = 0; n1 < A; ++n1) t[n1] = v[B * n1 + n2];
            dft<A, INV>(t);
#pragma unroll
            for (int k1 = 0; k1 < A; ++k1) {
                float2 x = t[k1];
                if (n2 * k1 != 0) {
                    const float c = Roots<R>::c((n2 * k1) % R), s = Roots<R>::s((n2 * k1) % R);
                    x = INV ? make_float2(x.x * c - x.y * s, x.x * s + x.y * c)
                            : make_float2(x.x * c + x.y * s, x.y * c - x.x * s);
                }
                y[n2 * A + k1] = x;
            }
        }
#pragma unroll
        for (int k1 = 0; k1 < A; ++k1) {
            float2 t[B];
#pragma unroll
            for (int n2 = 0; n2 < B; ++n2) t[n2] = y[n2 * A + k1];
            dft<B, INV>(t);
#pragma unroll
            for (int k2 = 0; k2 < B; ++k2) v[k1 + A * k2] = t[k2];
        }
    }
}

// ------------------------------------------------------------------ shared-memory access
template <int LOGB>
struct SmemLd {
    static constexpr bool kShared = true;
    const float2* p;
    __device__ __forceinline__ float2 operator()(int c, int i) const { return p[(pad16(i) << LOGB) + c]; }
    __device__ __forceinline__ float2 at(int c, int pi) const { return p[(pi << LOGB) + c]; }
};
template <int LOGB>
struct SmemSt {
    static constexpr bool kShared = true;
    float2* p;
    __device__ __forceinline__ void operator()(int c, int i, float2 v) const { p[(pad16(i) << LOGB) + c] = v; }
    __device__ __forceinline__ void at(int c, int pi, float2 v) const { p[(pi << LOGB) + c] = v; }
};

// First-pass source over an unpadded shared buffer (a staged input): element (c, i) at
// p[(i << LOGB) + c].  The first pass reads x[j + r N/R] with consecutive j on consecutive
// lanes, which needs no padding to stay free of bank conflicts.
template <int LOGB>
struct FlatLd {
    const float2* p;
    __device__ __forceinline__ float2 operator()(int c, int i) const { return p[(i << LOGB) + c]; }
};

template <class T, class = void>
struct IsShared { static constexpr bool value = false; };
template <class T>
struct IsShared<T, decltype((void)T::kShared)> { static constexpr bool value = T::kShared; };

struct PassArgs {
    int n, ns;
    uint32_t ns_magic;
    const float2* tw;
};

// One Stockham pass of radix R over a batch of 2^LOGB sequences.
template <int R, bool INV, int LOGB, class Ld, class St>
__device__ __forceinline__ void pass_r(const Ld& ld, const St& st, const PassArgs& a)
{
    const int nb = a.n / R;
    const int total = nb << LOGB;
    for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
        const int c = idx & ((1 << LOGB) - 1);
        const int j = idx >> LOGB;
        const int q = (a.ns == 1) ? j : (int)__umulhi((uint32_t)j, a.ns_magic);
        const int k = j - q * a.ns;
        float2 v[R];
        // Padded shared indices: pad16(j + r nb) = pad16(j) + r (nb + nb / 16) when 16 | nb.
        if constexpr (IsShared<Ld>::value) {
            if ((nb & 15) == 0) {
                const int p0 = pad16(j), ps = nb + (nb >> 4);
#pragma unroll
                for (int r = 0; r < R; ++r) v[r] = ld.at(c, p0 + r * ps);
            } else {
#pragma unroll
                for (int r = 0; r < R; ++r) v[r] = ld(c, j + r * nb);
            }
        } else {
#pragma unroll
            for (int r = 0; r < R; ++r) v[r] = ld(c, j + r * nb);
        }
        if (k > 0) {
            const float2* t = a.tw + k;
#pragma unroll
            for (int r = 1; r < R; ++r) v[r] = twiddle<INV>(v[r], __ldg(t + (r - 1) * a.ns));
        }
        dft<R, INV>(v);
        const int o = q * a.ns * R + k;
        // pad16(o + r ns) = pad16(o) + r (ns + ns / 16) when 16 | ns; a radix-16 first pass
        // (ns = 1, o = 16 q) writes 16 consecutive padded slots.
        if constexpr (IsShared<St>::value) {
            if ((a.ns & 15) == 0 || (R == 16 && a.ns == 1)) {
                const int p0 = pad16(o), ps = (a.ns == 1) ? 1 : a.ns + (a.ns >> 4);
#pragma unroll
                for (int r = 0; r < R; ++r) st.at(c, p0 + r * ps, v[r]);
            } else {
#pragma unroll
                for (int r = 0; r < R; ++r) st(c, o + r * a.ns, v[r]);
            }
        } else {
#pragma unroll
            for (int r = 0; r < R; ++r) st(c, o + r * a.ns, v[r]);
        }
    }
}

// Radices a plan may use (every one has a pass_r instantiation below).
#define WCSIM_FOR_EACH_RADIX(X) \
    X(2) X(3) X(4) X(5) X(6) X(7) X(8) X(10) X(12) X(14) X(15) X(16) X(20) X(24) X(25)

template <bool INV, int LOGB, class Ld, class St>
__device__ __forceinline__ void pass_any(int R, const Ld& ld, const St& st, const PassArgs& a)
{
    switch (R) {
#define WCSIM_CASE(RR) case RR: pass_r<RR, INV, LOGB>(ld, st, a); break;
        WCSIM_FOR_EACH_RADIX(WCSIM_CASE)
#undef WCSIM_CASE
        default: {   // R == 1: a copy
            for (int idx = threadIdx.x; idx < (a.n << LOGB); idx += blockDim.x) {
                const int c = idx & ((1 << LOGB) - 1), i = idx >> LOGB;
                st(c, i, ld(c, i));
            }
        }
    }
}

// Stage the input of an inverse real-pair transform: z[k] = X0[k] + i X1[k], k < n, for two
// Hermitian spectra given by their halves k < nh at columns w0, w1 of blocked slabs s0, s1
// (X1 = 0 when !has1), into the unpadded shared buffer z (read back through FlatLd).  Each
// stored element is read once and also gives the mirror z[n - k] (conj X0 + i conj X1);
// loads are issued in batches of kU per thread before their stores.  With amp (k < nh) the
// noise A(k) xi_w(k) of Eq. 1 is added to each half spectrum on the way (xi from noise_xi,
// key seed, wires w0 and w1).  Ends without a barrier.
__device__ __forceinline__ void stage_herm_pair(const float2* __restrict__ s0,
                                                const float2* __restrict__ s1, int w0, int w1,
                                                bool has1, int n_w, int nh, int n, float2* z,
                                                const float* __restrict__ amp = nullptr,
                                                uint64_t seed = 0, uint32_t plane_id = 0)
{
    constexpr int kU = 6;
    for (int base = threadIdx.x; base < nh; base += kU * blockDim.x) {
        float2 a[kU], b[kU];
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            const int kk = base + u * blockDim.x;
            a[u] = b[u] = make_float2(0.f, 0.f);
            if (kk < nh) {
                a[u] = __ldg(s0 + blk_index(kk, w0, n_w));
                if (has1) b[u] = __ldg(s1 + blk_index(kk, w1, n_w));
            }
        }
        if (amp) {
#pragma unroll
            for (int u = 0; u < kU; ++u) {
                const int kk = base + u * blockDim.x;
                if (kk < nh) {
                    const float A = __ldg(amp + kk);
                    const float2 x0 = noise_xi((uint32_t)w0, kk, n, plane_id, seed);
                    a[u].x = fmaf(A, x0.x, a[u].x);
                    a[u].y = fmaf(A, x0.y, a[u].y);
                    if (has1) {
                        const float2 x1 = noise_xi((uint32_t)w1, kk, n, plane_id, seed);
                        b[u].x = fmaf(A, x1.x, b[u].x);
                        b[u].y = fmaf(A, x1.y, b[u].y);
                    }
                }
            }
        }
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            const int kk = base + u * blockDim.x;
            if (kk < nh) {
                z[kk] = make_float2(a[u].x - b[u].y, a[u].y + b[u].x);
                if (kk > 0 && n - kk >= nh) z[n - kk] = make_float2(a[u].x + b[u].y, b[u].x - a[u].y);
            }
        }
    }
}

// Write the two real rows of an inverse real-pair transform held in the padded buffer z
// (row 0 in .x, row 1 in .y; o1 ignored when !has1), ticks t < n_t.  With vec (rows 16-byte
// aligned, n_t a multiple of 4) a thread writes 4 ticks of each row with one 16-byte store.
__device__ __forceinline__ void store_real_pair(const float2* z, float* __restrict__ o0,
                                                float* __restrict__ o1, int n_t, bool has1,
                                                bool vec)
{
    if (vec) {
        float4* p0 = reinterpret_cast<float4*>(o0);
        float4* p1 = reinterpret_cast<float4*>(o1);
        for (int q = threadIdx.x; q < (n_t >> 2); q += blockDim.x) {
            const int i = pad16(4 * q);            // 4q .. 4q + 3 share one 16-slot group
            const float2 a = z[i], b = z[i + 1], c = z[i + 2], e = z[i + 3];
            p0[q] = make_float4(a.x, b.x, c.x, e.x);
            if (has1) p1[q] = make_float4(a.y, b.y, c.y, e.y);
        }
    } else {
        for (int t = threadIdx.x; t < n_t; t += blockDim.x) {
            const float2 v = z[pad16(t)];
            o0[t] = v.x;
            if (has1) o1[t] = v.y;
        }
    }
}

// store_real_pair for a residual: o = M - target (one FP32 subtraction of the value
// store_real_pair would write) for rows 0 (.x, target t0) and 1 (.y, t1); returns this
// thread's FP32 sum of the squared residuals it wrote.  vec: rows and targets 16-byte
// aligned, n_t a multiple of 4.
__device__ __forceinline__ float store_residual_pair(const float2* z, float* __restrict__ o0,
                                                    float* __restrict__ o1,
                                                    const float* __restrict__ t0,
                                                    const float* __restrict__ t1, int n_t,
                                                    bool has1, bool vec)
{
    float ss = 0.0f;
    if (vec) {
        // the targets' 16-byte loads in batches of kU per row, issued before their use
        constexpr int kU = 6;
        const int nq = n_t >> 2;
        const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int base = threadIdx.x; base < nq; base += kU * blockDim.x) {
            float4 ta[kU], tb[kU];
#pragma unroll
            for (int u = 0; u < kU; ++u) {
                const int q = base + u * blockDim.x;
                ta[u] = tb[u] = zero;
                if (q < nq) {
                    ta[u] = __ldg(reinterpret_cast<const float4*>(t0) + q);
                    if (has1) tb[u] = __ldg(reinterpret_cast<const float4*>(t1) + q);
                }
            }
#pragma unroll
            for (int u = 0; u < kU; ++u) {
                const int q = base + u * blockDim.x;
                if (q < nq) {
                    const int i = pad16(4 * q);
                    const float2 a = z[i], b = z[i + 1], c = z[i + 2], e = z[i + 3];
                    const float4 r0 = make_float4(__fsub_rn(a.x, ta[u].x), __fsub_rn(b.x, ta[u].y),
                                                  __fsub_rn(c.x, ta[u].z), __fsub_rn(e.x, ta[u].w));
                    reinterpret_cast<float4*>(o0)[q] = r0;
                    ss += r0.x * r0.x + r0.y * r0.y + r0.z * r0.z + r0.w * r0.w;
                    if (has1) {
                        const float4 r1 = make_float4(__fsub_rn(a.y, tb[u].x), __fsub_rn(b.y, tb[u].y),
                                                      __fsub_rn(c.y, tb[u].z), __fsub_rn(e.y, tb[u].w));
                        reinterpret_cast<float4*>(o1)[q] = r1;
                        ss += r1.x * r1.x + r1.y * r1.y + r1.z * r1.z + r1.w * r1.w;
                    }
                }
            }
        }
    } else {
        for (int t = threadIdx.x; t < n_t; t += blockDim.x) {
            const float2 v = z[pad16(t)];
            const float r0 = __fsub_rn(v.x, t0[t]);
            o0[t] = r0;
            ss += r0 * r0;
            if (has1) {
                const float r1 = __fsub_rn(v.y, t1[t]);
                o1[t] = r1;
                ss += r1 * r1;
            }
        }
    }
    return ss;
}

// ADC code of waveform value m: clamp(floor(fl(fl(g m) + p) + 1/2), 0, top), each step one
// correctly rounded FP32 operation.
__device__ __forceinline__ uint16_t adc_code(float m, float g, float p, float top)
{
    const float x = __fadd_rn(__fmul_rn(g, m), p);
    const float c = floorf(__fadd_rn(x, 0.5f));
    return (uint16_t)fminf(fmaxf(c, 0.0f), top);
}

// store_real_pair for ADC codes: row 0 (.x) to o0, row 1 (.y) to o1, uint16.  With vec (rows
// 8-byte aligned, n_t a multiple of 4) a thread writes 4 codes per row with one 8-byte store.
__device__ __forceinline__ void store_real_pair_adc(const float2* z, uint16_t* __restrict__ o0,
                                                    uint16_t* __restrict__ o1, int n_t, bool has1,
                                                    bool vec, float g, float p, float top)
{
    if (vec) {
        uint2* p0 = reinterpret_cast<uint2*>(o0);
        uint2* p1 = reinterpret_cast<uint2*>(o1);
        for (int q = threadIdx.x; q < (n_t >> 2); q += blockDim.x) {
            const int i = pad16(4 * q);
            const float2 a = z[i], b = z[i + 1], c = z[i + 2], e = z[i + 3];
            auto pack = [&](float u, float v) {
                return (uint32_t)adc_code(u, g, p, top) | ((uint32_t)adc_code(v, g, p, top) << 16);
            };
            p0[q] = make_uint2(pack(a.x, b.x), pack(c.x, e.x));
            if (has1) p1[q] = make_uint2(pack(a.y, b.y), pack(c.y, e.y));
        }
    } else {
        for (int t = threadIdx.x; t < n_t; t += blockDim.x) {
            const float2 v = z[pad16(t)];
            o0[t] = adc_code(v.x, g, p, top);
            if (has1) o1[t] = adc_code(v.y, g, p, top);
        }
    }
}

// All passes of plan p.  The first pass reads through `first` (global memory or a shared
// buffer outside X/Y), later passes ping-pong between X and Y.  Returns the buffer holding
// the transform; ends with a block barrier.
template <bool INV, int LOGB, class FirstLd>
__device__ __forceinline__ float2* run_plan(const FftPlan& p, const FirstLd& first, float2* X, float2* Y)
{
    float2* dst = X;
    for (int i = 0; i < p.npass; ++i) {
        const PassArgs a = {p.n, p.ns[i], p.ns_magic[i], p.tw + p.tw_off[i]};
        dst = (i & 1) ? Y : X;
        if (i == 0) {
            pass_any<INV, LOGB>(p.radix[0], first, SmemSt<LOGB>{dst}, a);
        } else {
            const float2* src = (i & 1) ? X : Y;
            pass_any<INV, LOGB>(p.radix[i], SmemLd<LOGB>{src}, SmemSt<LOGB>{dst}, a);
        }
        __syncthreads();
    }
    return dst;
}

// ------------------------------------------------------------------ compile-time plans
// Apply the twiddles w^(r k), r = 1 .. R - 1, of a Stockham pass with stride NS to v[1 ..],
// t = the pass's table + k (entry (r - 1) NS = w^(r k)).  Radix 15 loads only the entries of
// r = 1, 5 and 10 and forms the rest as products of them (w^(3k) = w^(5k) conj(w^(2k)) and so
// on, each at most three roundings away from correctly rounded table values), so a butterfly
// reads 3 table entries instead of 14; other radices read every entry.
template <int R, int NS, bool INV>
__device__ __forceinline__ void apply_twiddles(float2* v, const float2* __restrict__ t)
{
    if constexpr (R == 15) {
        const float2 a = __ldg(t), b = __ldg(t + 4 * NS), c = __ldg(t + 9 * NS);
        const float2 na = make_float2(a.x, -a.y);                  // conj: w^(-k)
        const float2 a2 = cmul(a, a), na2 = make_float2(a2.x, -a2.y);
        const float2 a3 = cmul(b, na2), a4 = cmul(b, na);
        float2 w[15];
        w[1] = a;            w[2] = a2;            w[3] = a3;            w[4] = a4;
        w[5] = b;            w[6] = cmul(b, a);    w[7] = cmul(b, a2);   w[8] = cmul(c, na2);
        w[9] = cmul(c, na);  w[10] = c;            w[11] = cmul(c, a);   w[12] = cmul(c, a2);
        w[13] = cmul(c, a3); w[14] = cmul(c, a4);
#pragma unroll
        for (int r = 1; r < R; ++r) v[r] = twiddle<INV>(v[r], w[r]);
    } else {
#pragma unroll
        for (int r = 1; r < R; ++r) v[r] = twiddle<INV>(v[r], __ldg(t + (r - 1) * NS));
    }
}

// One Stockham pass (single sequence) whose length N, radix R and stride NS are template
// parameters, so that every divisor, stride and padded offset is a constant.  Same
// arithmetic and twiddle table layout as pass_r.
template <int R, bool INV, int N, int NS, class Ld, class St>
__device__ __forceinline__ void pass_fixed(const Ld& ld, const St& st, const float2* __restrict__ tw)
{
    constexpr int NB = N / R;
    for (int j = threadIdx.x; j < NB; j += blockDim.x) {
        const int q = j / NS, k = j - q * NS;
        float2 v[R];
        if constexpr (IsShared<Ld>::value && NB % 16 == 0) {
            const int p0 = pad16(j);
#pragma unroll
            for (int r = 0; r < R; ++r) v[r] = ld.at(0, p0 + r * (NB + NB / 16));
        } else {
#pragma unroll
            for (int r = 0; r < R; ++r) v[r] = ld(0, j + r * NB);
        }
        if constexpr (NS > 1) {
            if (k > 0) apply_twiddles<R, NS, INV>(v, tw + k);
        }
        dft<R, INV>(v);
        const int o = q * NS * R + k;
        if constexpr (NS % 16 == 0 || (R == 16 && NS == 1)) {
            constexpr int PS = (NS == 1) ? 1 : NS + NS / 16;
            const int p0 = pad16(o);
#pragma unroll
            for (int r = 0; r < R; ++r) st.at(0, p0 + r * PS, v[r]);
        } else {
#pragma unroll
            for (int r = 0; r < R; ++r) st(0, o + r * NS, v[r]);
        }
    }
}

// The three passes of a plan with radices R0, R1, R2 (p's twiddle table): first -> X,
// X -> Y, Y -> X.  Returns X; ends with a block barrier.
template <bool INV, int R0, int R1, int R2, class FirstLd>
__device__ __forceinline__ float2* run_plan_fixed(const FftPlan& p, const FirstLd& first,
                                                  float2* X, float2* Y)
{
    constexpr int N = R0 * R1 * R2;
    pass_fixed<R0, INV, N, 1>(first, SmemSt<0>{X}, p.tw + p.tw_off[0]);
    __syncthreads();
    pass_fixed<R1, INV, N, R0>(SmemLd<0>{X}, SmemSt<0>{Y}, p.tw + p.tw_off[1]);
    __syncthreads();
    pass_fixed<R2, INV, N, R0 * R1>(SmemLd<0>{Y}, SmemSt<0>{X}, p.tw + p.tw_off[2]);
    __syncthreads();
    return X;
}

// In-place variant of pass_fixed for a block of exactly T threads: every thread first loads
// the inputs of all its butterflies (at most ceil(N / R / T)) into registers, the block
// synchronises, and the outputs are written over the same buffer.  One buffer per sequence
// instead of two, for more CTAs per SM.  Ends with a block barrier.
template <int R, bool INV, int N, int NS, int T, class Ld>
__device__ __forceinline__ void pass_fixed_inplace(const Ld& ld, float2* buf,
                                                   const float2* __restrict__ tw)
{
    constexpr int NB = N / R;
    constexpr int NI = (NB + T - 1) / T;
    float2 v[NI][R];
#pragma unroll
    for (int i = 0; i < NI; ++i) {
        const int j = threadIdx.x + i * T;
        if (j < NB) {
            if constexpr (IsShared<Ld>::value && NB % 16 == 0) {
                const int p0 = pad16(j);
#pragma unroll
                for (int r = 0; r < R; ++r) v[i][r] = ld.at(0, p0 + r * (NB + NB / 16));
            } else {
#pragma unroll
                for (int r = 0; r < R; ++r) v[i][r] = ld(0, j + r * NB);
            }
        }
    }
    __syncthreads();
    const SmemSt<0> st{buf};
#pragma unroll
    for (int i = 0; i < NI; ++i) {
        const int j = threadIdx.x + i * T;
        if (j < NB) {
            const int q = j / NS, k = j - q * NS;
            if constexpr (NS > 1) {
                if (k > 0) apply_twiddles<R, NS, INV>(v[i], tw + k);
            }
            dft<R, INV>(v[i]);
            const int o = q * NS * R + k;
            if constexpr (NS % 16 == 0 || (R == 16 && NS == 1)) {
                constexpr int PS = (NS == 1) ? 1 : NS + NS / 16;
                const int p0 = pad16(o);
#pragma unroll
                for (int r = 0; r < R; ++r) st.at(0, p0 + r * PS, v[i][r]);
            } else {
#pragma unroll
                for (int r = 0; r < R; ++r) st(0, o + r * NS, v[i][r]);
            }
        }
    }
    __syncthreads();
}

// The three passes of plan (R0, R1, R2) in place in X (padded layout on return), the first
// reading through `first` (which may alias X, e.g. FlatLd over the staged input).  A block of
// exactly T threads.  Returns X.
template <bool INV, int R0, int R1, int R2, int T, class FirstLd>
__device__ __forceinline__ float2* run_plan_fixed_inplace(const FftPlan& p, const FirstLd& first,
                                                          float2* X)
{
    constexpr int N = R0 * R1 * R2;
    pass_fixed_inplace<R0, INV, N, 1, T>(first, X, p.tw + p.tw_off[0]);
    pass_fixed_inplace<R1, INV, N, R0, T>(SmemLd<0>{X}, X, p.tw + p.tw_off[1]);
    pass_fixed_inplace<R2, INV, N, R0 * R1, T>(SmemLd<0>{X}, X, p.tw + p.tw_off[2]);
    return X;
}

// Plans with a compile-time variant: the 6000-point transform as radices 16, 25, 15.
enum FixedPlan : int { kPlanRuntime = 0, kPlan6000 = 1 };

__host__ inline int fixed_plan_of(const FftPlan& p)
{
    if (p.n == 6000 && p.npass == 3 && p.radix[0] == 16 && p.radix[1] == 25 && p.radix[2] == 15)
        return kPlan6000;
    return kPlanRuntime;
}

// All passes of a single-sequence plan for a block of T threads whose first pass reads the
// staged input in Z (through FlatLd) and whose result may land in Z or W.  The compile-time
// variant FIX (which must equal fixed_plan_of(p)) runs in place in Z alone; the runtime plan
// ping-pongs between W and Z.  Returns the buffer holding the transform (padded layout).
template <bool INV, int FIX, int T>
__device__ __forceinline__ float2* run_row_plan(const FftPlan& p, float2* Z, float2* W)
{
    if constexpr (FIX == kPlan6000) return run_plan_fixed_inplace<INV, 16, 25, 15, T>(p, FlatLd<0>{Z}, Z);
    else return run_plan<INV, 0>(p, FlatLd<0>{Z}, W, Z);
}

// Shared bytes of a row kernel for transform length n: one padded buffer for the in-place
// compile-time plans, two for the runtime plans.
__host__ inline size_t row_plan_smem(int fix, int n)
{
    return (fix == kPlanRuntime ? 2 : 1) * (size_t)padded_len(n) * sizeof(float2);
}

}  // namespace wcsim
