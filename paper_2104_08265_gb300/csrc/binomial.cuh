// Exact binomial draws, Binomial(n, p), by inversion of the CDF in FP32: the per-bin
// fluctuation that the paper's CPU reference draws from a binomial distribution (Sec. 4.3.1,
// 4.3.2).  x = the smallest k with u < F(k; n, p).
//
// The mass at the mode comes from the saddle-point form of the binomial pmf (C. Loader,
// "Fast and accurate computation of binomial probabilities", 2000):
//   log P(k) = d(n) - d(k) - d(n - k) - D(k, n p) - D(n - k, n q) + 1/2 log(n / (2 pi k (n - k)))
// with d(m) = log m! - [(m + 1/2) log m - m + 1/2 log 2 pi] (Stirling's remainder) and the
// deviance D(x, M) = x log(x / M) + M - x; each term is small near the mode, so FP32 keeps
// about 1e-7 relative precision where log-gamma differences would lose several digits.  The
// rest of the CDF follows from the ratio recurrence P(k - 1) = P(k) k q / ((n - k + 1) p).
#pragma once

#include <math.h>
#include <stdint.h>

namespace wcsim {

// Terms of the CDF below this are dropped from the sum at the mode (the uniforms have 23
// bits, the smallest is 2^-24; the dropped tail stays below 1e-8).
constexpr float kBinomTiny = 2.3283064e-10f;   // 2^-32

// Stirling's remainder d(m) for whole m >= 1: a table (made on the host from log-gamma in
// FP64) up to 15, the asymptotic series 1/(12 m) - 1/(360 m^3) + 1/(1260 m^5) above
// (the next term is below 4e-10 of the first there).
__device__ __forceinline__ float stirling_remainder(float m, const float* tab)
{
    if (m <= 15.0f) return tab[(int)m];
    const float r = 1.0f / m, r2 = r * r;
    return r * (0.0833333333f - r2 * (0.00277777778f - r2 * 0.000793650794f));
}

// The deviance D(x, M) = x log(x / M) + M - x >= 0.  Near x = M, with v = (x - M)/(x + M),
// x log(x / M) = 2 x atanh v, so D = (x - M) v + 2 x (v^3 / 3 + v^5 / 5 + ...), summed
// until it stops changing.
__device__ __forceinline__ float deviance(float x, float M)
{
    const float d = x - M;
    if (fabsf(d) < 0.1f * (x + M)) {
        const float v = __fdividef(d, x + M), v2 = v * v;
        float s = d * v, e = 2.0f * x * v;
#pragma unroll 1
        for (int j = 1; j < 16; ++j) {
            e *= v2;
            const float s1 = s + __fdividef(e, (float)(2 * j + 1));
            if (s1 == s) break;
            s = s1;
        }
        return s;
    }
    return x * logf(x / M) + M - x;
}

// P(k) of Binomial(n, p), q = 1 - p.
__device__ __forceinline__ float binomial_pmf(float k, float n, float p, float q, const float* tab)
{
    if (k == 0.0f) return expf(n * log1pf(-p));
    if (k == n) return expf(n * logf(p));
    const float lc = stirling_remainder(n, tab) - stirling_remainder(k, tab) -
                     stirling_remainder(n - k, tab) - deviance(k, n * p) - deviance(n - k, n * q);
    const float lf = 0.5f * (logf(n / (k * (n - k))) - 1.83787706640934548f);   // - log 2 pi
    return expf(lc + lf);
}

// Kahan's compensated addition: sum + x with the rounding error carried in comp (the sum
// is sum - comp).  Plain IEEE operations, which nvcc does not reassociate.
__device__ __forceinline__ void kahan_add(float& sum, float& comp, float x)
{
    const float y = __fsub_rn(x, comp);
    const float t = __fadd_rn(sum, y);
    comp = __fsub_rn(__fsub_rn(t, sum), y);
    sum = t;
}

// P(k - 1) (down) or P(k + 1) (up) from P(k) = f by the ratio recurrence, re-anchored on the
// saddle-point form every 32nd step (step counter j) so that rounding does not build up
// along a wide distribution.
__device__ __forceinline__ float binomial_step(bool up, float k, float f, int j, float n, float p,
                                               float q, float qp, float pq, const float* tab)
{
    if ((j & 31) == 0) return binomial_pmf(up ? k + 1.0f : k - 1.0f, n, p, q, tab);
    return up ? f * __fdividef((n - k) * pq, k + 1.0f) : f * __fdividef(k * qp, n - k + 1.0f);
}

// The smallest k with u < F(k; n, p), for whole n in [1, 2^24], 0 < p < 1 and moderate
// n p q (the caller hands larger variances to the normal approximation).  F at the mode
// m = floor((n + 1) p) is summed (compensated) downwards from P(m); the walk then goes down
// while u lies below F(k - 1), or up adding P(k + 1), until u < F(k).  Every loop ends
// within a few standard deviations of the mode, where the terms fall below 2^-32 (u >= 2^-24),
// and the loop counters bound them by n in any case.
__device__ __forceinline__ float binomial_inverse(float n, float p, float u, const float* tab)
{
    const float q = 1.0f - p;
    const float m = fminf(floorf((n + 1.0f) * p), n);
    const float fm = binomial_pmf(m, n, p, q, tab);
    const float qp = __fdividef(q, p), pq = __fdividef(p, q);
    float C = fm, comp = 0.0f, f = fm, k = m;
    // the sum below the mode in segments: 31 recurrence steps, then the 32nd re-anchored
#pragma unroll 1
    while (true) {
        int i = 0;
#pragma unroll 1
        for (; i < 31 && k > 0.0f && f >= kBinomTiny; ++i) {
            f *= __fdividef(k * qp, n - k + 1.0f);
            kahan_add(C, comp, f);
            k -= 1.0f;
        }
        if (i < 31 || !(k > 0.0f && f >= kBinomTiny)) break;
        f = binomial_pmf(k - 1.0f, n, p, q, tab);
        kahan_add(C, comp, f);
        k -= 1.0f;
    }
    C = __fsub_rn(C, comp);
    k = m;
    f = fm;
    int j = 0;
    if (u < C) {
        // (a u below the rounding residue of the sum, ~1e-7, stops where the terms vanish)
#pragma unroll 1
        while (k > 0.0f && f >= kBinomTiny) {
            const float c = C - f;
            if (!(u < c)) break;
            C = c;
            f = binomial_step(false, k, f, ++j, n, p, q, qp, pq, tab);
            k -= 1.0f;
        }
    } else {
        comp = 0.0f;
#pragma unroll 1
        while (k < n) {
            f = binomial_step(true, k, f, ++j, n, p, q, qp, pq, tab);
            k += 1.0f;
            kahan_add(C, comp, f);
            if (u < __fsub_rn(C, comp) || f < kBinomTiny) break;
        }
    }
    return k;
}

// The 23-bit uniform of a Philox word, (floor(x / 2^9) + 1/2) 2^-23 (exact in FP32).
__device__ __forceinline__ float uniform23(uint32_t x)
{
    return (__uint2float_rn(x >> 9) + 0.5f) * 1.1920928955078125e-7f;
}

}  // namespace wcsim
