// Per-depo drift and bin decision shared by the rasterizers and the adjoint (Sec. 2.1.1
// "rasterization"; drift and diffusion as in Fig. 2): the FP64 placement of a depo on the
// impact x tick grid, the FP32 window half-widths, and the FP32 bin masses from erfc edge
// terms.  Every kernel that rasterizes a depo takes its window and weights from these
// functions, so that all of them add the same values.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "async_copy.cuh"
#include "wcsim_internal.cuh"

namespace wcsim {

struct Decision {                // 64 bytes, no padding
    int64_t i0p, i0t;           // floor of the depo position in bin units
    int32_t ok;                 // covers >= 1 bin and carries charge
    int32_t r_lo, r_hi, k_lo, k_hi;
    float frac_p, frac_t;       // position - floor, FP32
    float sp, st;               // sigma_T [mm], sigma_t [us] (FP32)
    float qatt;                 // Q' = Q exp(-t_d / lifetime)
    float qw;                   // scale of the weight products: Q', or Q' / (T_p T_t) when
                                // each axis is renormalised over its window
    uint32_t id;                // depo id (fluctuation key)
};
static_assert(sizeof(Decision) == kDecisionBytes, "Decision packs into 64 bytes");

// Normal mass between two edges at u = offset / (sqrt(2) sigma) from their edge terms
// ea = erfc|ua|, eb = erfc|ub|: 0.5 (erfc ua - erfc ub) on the upper side of the mean,
// 0.5 (erfc -ub - erfc -ua) on the lower side (both keep relative precision in the tails),
// 1 - 0.5 (ea + eb) for a span holding the mean.
static __device__ __forceinline__ float span_mass(float ua, float ub, float ea, float eb)
{
    if (ua >= 0.0f) return 0.5f * (ea - eb);
    if (ub <= 0.0f) return 0.5f * (eb - ea);
    return 1.0f - 0.5f * (ea + eb);
}

// Edge u of one axis' n-sigma window before it is clipped to the grid: the lower edge
// floor(frac - hw) or the upper edge floor(frac + hw) + 1 (offsets from the floor of the
// position, in bins; the same FP32 operations as the bin decision).
static __device__ __forceinline__ float outer_edge_u(float frac, float hw, float s, bool upper)
{
    const float e = upper ? floorf(__fadd_rn(frac, hw)) + 1.0f : floorf(__fsub_rn(frac, hw));
    return (e - frac) * s;
}

// Total weight T of one axis' unclipped window: the bin masses telescope to the mass
// between its outer edges, which lie on either side of the mean, so T >= erf(n / sqrt 2).
// sigma == 0 (s == 0) puts the whole weight in the window's one bin.
static __device__ __forceinline__ float window_mass(float frac, float hw, float s)
{
    if (!(s > 0.0f)) return 1.0f;
    const float ua = outer_edge_u(frac, hw, s, false);
    const float ub = outer_edge_u(frac, hw, s, true);
    return span_mass(ua, ub, erfcf(fabsf(ua)), erfcf(fabsf(ub)));
}

// One axis of the bin decision.  Every operation is an explicitly rounded IEEE operation
// (no contraction), so that the result is a function of the inputs alone.  The window edges
// i0 + floor(frac -+ hw) are sums of whole numbers below 2^53, exact in FP64 and formed here
// in 64-bit integers instead (FP64 runs at a small fraction of the FP32 rate on this part):
// floor of a float is floorf, and clamping it to +-2^42 (far beyond |i0| < 10^12 and the grid)
// changes no clipped edge.
static __device__ __forceinline__ bool axis_window(double x, float hw, int64_t n, int32_t& lo,
                                            int32_t& hi, int64_t& i0i, float& frac)
{
    if (!(fabs(x) < 1e12)) return false;
    const double i0 = floor(x);
    frac = __double2float_rn(__dsub_rn(x, i0));
    const float a = __fsub_rn(frac, hw);
    const float b = __fadd_rn(frac, hw);
    constexpr float kEdge = 4398046511104.0f;      // 2^42
    i0i = (int64_t)i0;
    int64_t l = i0i + (int64_t)fminf(fmaxf(floorf(a), -kEdge), kEdge);
    int64_t h = i0i + (int64_t)fminf(fmaxf(floorf(b), -kEdge), kEdge);
    if (l < 0) l = 0;
    if (h > n - 1) h = n - 1;
    if (l > h) return false;
    lo = (int32_t)l;
    hi = (int32_t)h;
    return true;
}

// isfinite for a double by its exponent bits (integer operations, not the FP64 pipe).
static __device__ __forceinline__ bool finite_bits(double x)
{
    return ((__double_as_longlong(x) >> 52) & 0x7ff) != 0x7ff;
}

// Drift (t_a = t + t_d, Q' = Q e^{-t_d/tau}, sigma = sqrt(2 D t_d)) and the window of bins
// whose span meets [mu - n sigma, mu + n sigma], clipped to the grid.  The weight scale qw
// is formed only when `weights` is set (the forward); elsewhere it is left at Q'.
static __device__ __forceinline__ Decision decide(const RasterConsts& c, const DepoArrays& d,
                                           int64_t i, int* flags, bool weights = false)
{
    Decision r;
    r.ok = 0;
    const double p = d.p[i], t = d.t[i], td = d.td[i];
    const float q = d.q[i];
    // td >= 0 (or -0) and every input finite: sign and exponent bits, integer operations
    const int64_t tdb = __double_as_longlong(td);
    const bool td_neg = tdb < 0 && (tdb & 0x7fffffffffffffffll) != 0;
    if (td_neg || !finite_bits(p) || !finite_bits(t) || !finite_bits(td) || !(q >= 0.0f) ||
        !isfinite(q)) {
        atomicOr(flags, kErrInvalidDepo);
        return r;
    }
    if (!(q > 0.0f)) return r;
    const float td_f = __double2float_rn(td);
    r.sp = __fsqrt_rn(__fmul_rn(c.two_dt, td_f));
    r.st = __fmul_rn(__fsqrt_rn(__fmul_rn(c.two_dl, td_f)), c.inv_v);
    const float hw_p = __fmul_rn(__fmul_rn(c.nsig, r.sp), c.inv_dp_f);
    const float hw_t = __fmul_rn(__fmul_rn(c.nsig, r.st), c.inv_dt_f);
    const double ta = __dadd_rn(t, td);
    const double xp = __dmul_rn(__dsub_rn(p, c.p0), c.inv_dp);
    const double xt = __dmul_rn(__dsub_rn(ta, c.t0), c.inv_dt);
    if (!axis_window(xp, hw_p, c.n_rows, r.r_lo, r.r_hi, r.i0p, r.frac_p)) return r;
    if (!axis_window(xt, hw_t, c.n_ticks, r.k_lo, r.k_hi, r.i0t, r.frac_t)) return r;
    r.qatt = q * expf(-td_f * c.inv_tau);
    r.qw = r.qatt;
    if (weights && c.renorm) {
        // each axis' weights divided by their sum T over the n-sigma window before it is
        // clipped to the grid: the truncation is compensated, charge beyond the grid's
        // border stays lost
        const float s_p = (r.sp > 0.0f) ? c.dp_f / (1.41421356237309505f * r.sp) : 0.0f;
        const float s_t = (r.st > 0.0f) ? c.dt_f / (1.41421356237309505f * r.st) : 0.0f;
        r.qw = r.qatt / (window_mass(r.frac_p, hw_p, s_p) * window_mass(r.frac_t, hw_t, s_t));
    }
    r.ok = 1;
    return r;
}

// erfc(|u|) at bin edge u = (koff - frac) s: the edge term of the bin masses below.
static __device__ __forceinline__ float edge_erfc(int64_t koff, float frac, float s)
{
    return erfcf(fabsf(((float)koff - frac) * s));
}

// Mass of the bin [koff, koff + 1) (offset from the floor of the position, in bins) from
// its edge terms ea = erfc|ua|, eb = erfc|ub|.
static __device__ __forceinline__ float bin_mass(int64_t koff, float frac, float s, float ea, float eb)
{
    const float ua = ((float)koff - frac) * s;
    const float ub = ((float)(koff + 1) - frac) * s;
    return span_mass(ua, ub, ea, eb);
}

}  // namespace wcsim
