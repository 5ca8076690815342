/*
 * FP64 CPU oracle for the per-depo stages of the LArTPC signal simulation.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain reference that the CUDA path is
 * checked against.  It shares no code, header or table with the CUDA library, and only the
 * test suite, the smoke check and the benchmark's CPU-baseline leg may load it.
 *
 * What it computes (paper Sec. 2.1.1: "rasterization" and "scatter adding"; Fig. 2: drift
 * and diffusion of the electron clouds; Sec. 4.3.1 and Table 1: fluctuation with a
 * Box-Muller normal):
 *
 *   a1  drift:      t_a = t + t_d,  Q' = Q exp(-t_d / tau),
 *                   sigma_T = sqrt(2 D_T t_d) [mm],  sigma_t = sqrt(2 D_L t_d) / v [us]
 *   a2  rasterize:  per axis, the bins meeting [mu - n sigma, mu + n sigma] (whole bins),
 *                   weight w_k = Phi((e_{k+1}-mu)/sigma) - Phi((e_k-mu)/sigma); patch =
 *                   Q' w^p (x) w^t
 *   a2f fluctuate:  x_b = max(0, mu_b + sqrt(mu_b (1 - mu_b/Q')) z_b), z_b standard normal
 *                   from Philox4x32-10 (Salmon et al., SC'11) and Box-Muller (fluctuate 1);
 *                   or x_b ~ Binomial(N, p_b) exactly (fluctuate 2), N = Q' in whole
 *                   electrons, p_b = mu_b / Q', drawn by inversion of its CDF
 *   a3  scatter:    S[r][k] += x_b, in depo order, in double precision
 *   a7  adjoint:    per-depo gradients of L given dL/dS, with the window held fixed
 *
 * The paper states none of the formulas above; the readings used are:
 *   - which bins a depo covers is an integer decision.  It is taken in the precision the
 *     CUDA kernel uses (position in FP64 bin units, half-width n*sigma/bin in FP32), so that
 *     both sides pick the same bins; everything else here is FP64;
 *   - sigma == 0 (in that FP32 decision) puts all of an axis' weight into the single bin;
 *   - no renormalisation after truncation, unless renormalize is set: then each axis'
 *     weights are divided by their sum T over the whole n-sigma window before it is clipped
 *     to the grid, so that the patch carries Q' less only what falls outside the grid (the
 *     truncation is compensated, the grid border is not).  That window holds the mean, so
 *     T >= erf(n / sqrt 2) never underflows;
 *   - one Philox block per aligned group of four ticks of a row: counter = (k div 4, row r,
 *     depo id, plane id), key = (seed lo, seed hi).  Its four words form two Box-Muller
 *     pairs, u = (x + 0.5) 2^-32, giving four normals
 *       z0 = sqrt(-2 ln u0) cos(2 pi u1),  z1 = sqrt(-2 ln u0) sin(2 pi u1),
 *       z2 = sqrt(-2 ln u2) cos(2 pi u3),  z3 = sqrt(-2 ln u2) sin(2 pi u3);
 *     bin (r, k) takes z_(k mod 4);
 *   - the exact binomial (fluctuate 2; the paper's CPU reference draws from a binomial, Sec.
 *     4.3.2) takes from the same block the uniform u = (floor(x / 2^9) + 0.5) 2^-23 of word
 *     k mod 4 and returns the smallest k with u < F(k; N, p_b), F the binomial CDF.  N is
 *     rint(Q') with Q' formed in FP32 as the kernel forms it (an integer decision taken in
 *     the kernel's precision).  Above N p (1 - p) = 65536 or N = 2^24 the normal
 *     approximation above is used instead;
 *
 * Build: cc -O2 -ffp-contract=off -fopenmp -fPIC -shared wcsim_oracle.c -lm
 * (no FMA contraction: the bin decision must be evaluated operation by operation; OpenMP
 * only spreads og_rasterize_mt's row bands over host threads).
 */
#include <math.h>
#include <omp.h>
#include <stdint.h>
#include <stddef.h>

#define OG_PI 3.14159265358979323846
#define OG_SQRT2 1.41421356237309504880

typedef struct {
    int32_t n_wires, n_imp, n_ticks, pad_;
    double pitch_mm, p0_mm, tick_us, t0_us;
} og_geom;

typedef struct {
    double v_mm_per_us, DL_cm2_s, DT_cm2_s, lifetime_us, nsigma;
    int32_t fluctuate;
    uint32_t plane_id;
    uint64_t seed;
    int32_t renormalize;   /* 1: each axis' weights divided by their sum over the n-sigma
                              window before clipping to the grid */
    int32_t reserved;
} og_params;

/* ---- Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11, "Parallel random numbers: as
 * easy as 1, 2, 3").  Round: (hi0, lo0) = M0 * c0, (hi1, lo1) = M1 * c2,
 * c' = (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0); the key is bumped by the Weyl
 * constants after every round. */
void og_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)M1 * (uint64_t)c2;
        uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
        uint32_t n1 = (uint32_t)p1;
        uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
        uint32_t n3 = (uint32_t)p0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += W0; k1 += W1;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Box-Muller (Box & Muller 1958): two independent standard normals from two words,
 * u = (x + 0.5) 2^-32, in FP64.  which = 0 gives the cosine member, 1 the sine member. */
double og_normal(uint32_t x0, uint32_t x1, int which)
{
    const double two_m32 = 1.0 / 4294967296.0;
    double u1 = ((double)x0 + 0.5) * two_m32;
    double u2 = ((double)x1 + 0.5) * two_m32;
    double rad = sqrt(-2.0 * log(u1));
    return which ? rad * sin(2.0 * OG_PI * u2) : rad * cos(2.0 * OG_PI * u2);
}

/* The normal of bin (row r, tick k): member k mod 4 of the block keyed by k div 4. */
double og_bin_normal(int64_t r, int64_t k, uint32_t id, uint32_t plane_id, const uint32_t key[2])
{
    uint32_t ctr[4] = {(uint32_t)(k >> 2), (uint32_t)r, id, plane_id};
    uint32_t x[4];
    og_philox4x32_10(ctr, key, x);
    int m = (int)(k & 3);
    return (m < 2) ? og_normal(x[0], x[1], m) : og_normal(x[2], x[3], m - 2);
}

/* The uniform of bin (row r, tick k) for the exact binomial: word k mod 4 of the same block,
 * its top 23 bits, (floor(x / 2^9) + 0.5) 2^-23 (exact in FP32 and FP64). */
double og_bin_uniform(int64_t r, int64_t k, uint32_t id, uint32_t plane_id, const uint32_t key[2])
{
    uint32_t ctr[4] = {(uint32_t)(k >> 2), (uint32_t)r, id, plane_id};
    uint32_t x[4];
    og_philox4x32_10(ctr, key, x);
    return ((double)(x[k & 3] >> 9) + 0.5) / 8388608.0;
}

/* Binomial(n, p) drawn by inversion: the smallest k with u < F(k) = sum_{j <= k} P(j),
 * P(j) = C(n, j) p^j (1 - p)^(n - j) evaluated through lgamma, summed from j = 0. */
int64_t og_binomial_draw(int64_t n, double p, double u)
{
    if (n <= 0 || !(p > 0.0)) return 0;
    if (p >= 1.0) return n;
    const double lnf = lgamma((double)n + 1.0), lp = log(p), lq = log1p(-p);
    double F = 0.0;
    for (int64_t j = 0; j < n; ++j) {
        F += exp(lnf - lgamma((double)j + 1.0) - lgamma((double)(n - j) + 1.0) +
                 (double)j * lp + (double)(n - j) * lq);
        if (u < F) return j;
    }
    return n;
}

/* ---- noise (Eq. 1's additive term N(t, x); the paper gives no model, the readings are):
 *   per wire w, the noise is the normalised inverse DFT over n_ft points of A(k) xi_w(k),
 *   with A the plane's amplitude spectrum (k < n_ft/2 + 1, extended as A(n_ft - k) = A(k))
 *   and xi_w(n_ft - k) = conj(xi_w(k)) complex Gaussians of unit mean square:
 *     xi = (z_re + i z_im) / sqrt 2 for 0 < k < n_ft / 2,  xi = z_re at k = 0 and, for even
 *     n_ft, at k = n_ft / 2;
 *   z from Philox4x32-10 with counter (k div 2, w, OG_NOISE_TAG, plane id) and key = the
 *   noise seed: the block's first Box-Muller pair gives (z_re, z_im) of k = 2 (k div 2), the
 *   second those of k + 1. */
#define OG_NOISE_TAG 0x4E4F4953u

/* xi_w(k) for w < n_w, k < nh (nh = n_ft / 2 + 1), row-major [n_w][nh]. */
void og_noise_spectrum(int32_t n_w, int32_t n_ft, uint32_t plane_id, const uint32_t key[2],
                       double* re, double* im)
{
    const int32_t nh = n_ft / 2 + 1;
    for (int32_t w = 0; w < n_w; ++w) {
        for (int32_t k = 0; k < nh; ++k) {
            uint32_t ctr[4] = {(uint32_t)(k >> 1), (uint32_t)w, OG_NOISE_TAG, plane_id};
            uint32_t x[4];
            og_philox4x32_10(ctr, key, x);
            const int m = k & 1;
            const double zr = og_normal(x[2 * m], x[2 * m + 1], 0);
            const double zi = og_normal(x[2 * m], x[2 * m + 1], 1);
            const int real_only = (k == 0) || (2 * k == n_ft);
            re[(size_t)w * nh + k] = real_only ? zr : zr / OG_SQRT2;
            im[(size_t)w * nh + k] = real_only ? 0.0 : zi / OG_SQRT2;
        }
    }
}

/* Per-call constants of the bin decision, formed the same way for every depo. */
typedef struct {
    double inv_dp, inv_dt;          /* 1/(pitch/n_imp), 1/tick, FP64 */
    float two_dt_f, two_dl_f, inv_v_f, nsig_f, inv_dp_f, inv_dt_f;
    float inv_tau_f;                /* 1/lifetime, FP32 (the binomial's trial count) */
} og_consts;

static og_consts make_consts(const og_geom* g, const og_params* pr)
{
    og_consts c;
    double dp = g->pitch_mm / (double)g->n_imp;
    c.inv_dp = 1.0 / dp;
    c.inv_dt = 1.0 / g->tick_us;
    c.two_dt_f = (float)(2.0 * (pr->DT_cm2_s * 1e-4));
    c.two_dl_f = (float)(2.0 * (pr->DL_cm2_s * 1e-4));
    c.inv_v_f = (float)(1.0 / pr->v_mm_per_us);
    c.nsig_f = (float)pr->nsigma;
    c.inv_dp_f = (float)c.inv_dp;
    c.inv_dt_f = (float)c.inv_dt;
    c.inv_tau_f = (float)(1.0 / pr->lifetime_us);
    return c;
}

/* One axis of the bin decision.  x: depo position in bin units (FP64), hw: half-width
 * n*sigma/bin (FP32).  lo_u, hi_u receive the window before clipping to [0, n), lo, hi the
 * clipped one.  Returns 0 if no bin of [0, n) is covered. */
static int axis_window(double x, float hw, int64_t n, int64_t* lo, int64_t* hi,
                       int64_t* lo_u, int64_t* hi_u)
{
    if (!(x > -1e12 && x < 1e12)) return 0;       /* also rejects NaN */
    double i0 = floor(x);
    float frac = (float)(x - i0);
    float a = frac - hw;
    float b = frac + hw;
    double l = i0 + floor((double)a);
    double h = i0 + floor((double)b);
    *lo_u = (int64_t)l;
    *hi_u = (int64_t)h;
    if (l < 0.0) l = 0.0;
    if (h > (double)(n - 1)) h = (double)(n - 1);
    if (l > h) return 0;
    *lo = (int64_t)l;
    *hi = (int64_t)h;
    return 1;
}

/* Everything the oracle derives for one depo (drift, window, FP64 sigmas). */
typedef struct {
    int ok;                        /* 0: contributes nothing */
    int64_t r_lo, r_hi, k_lo, k_hi;
    int64_t r_lo_u, r_hi_u, k_lo_u, k_hi_u;   /* the same windows before clipping */
    double mu_p, mu_t;             /* pitch position [mm] and arrival time [us] */
    double sig_p, sig_t;           /* FP64 sigma_T [mm], sigma_t [us] */
    int delta_p, delta_t;          /* sigma == 0 in the FP32 decision */
    double qatt;                   /* attenuated charge Q' */
    double att;                    /* exp(-t_d / tau) */
} og_depo;

static og_depo drift_and_window(const og_geom* g, const og_params* pr, const og_consts* c,
                                double p, double t, double td, float q)
{
    og_depo d;
    d.ok = 0;
    if (!(td >= 0.0) || !isfinite(p) || !isfinite(t) || !isfinite(td) || !(q >= 0.0f)
        || !isfinite(q))
        return d;
    /* a1: drift */
    d.mu_p = p;
    d.mu_t = t + td;
    d.att = exp(-td / pr->lifetime_us);
    d.qatt = (double)q * d.att;
    if (!(q > 0.0f)) return d;                    /* no charge: covers nothing */
    d.sig_p = sqrt(2.0 * (pr->DT_cm2_s * 1e-4) * td);
    d.sig_t = sqrt(2.0 * (pr->DL_cm2_s * 1e-4) * td) / pr->v_mm_per_us;
    /* the bin decision, in the kernel's precision */
    float td_f = (float)td;
    float sp_f = sqrtf(c->two_dt_f * td_f);
    float st_f = sqrtf(c->two_dl_f * td_f) * c->inv_v_f;
    float hw_p = (c->nsig_f * sp_f) * c->inv_dp_f;
    float hw_t = (c->nsig_f * st_f) * c->inv_dt_f;
    d.delta_p = (sp_f == 0.0f);
    d.delta_t = (st_f == 0.0f);
    double xp = (p - g->p0_mm) * c->inv_dp;
    double xt = (d.mu_t - g->t0_us) * c->inv_dt;
    int64_t nrows = (int64_t)g->n_wires * g->n_imp;
    if (!axis_window(xp, hw_p, nrows, &d.r_lo, &d.r_hi, &d.r_lo_u, &d.r_hi_u)) return d;
    if (!axis_window(xt, hw_t, g->n_ticks, &d.k_lo, &d.k_hi, &d.k_lo_u, &d.k_hi_u)) return d;
    d.ok = 1;
    return d;
}

/* Phi(b') - Phi(a') for a' = ua*sqrt(2), b' = ub*sqrt(2), with the erfc forms in the tails
 * so that far-tail bins keep their relative precision. */
static double gauss_mass(double ua, double ub)
{
    if (ua >= 0.0) return 0.5 * (erfc(ua) - erfc(ub));
    if (ub <= 0.0) return 0.5 * (erfc(-ub) - erfc(-ua));
    return 0.5 * (erf(ub) - erf(ua));
}

/* 1D weights of bins lo..hi: w[i] for bin lo+i, origin/bin in physical units. */
static void axis_weights(double mu, double sig, int delta, double origin, double bin,
                         int64_t lo, int64_t hi, double* w)
{
    int64_t n = hi - lo + 1;
    if (delta) {
        /* sigma == 0: the whole charge sits in the one bin of the window */
        for (int64_t i = 0; i < n; ++i) w[i] = (i == 0) ? 1.0 : 0.0;
        return;
    }
    double s = 1.0 / (OG_SQRT2 * sig);
    for (int64_t i = 0; i < n; ++i) {
        double ea = (origin + (double)(lo + i) * bin) - mu;
        double eb = (origin + (double)(lo + i + 1) * bin) - mu;
        w[i] = gauss_mass(ea * s, eb * s);
    }
}

/* dw/dmu and dw/dsigma of the same bins (window held fixed). */
static void axis_weight_derivs(double mu, double sig, int delta, double origin, double bin,
                               int64_t lo, int64_t hi, double* dmu, double* dsig)
{
    int64_t n = hi - lo + 1;
    if (delta) {
        for (int64_t i = 0; i < n; ++i) { dmu[i] = 0.0; dsig[i] = 0.0; }
        return;
    }
    const double inv_sqrt_2pi = 0.39894228040143267794;
    for (int64_t i = 0; i < n; ++i) {
        double a = ((origin + (double)(lo + i) * bin) - mu) / sig;
        double b = ((origin + (double)(lo + i + 1) * bin) - mu) / sig;
        double pa = inv_sqrt_2pi * exp(-0.5 * a * a);
        double pb = inv_sqrt_2pi * exp(-0.5 * b * b);
        dmu[i] = -(pb - pa) / sig;
        dsig[i] = -(b * pb - a * pa) / sig;
    }
}

#define OG_MAXB 4096

/* Sums over the bins lo..hi of one axis of the weights (T) and, when wanted, of their mu
 * and sigma derivatives (sm, ss), bin by bin with the definitions above, OG_MAXB bins at a
 * time.  Returns 0, or -1 for a window of more than 2^26 bins. */
static int axis_sums(double mu, double sig, int delta, double origin, double bin, int64_t lo,
                     int64_t hi, double* T, double* sm, double* ss)
{
    double w[OG_MAXB], dm[OG_MAXB], ds[OG_MAXB];    /* on the stack: called from threads */
    *T = 0.0;
    if (sm) *sm = 0.0;
    if (ss) *ss = 0.0;
    if (hi - lo + 1 > ((int64_t)1 << 26)) return -1;
    for (int64_t c0 = lo; c0 <= hi; c0 += OG_MAXB) {
        int64_t c1 = (c0 + OG_MAXB - 1 < hi) ? c0 + OG_MAXB - 1 : hi;
        axis_weights(mu, sig, delta, origin, bin, c0, c1, w);
        if (sm) axis_weight_derivs(mu, sig, delta, origin, bin, c0, c1, dm, ds);
        for (int64_t i = 0; i <= c1 - c0; ++i) {
            *T += w[i];
            if (sm) { *sm += dm[i]; *ss += ds[i]; }
        }
    }
    return 0;
}

/* Post-truncation renormalisation of one axis: the n window weights w (and, if not NULL,
 * their derivatives dmu, dsig) divided by the totals T, sm, ss of the unclipped window, by
 * the quotient rule d(w/T) = (dw - (w/T) dT) / T. */
static void renormalize_axis(int64_t n, double* w, double* dmu, double* dsig, double T,
                             double sm, double ss)
{
    for (int64_t i = 0; i < n; ++i) {
        w[i] /= T;
        if (dmu) dmu[i] = (dmu[i] - w[i] * sm) / T;
        if (dsig) dsig[i] = (dsig[i] - w[i] * ss) / T;
    }
}

/* Renormalisation of both axes of depo d (weights, and derivatives when dwp_mu != NULL). */
static int renormalize_depo(const og_geom* g, const og_depo* d, double* wp, double* wt,
                            double* dwp_mu, double* dwp_s, double* dwt_mu, double* dwt_s)
{
    const double dp = g->pitch_mm / (double)g->n_imp;
    double T, sm, ss;
    if (axis_sums(d->mu_p, d->sig_p, d->delta_p, g->p0_mm, dp, d->r_lo_u, d->r_hi_u, &T,
                  dwp_mu ? &sm : NULL, dwp_mu ? &ss : NULL))
        return -1;
    renormalize_axis(d->r_hi - d->r_lo + 1, wp, dwp_mu, dwp_s, T, dwp_mu ? sm : 0.0,
                     dwp_mu ? ss : 0.0);
    if (axis_sums(d->mu_t, d->sig_t, d->delta_t, g->t0_us, g->tick_us, d->k_lo_u, d->k_hi_u,
                  &T, dwt_mu ? &sm : NULL, dwt_mu ? &ss : NULL))
        return -1;
    renormalize_axis(d->k_hi - d->k_lo + 1, wt, dwt_mu, dwt_s, T, dwt_mu ? sm : 0.0,
                     dwt_mu ? ss : 0.0);
    return 0;
}


/* Bins each depo covers: out[4*i + (0..3)] = r_lo, r_hi, k_lo, k_hi, or -1s if none. */
void og_windows(const og_geom* g, const og_params* pr, int64_t n, const double* p,
                const double* t, const double* td, const float* q, int64_t* out)
{
    og_consts c = make_consts(g, pr);
    for (int64_t i = 0; i < n; ++i) {
        og_depo d = drift_and_window(g, pr, &c, p[i], t[i], td[i], q[i]);
        if (d.ok) {
            out[4 * i + 0] = d.r_lo; out[4 * i + 1] = d.r_hi;
            out[4 * i + 2] = d.k_lo; out[4 * i + 3] = d.k_hi;
        } else {
            out[4 * i + 0] = out[4 * i + 1] = out[4 * i + 2] = out[4 * i + 3] = -1;
        }
    }
}

/* 1D weights of one depo along both axes (for the closed-form tests).  wp/wt receive
 * r_hi-r_lo+1 and k_hi-k_lo+1 values; returns 0 if the depo covers nothing. */
int og_depo_weights(const og_geom* g, const og_params* pr, double p, double t, double td,
                    float q, double* qatt, double* wp, double* wt)
{
    og_consts c = make_consts(g, pr);
    og_depo d = drift_and_window(g, pr, &c, p, t, td, q);
    if (!d.ok) return 0;
    double dp = g->pitch_mm / (double)g->n_imp;
    axis_weights(d.mu_p, d.sig_p, d.delta_p, g->p0_mm, dp, d.r_lo, d.r_hi, wp);
    axis_weights(d.mu_t, d.sig_t, d.delta_t, g->t0_us, g->tick_us, d.k_lo, d.k_hi, wt);
    if (pr->renormalize && renormalize_depo(g, &d, wp, wt, NULL, NULL, NULL, NULL)) return 0;
    *qatt = d.qatt;
    return 1;
}

/* What one depo adds, prepared once: its drift and window (d), the exact binomial's trial
 * count n_e = rint(Q') with Q' formed in FP32 as the kernel forms it (an integer decision
 * taken in the kernel's precision). */
typedef struct {
    og_depo d;
    double n_e;
} og_patch;

static og_patch prepare_patch(const og_geom* g, const og_params* pr, const og_consts* c,
                              double p, double t, double td, float q)
{
    og_patch pt;
    pt.d = drift_and_window(g, pr, c, p, t, td, q);
    const float qf = q * expf(-(float)td * c->inv_tau_f);
    pt.n_e = rint((double)qf);
    return pt;
}

/* FP64 weights of rows r0..r1 and ticks k0..k1 of the patch (sub-ranges of its window),
 * renormalised over the unclipped window when asked.  Returns 0, or -1 for a window the
 * fixed buffers cannot hold. */
static int patch_weights(const og_geom* g, const og_params* pr, const og_depo* d, int64_t r0,
                         int64_t r1, int64_t k0, int64_t k1, double* wp, double* wt)
{
    const double dp = g->pitch_mm / (double)g->n_imp;
    if (r1 - r0 + 1 > OG_MAXB || k1 - k0 + 1 > OG_MAXB) return -1;
    axis_weights(d->mu_p, d->sig_p, d->delta_p, g->p0_mm, dp, r0, r1, wp);
    axis_weights(d->mu_t, d->sig_t, d->delta_t, g->t0_us, g->tick_us, k0, k1, wt);
    if (d->delta_p && r0 != d->r_lo) wp[0] = 0.0;   /* the one bin is the window's first */
    if (d->delta_t && k0 != d->k_lo) wt[0] = 0.0;
    if (pr->renormalize) {
        double T;
        if (axis_sums(d->mu_p, d->sig_p, d->delta_p, g->p0_mm, dp, d->r_lo_u, d->r_hi_u, &T,
                      NULL, NULL))
            return -1;
        renormalize_axis(r1 - r0 + 1, wp, NULL, NULL, T, 0.0, 0.0);
        if (axis_sums(d->mu_t, d->sig_t, d->delta_t, g->t0_us, g->tick_us, d->k_lo_u,
                      d->k_hi_u, &T, NULL, NULL))
            return -1;
        renormalize_axis(k1 - k0 + 1, wt, NULL, NULL, T, 0.0, 0.0);
    }
    return 0;
}

/* The value a depo adds to bin (r, k) given its weights there: the mean Q' wp wt, or its
 * normal approximation (fluctuate 1), or the exact binomial draw (fluctuate 2).  When n_out
 * is not NULL it receives the draw's trial count, p_b and uniform (n_out = -1: no draw). */
static double bin_value(const og_params* pr, const og_patch* pt, double wpr, double wtk,
                        int64_t r, int64_t k, uint32_t id, const uint32_t key[2],
                        double* n_out, double* p_out, double* u_out)
{
    const og_depo* d = &pt->d;
    double mean = d->qatt * wpr * wtk;
    double val = mean;
    double pb = wpr * wtk;                       /* mu_b / Q' */
    if (pb > 1.0) pb = 1.0;
    if (n_out) { *n_out = -1.0; *p_out = pb; *u_out = 0.0; }
    if (pr->fluctuate == 2 && pt->n_e * pb * (1.0 - pb) <= 65536.0 && pt->n_e <= 16777216.0) {
        if (mean > 0.0) {
            double u = og_bin_uniform(r, k, id, pr->plane_id, key);
            val = (double)og_binomial_draw((int64_t)pt->n_e, pb, u);
            if (n_out) { *n_out = pt->n_e; *u_out = u; }
        }
    } else if (pr->fluctuate) {
        /* normal approximation to Binomial(Q', mean/Q') */
        double z = og_bin_normal(r, k, id, pr->plane_id, key);
        double var = mean * (1.0 - mean / d->qatt);
        if (var < 0.0) var = 0.0;
        val = mean + sqrt(var) * z;
        if (val < 0.0) val = 0.0;
    }
    return val;
}

/* a1-a3 (+a2f): accumulate every depo's patch into grid[n_rows][n_ticks] (FP64), in depo
 * order.  row_slot (may be NULL) restricts it to rows r with row_slot[r] >= 0, written to
 * row row_slot[r] of grid instead. */
static int rasterize_into(const og_geom* g, const og_params* pr, int64_t n, const double* p,
                          const double* t, const double* td, const float* q,
                          const uint32_t* id, const int64_t* row_slot, double* grid)
{
    static double wp[OG_MAXB], wt[OG_MAXB];
    og_consts c = make_consts(g, pr);
    const int64_t nt = g->n_ticks;
    const uint32_t key[2] = {(uint32_t)pr->seed, (uint32_t)(pr->seed >> 32)};
    for (int64_t i = 0; i < n; ++i) {
        og_patch pt = prepare_patch(g, pr, &c, p[i], t[i], td[i], q[i]);
        const og_depo* d = &pt.d;
        if (!d->ok || !(d->qatt > 0.0)) continue;   /* Q' underflowed: adds nothing */
        if (patch_weights(g, pr, d, d->r_lo, d->r_hi, d->k_lo, d->k_hi, wp, wt)) return -1;
        for (int64_t r = d->r_lo; r <= d->r_hi; ++r) {
            if (row_slot && row_slot[r] < 0) continue;
            double* row = grid + (row_slot ? row_slot[r] : r) * nt;
            for (int64_t k = d->k_lo; k <= d->k_hi; ++k)
                row[k] += bin_value(pr, &pt, wp[r - d->r_lo], wt[k - d->k_lo], r, k, id[i],
                                    key, NULL, NULL, NULL);
        }
    }
    return 0;
}

int og_rasterize(const og_geom* g, const og_params* pr, int64_t n, const double* p,
                 const double* t, const double* td, const float* q, const uint32_t* id,
                 double* grid)
{
    return rasterize_into(g, pr, n, p, t, td, q, id, NULL, grid);
}

/* og_rasterize restricted to the n_sel rows rows[] (distinct): out[j][n_ticks] receives row
 * rows[j] of the grid og_rasterize would produce, bit for bit.  row_slot: scratch of
 * n_wires * n_imp entries. */
int og_rasterize_rows(const og_geom* g, const og_params* pr, int64_t n, const double* p,
                      const double* t, const double* td, const float* q, const uint32_t* id,
                      int64_t n_sel, const int64_t* rows, int64_t* row_slot, double* out)
{
    const int64_t n_rows = (int64_t)g->n_wires * g->n_imp;
    for (int64_t r = 0; r < n_rows; ++r) row_slot[r] = -1;
    for (int64_t j = 0; j < n_sel; ++j) {
        if (rows[j] < 0 || rows[j] >= n_rows || row_slot[rows[j]] >= 0) return -2;
        row_slot[rows[j]] = j;
    }
    return rasterize_into(g, pr, n, p, t, td, q, id, row_slot, out);
}

/* The terms of bin (r, k): for each depo whose window holds the bin, in depo order, its
 * index, the value it adds, and the trial count, p_b and uniform of its binomial draw
 * (n_e = -1 where it draws none).  At most max_out terms; returns their count, or -1. */
int64_t og_bin_terms(const og_geom* g, const og_params* pr, int64_t n, const double* p,
                     const double* t, const double* td, const float* q, const uint32_t* id,
                     int64_t r, int64_t k, int64_t max_out, int64_t* idx, double* val,
                     double* n_e, double* pb, double* u)
{
    double wpr, wtk;
    og_consts c = make_consts(g, pr);
    const uint32_t key[2] = {(uint32_t)pr->seed, (uint32_t)(pr->seed >> 32)};
    int64_t m = 0;
    for (int64_t i = 0; i < n; ++i) {
        og_patch pt = prepare_patch(g, pr, &c, p[i], t[i], td[i], q[i]);
        const og_depo* d = &pt.d;
        if (!d->ok || !(d->qatt > 0.0)) continue;
        if (r < d->r_lo || r > d->r_hi || k < d->k_lo || k > d->k_hi) continue;
        if (m >= max_out) return -1;
        if (patch_weights(g, pr, d, r, r, k, k, &wpr, &wtk)) return -1;
        idx[m] = i;
        val[m] = bin_value(pr, &pt, wpr, wtk, r, k, id[i], key, &n_e[m], &pb[m], &u[m]);
        ++m;
    }
    return m;
}

/* og_rasterize on n_threads host threads (OpenMP; 0: the runtime's default), bit for bit
 * the same grid: the depos' drift and windows are prepared in parallel, then each thread
 * fills whole bands of rows, adding every depo that reaches the band in depo order, so that
 * every bin sums its terms in the same order as the serial loop (no reduction). */
int og_rasterize_mt(const og_geom* g, const og_params* pr, int64_t n, const double* p,
                    const double* t, const double* td, const float* q, const uint32_t* id,
                    int n_threads, og_patch* scratch, double* grid)
{
    og_consts c = make_consts(g, pr);
    const int64_t nt = g->n_ticks, n_rows = (int64_t)g->n_wires * g->n_imp;
    const uint32_t key[2] = {(uint32_t)pr->seed, (uint32_t)(pr->seed >> 32)};
    const int64_t band = 32;
    const int64_t n_bands = (n_rows + band - 1) / band;
    int rc = 0;
    if (n_threads <= 0) n_threads = omp_get_max_threads();
#pragma omp parallel for num_threads(n_threads) schedule(static)
    for (int64_t i = 0; i < n; ++i) scratch[i] = prepare_patch(g, pr, &c, p[i], t[i], td[i], q[i]);
#pragma omp parallel num_threads(n_threads)
    {
        double wp[OG_MAXB], wt[OG_MAXB];
#pragma omp for schedule(dynamic, 1)
        for (int64_t b = 0; b < n_bands; ++b) {
            const int64_t b0 = b * band, b1 = (b0 + band - 1 < n_rows) ? b0 + band - 1 : n_rows - 1;
            for (int64_t i = 0; i < n; ++i) {
                const og_patch* pt = &scratch[i];
                const og_depo* d = &pt->d;
                if (!d->ok || !(d->qatt > 0.0)) continue;
                if (d->r_hi < b0 || d->r_lo > b1) continue;
                const int64_t r0 = d->r_lo > b0 ? d->r_lo : b0;
                const int64_t r1 = d->r_hi < b1 ? d->r_hi : b1;
                if (patch_weights(g, pr, d, r0, r1, d->k_lo, d->k_hi, wp, wt)) {
#pragma omp atomic write
                    rc = -1;
                    continue;
                }
                for (int64_t r = r0; r <= r1; ++r) {
                    double* row = grid + r * nt;
                    for (int64_t k = d->k_lo; k <= d->k_hi; ++k)
                        row[k] += bin_value(pr, pt, wp[r - r0], wt[k - d->k_lo], r, k, id[i],
                                            key, NULL, NULL, NULL);
                }
            }
        }
    }
    return rc;
}

/* Size of one og_rasterize_mt scratch entry, for the caller's allocation. */
int64_t og_patch_bytes(void) { return (int64_t)sizeof(og_patch); }

/* a7, per-depo part: given dS = dL/dS (FP64 grid), the gradients of L with respect to
 * each depo's charge Q, pitch position p, time t, sigma_L [mm], sigma_T [mm] (mean path,
 * window fixed), and the sums over depos for D_L, D_T [cm^2/s] and tau [us].
 * glob[0..2] = dL/dD_L, dL/dD_T, dL/dtau. */
int og_depo_grads(const og_geom* g, const og_params* pr, int64_t n, const double* p,
                  const double* t, const double* td, const float* q, const double* dS,
                  double* dq, double* dpos, double* dt, double* dsl, double* dst,
                  double* glob)
{
    static double wp[OG_MAXB], wt[OG_MAXB], dwp_mu[OG_MAXB], dwp_s[OG_MAXB],
        dwt_mu[OG_MAXB], dwt_s[OG_MAXB];
    og_consts c = make_consts(g, pr);
    double dpitch = g->pitch_mm / (double)g->n_imp;
    const int64_t nt = g->n_ticks;
    glob[0] = glob[1] = glob[2] = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        dq[i] = dpos[i] = dt[i] = dsl[i] = dst[i] = 0.0;
        og_depo d = drift_and_window(g, pr, &c, p[i], t[i], td[i], q[i]);
        if (!d.ok) continue;
        if (d.r_hi - d.r_lo + 1 > OG_MAXB || d.k_hi - d.k_lo + 1 > OG_MAXB) return -1;
        axis_weights(d.mu_p, d.sig_p, d.delta_p, g->p0_mm, dpitch, d.r_lo, d.r_hi, wp);
        axis_weights(d.mu_t, d.sig_t, d.delta_t, g->t0_us, g->tick_us, d.k_lo, d.k_hi, wt);
        axis_weight_derivs(d.mu_p, d.sig_p, d.delta_p, g->p0_mm, dpitch, d.r_lo, d.r_hi,
                           dwp_mu, dwp_s);
        axis_weight_derivs(d.mu_t, d.sig_t, d.delta_t, g->t0_us, g->tick_us, d.k_lo,
                           d.k_hi, dwt_mu, dwt_s);
        if (pr->renormalize &&
            renormalize_depo(g, &d, wp, wt, dwp_mu, dwp_s, dwt_mu, dwt_s))
            return -1;
        double a_q = 0.0, a_pm = 0.0, a_ps = 0.0, a_tm = 0.0, a_ts = 0.0;
        for (int64_t r = d.r_lo; r <= d.r_hi; ++r) {
            const double* row = dS + r * nt;
            int64_t ir = r - d.r_lo;
            for (int64_t k = d.k_lo; k <= d.k_hi; ++k) {
                int64_t ik = k - d.k_lo;
                double s = row[k];
                a_q += s * wp[ir] * wt[ik];
                a_pm += s * dwp_mu[ir] * wt[ik];
                a_ps += s * dwp_s[ir] * wt[ik];
                a_tm += s * wp[ir] * dwt_mu[ik];
                a_ts += s * wp[ir] * dwt_s[ik];
            }
        }
        double dqatt = a_q;                         /* dL/dQ' */
        dq[i] = dqatt * d.att;                      /* Q' = Q exp(-t_d/tau) */
        dpos[i] = d.qatt * a_pm;                    /* mu_p = p */
        dt[i] = d.qatt * a_tm;                      /* t_a = t + t_d */
        dst[i] = d.qatt * a_ps;                     /* sigma_T [mm] */
        double dsig_t = d.qatt * a_ts;              /* sigma_t [us] */
        dsl[i] = dsig_t / pr->v_mm_per_us;          /* sigma_t = sigma_L / v */
        /* sigma = sqrt(2 D t_d): dsigma/dD = sigma / (2 D) */
        if (pr->DL_cm2_s > 0.0) glob[0] += dsl[i] * (d.sig_t * pr->v_mm_per_us) / (2.0 * pr->DL_cm2_s);
        if (pr->DT_cm2_s > 0.0) glob[1] += dst[i] * d.sig_p / (2.0 * pr->DT_cm2_s);
        /* dQ'/dtau = Q' t_d / tau^2 */
        glob[2] += dqatt * d.qatt * td[i] / (pr->lifetime_us * pr->lifetime_us);
    }
    return 0;
}
