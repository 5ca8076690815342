// Host side of the FFT engine: choosing the radices of a plan and its twiddle table.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <vector>

#include "wcsim_internal.cuh"

namespace wcsim {

namespace {

// Radices with a register DFT (the WCSIM_FOR_EACH_RADIX list in fft_engine.cuh), with a rough per-element
// arithmetic cost used to rank plans of the same pass count.
struct RadixCost {
    int r;
    double cost;
};
const RadixCost kRadices[] = {{2, 2.0},  {3, 4.0},  {4, 4.0},  {5, 6.8},  {6, 6.0},
                              {7, 10.0}, {8, 5.5},  {10, 7.2}, {12, 7.3}, {14, 11.0},
                              {15, 9.0}, {16, 6.5}, {20, 8.5}, {24, 8.7}, {25, 10.8}};

// Fewest passes first (each pass is a round trip through shared memory), then the
// smallest arithmetic; depth-first over divisors.
void search(int n, int depth, int* cur, double cost, int* best, int* best_len, double* best_cost)
{
    if (n == 1) {
        const double total = cost + 100.0 * depth;
        if (*best_len < 0 || total < *best_cost) {
            *best_cost = total;
            *best_len = depth;
            for (int i = 0; i < depth; ++i) best[i] = cur[i];
        }
        return;
    }
    if (depth >= kMaxPasses) return;
    if (*best_len >= 0 && cost + 100.0 * (depth + 1) >= *best_cost) return;
    const int nr = (int)(sizeof(kRadices) / sizeof(kRadices[0]));
    for (int i = nr - 1; i >= 0; --i) {       // large radices first: good plans early
        const RadixCost& rc = kRadices[i];
        if (n % rc.r) continue;
        cur[depth] = rc.r;
        search(n / rc.r, depth + 1, cur, cost + rc.cost, best, best_len, best_cost);
    }
}

uint32_t magic_for(int d) { return d <= 1 ? 0u : (uint32_t)((0x100000000ull + d - 1) / (uint64_t)d); }

}  // namespace

bool fft_factor(int n, int32_t* radix, int32_t* npass)
{
    if (n < 1) return false;
    if (n == 1) {
        radix[0] = 1;
        *npass = 1;
        return true;
    }
    int cur[kMaxPasses], best[kMaxPasses], best_len = -1;
    double best_cost = 0.0;
    search(n, 0, cur, 0.0, best, &best_len, &best_cost);
    if (best_len < 0) return false;
    // larger radices first: the first pass carries no twiddles
    for (int i = 0; i < best_len; ++i)
        for (int k = i + 1; k < best_len; ++k)
            if (best[k] > best[i]) { int t = best[i]; best[i] = best[k]; best[k] = t; }
    // A radix-16 first pass writes with stride 16, which the one-slot-per-16 padding of
    // the shared buffers spreads over all banks; other even first radices (12, 20, 24)
    // collide 2-8 ways.  Take 16 first whenever that costs no extra pass.
    if (n % 16 == 0 && n > 16) {
        int rest[kMaxPasses], rest_len = -1;
        double rest_cost = 0.0;
        search(n / 16, 0, cur, 0.0, rest, &rest_len, &rest_cost);
        if (rest_len >= 0 && rest_len + 1 <= best_len) {
            for (int i = 0; i < rest_len; ++i)
                for (int k = i + 1; k < rest_len; ++k)
                    if (rest[k] > rest[i]) { int t = rest[i]; rest[i] = rest[k]; rest[k] = t; }
            best[0] = 16;
            for (int i = 0; i < rest_len; ++i) best[i + 1] = rest[i];
            best_len = rest_len + 1;
        }
    }
    for (int i = 0; i < best_len; ++i) radix[i] = best[i];
    *npass = best_len;
    return true;
}

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
        // twiddle (k, r) = exp(-2 pi i r k / (ns R)), stored at (r - 1) ns + k so that the
        // lanes of a warp (consecutive k) read consecutive entries
        for (int r = 1; r < R; ++r)
            for (int k = 0; k < ns; ++k) {
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

}  // namespace wcsim

namespace wcsim {

int fft_plan_describe(int n, FftPlan* plan)
{
    FftPlan p{};
    p.n = n;
    if (!fft_factor(n, p.radix, &p.npass)) return -1;
    int ns = 1, len = 0;
    for (int i = 0; i < p.npass; ++i) {
        const int R = p.radix[i];
        p.ns[i] = ns;
        p.tw_off[i] = len;
        p.ns_magic[i] = magic_for(ns);
        len += (R - 1) * ns;
        ns *= R;
    }
    p.tw = nullptr;
    *plan = p;
    return len < 1 ? 1 : len;
}

}  // namespace wcsim

namespace wcsim {

namespace {

void collect(int n, int depth, int max_depth, int* cur, double cost, int (*out)[kMaxPasses],
             int* lens, double* costs, int* count, int cap)
{
    if (n == 1) {
        // keep the `cap` cheapest (insertion into a short sorted list)
        int pos = *count < cap ? (*count)++ : cap - 1;
        if (pos == cap - 1 && *count == cap && costs[pos] <= cost && lens[pos] > 0) return;
        while (pos > 0 && costs[pos - 1] > cost) {
            costs[pos] = costs[pos - 1];
            lens[pos] = lens[pos - 1];
            for (int i = 0; i < kMaxPasses; ++i) out[pos][i] = out[pos - 1][i];
            --pos;
        }
        costs[pos] = cost;
        lens[pos] = depth;
        for (int i = 0; i < depth; ++i) out[pos][i] = cur[i];
        return;
    }
    if (depth >= max_depth) return;
    const int nr = (int)(sizeof(kRadices) / sizeof(kRadices[0]));
    // non-increasing radices: each multiset once
    for (int i = nr - 1; i >= 0; --i) {
        const int r = kRadices[i].r;
        if (n % r || (depth > 0 && r > cur[depth - 1])) continue;
        cur[depth] = r;
        collect(n / r, depth + 1, max_depth, cur, cost + kRadices[i].cost, out, lens, costs, count, cap);
    }
}

}  // namespace

int fft_plan_candidates(int n, int32_t (*radix)[kMaxPasses], int32_t* npass, int max_out)
{
    int32_t best[kMaxPasses], nb;
    if (!fft_factor(n, best, &nb)) return 0;
    int count = 0;
    for (int i = 0; i < nb && count < max_out; ++i) radix[count][i] = best[i];
    npass[count++] = nb;
    if (nb <= 1) return count;
    // other radix sets with the same number of passes, cheapest first, each tried with its
    // radices in decreasing order and, where it has one, a radix-16 first pass
    const int cap = 8;
    int out[cap][kMaxPasses], lens[cap];
    double costs[cap];
    int cnt = 0, cur[kMaxPasses];
    for (int i = 0; i < cap; ++i) { lens[i] = 0; costs[i] = 1e300; }
    collect(n, 0, nb, cur, 0.0, out, lens, costs, &cnt, cap);
    for (int c = 0; c < cnt && count < max_out; ++c) {
        for (int variant = 0; variant < 2 && count < max_out; ++variant) {
            int32_t r[kMaxPasses];
            for (int i = 0; i < lens[c]; ++i) r[i] = out[c][i];     // decreasing already
            if (variant == 1) {
                int k = -1;
                for (int i = 0; i < lens[c]; ++i) if (r[i] == 16) k = i;
                if (k <= 0) continue;
                for (int i = k; i > 0; --i) r[i] = r[i - 1];
                r[0] = 16;
            }
            bool dup = false;
            for (int q = 0; q < count && !dup; ++q) {
                if (npass[q] != lens[c]) continue;
                bool same = true;
                for (int i = 0; i < lens[c]; ++i) same = same && radix[q][i] == r[i];
                dup = same;
            }
            if (dup) continue;
            for (int i = 0; i < lens[c]; ++i) radix[count][i] = r[i];
            npass[count++] = lens[c];
        }
    }
    return count;
}

cudaError_t fft_plan_create_radices(int n, const int32_t* radices, int npass, FftPlan* plan,
                                    float2** dev_tw)
{
    FftPlan p{};
    p.n = n;
    p.npass = npass;
    int prod = 1;
    for (int i = 0; i < npass; ++i) { p.radix[i] = radices[i]; prod *= radices[i]; }
    if (prod != n || npass < 1 || npass > kMaxPasses) return cudaErrorInvalidValue;
    std::vector<float2> tw;
    int ns = 1;
    for (int i = 0; i < p.npass; ++i) {
        const int R = p.radix[i];
        p.ns[i] = ns;
        p.tw_off[i] = (int32_t)tw.size();
        p.ns_magic[i] = magic_for(ns);
        for (int r = 1; r < R; ++r)
            for (int k = 0; k < ns; ++k) {
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

}  // namespace wcsim
