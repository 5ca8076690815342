// Building blocks of the one-warp-per-time-frequency wire-axis kernels (n_fw = 32 M points,
// a CTA of kBlockCols warps owning one 4-column block of the blocked spectra).
//
// A block tile is [row][4] float2 in global memory (one 32-byte sector per row).  Warps
// read their column straight into registers (all loads of a lane in flight together); tiles
// leave shared memory column by column, s[c * ld + row], written by each warp with
// consecutive lanes on consecutive words and stored by the whole CTA with 16-byte accesses
// (with ld = n + kColPad the four columns start 32 bytes apart modulo 128, so the
// transposing reads are free of bank conflicts).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "fft_engine.cuh"
#include "wcsim_internal.cuh"

namespace wcsim {

constexpr int kColPad = 4;

__host__ __device__ constexpr int tile_ld(int n) { return n + kColPad; }

// tile[row][c] <- s[c * ld + row] for row < rows, 16-byte stores.  Ends without a barrier.
__device__ __forceinline__ void store_tile_cols(const float2* s, int rows, int ld,
                                                float2* __restrict__ tile)
{
    float4* t4 = reinterpret_cast<float4*>(tile);
    for (int e = threadIdx.x; e < rows * 2; e += blockDim.x) {
        const int row = e >> 1, c0 = (e & 1) * 2;
        const float2 a = s[c0 * ld + row], b = s[(c0 + 1) * ld + row];
        t4[e] = make_float4(a.x, a.y, b.x, b.y);
    }
}

// Twiddles of the wire FFTs, [2][n]: W^(l k2) at k2 * 32 + l, then W^(k2 n2) at n2 M + k2.
template <int M>
__device__ __forceinline__ void load_wire_twiddles(const float2* __restrict__ tw2, float2* s_twf,
                                                   float2* s_twi)
{
    constexpr int N = 32 * M;
    for (int e = threadIdx.x; e < N; e += blockDim.x) {
        if (s_twf) s_twf[e] = tw2[e];
        if (s_twi) s_twi[e] = tw2[N + e];
    }
    __syncthreads();
}

// Forward n-point FFT (n = 32 M) of one column, lane l holding x[l + 32 m] in v[m]: an
// M-point DFT per lane, the twiddle W^(l k2), a transpose through the warp's padded tile tr
// (33 M entries) and a 32-point DFT in lanes k2 < M, which then hold X[k2 + M k1] in u[k1].
// On return the warp may overwrite tr.
template <int M>
__device__ __forceinline__ void warp_fft_fwd(float2 (&v)[M], const float2* s_twf, float2* tr,
                                             int lane, float2 (&u)[32])
{
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
        __syncwarp((1u << M) - 1);            // every reading lane is past its reads
        dft<32, false>(u);
    }
}

// Column c of a blocked tile in global memory into lane registers: v[m] = x[l + 32 m]
// (zero at and above n_valid).  All M loads of a lane are in flight together.
template <int M>
__device__ __forceinline__ void load_col(const float2* __restrict__ tile, int c, int n_valid,
                                         int lane, float2 (&v)[M])
{
#pragma unroll
    for (int m = 0; m < M; ++m) {
        const int w = lane + 32 * m;
        v[m] = (w < n_valid) ? __ldg(tile + (int64_t)w * kBlockCols + c) : make_float2(0.f, 0.f);
    }
}

// Inverse of the above: lanes k2 < M hold X[k2 + M k1] in u[k1] (destroyed); after the call
// every lane l holds x[l + 32 n1] in v[n1].  tr needs 32 (M + 1) entries.
template <int M>
__device__ __forceinline__ void warp_fft_inv(float2 (&u)[32], const float2* s_twi, float2* tr,
                                             int lane, float2 (&v)[M])
{
    if (lane < M) {
        dft<32, true>(u);
#pragma unroll
        for (int n2 = 1; n2 < 32; ++n2) u[n2] = twiddle<true>(u[n2], s_twi[n2 * M + lane]);
#pragma unroll
        for (int n2 = 0; n2 < 32; ++n2) tr[n2 * (M + 1) + lane] = u[n2];
    }
    __syncwarp();
#pragma unroll
    for (int k2 = 0; k2 < M; ++k2) v[k2] = tr[lane * (M + 1) + k2];
    __syncwarp();
    dft<M, true>(v);
}

}  // namespace wcsim
