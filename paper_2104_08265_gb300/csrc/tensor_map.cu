// Tensor maps over blocked spectra, for TMA box copies between shared memory and the
// [n_ev][n_j][nkb][n_w][4] complex layout of the time-axis spectra.
//
// The map views one blocked array as a 5-D FP32 tensor (innermost first): the 8 floats of
// one wire's 4-frequency block (32 bytes), the wire, the frequency block, the impact (or
// the single row set, n_j = 1) and the event.  A box of {8, 1, bk, 1, 1} is one row's half
// spectrum for bk consecutive frequency blocks: 4 bk consecutive complex values in shared
// memory, natural frequency order.  The encoder (cuTensorMapEncodeTiled) is taken from the
// driver once through the runtime's entry-point query, so the library links no driver
// library of its own.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>
#include <stdint.h>

#include <mutex>

#include "wcsim_internal.cuh"

namespace wcsim {
namespace {

PFN_cuTensorMapEncodeTiled_v12000 encoder()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        else
            cudaGetLastError();
    });
    return fn;
}

}  // namespace

int blocked_box_kb(int nkb)
{
    if (nkb <= kMapBoxKb) return nkb;
    const int nbox = (nkb + kMapBoxKb - 1) / kMapBoxKb;
    return (((nkb + nbox - 1) / nbox) + 3) & ~3;    // balanced boxes, 128-byte multiples
}

bool blocked_spectra_map(const float2* base, int n_w, int nkb, int n_j, int n_ev,
                         int64_t ev_stride, ::CUtensorMap_st* out)
{
    if (!base || n_w <= 0 || nkb <= 0 || n_j <= 0 || n_ev <= 0) return false;
    if ((reinterpret_cast<uintptr_t>(base) & 15) != 0) return false;
    PFN_cuTensorMapEncodeTiled_v12000 fn = encoder();
    if (!fn) return false;
    const uint64_t blk = (uint64_t)kBlockCols * sizeof(float2);        // 32 bytes
    const uint64_t plane = (uint64_t)n_j * nkb * n_w * blk;
    const uint64_t evs = n_ev > 1 ? (uint64_t)ev_stride * sizeof(float2) : plane;
    if (evs % 16 != 0) return false;
    cuuint64_t dims[5] = {2 * kBlockCols, (cuuint64_t)n_w, (cuuint64_t)nkb, (cuuint64_t)n_j,
                          (cuuint64_t)n_ev};
    cuuint64_t strides[4] = {blk, (cuuint64_t)n_w * blk, (cuuint64_t)nkb * n_w * blk, evs};
    cuuint32_t box[5] = {2 * kBlockCols, 1, (cuuint32_t)blocked_box_kb(nkb), 1, 1};
    cuuint32_t estr[5] = {1, 1, 1, 1, 1};
    const CUresult r = fn(out, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 5,
                          const_cast<float2*>(base), dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                          CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

}  // namespace wcsim
