// tma.cu -- host side of the tensor-map helpers (internal).
#include <atomic>

#include <cudaTypedefs.h>

#include "tma.h"

namespace stokes {

namespace {
std::atomic<PFN_cuTensorMapEncodeTiled_v12000> g_encode{nullptr};

cudaError_t encoder(PFN_cuTensorMapEncodeTiled_v12000 *out)
{
    PFN_cuTensorMapEncodeTiled_v12000 f = g_encode.load();
    if (!f) {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        const cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                               cudaEnableDefault, &q);
        if (e != cudaSuccess) return e;
        if (q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
        f = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
        g_encode.store(f);
    }
    *out = f;
    return cudaSuccess;
}
} // namespace

cudaError_t make_tmap_2d(CUtensorMap *map, const void *base, int elem_bytes, int width, int height,
                         long pitch_bytes, int box_w, int box_h)
{
    PFN_cuTensorMapEncodeTiled_v12000 enc = nullptr;
    const cudaError_t e = encoder(&enc);
    if (e != cudaSuccess) return e;
    const cuuint64_t dims[2] = {(cuuint64_t)width, (cuuint64_t)height};
    const cuuint64_t strides[1] = {(cuuint64_t)pitch_bytes};
    const cuuint32_t box[2] = {(cuuint32_t)box_w, (cuuint32_t)box_h};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r =
        enc(map, elem_bytes == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
            const_cast<void *>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

} // namespace stokes
