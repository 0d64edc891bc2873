// Host side of the TMA staging: tensor-map descriptors of a workspace's
// basis slab.  The encoder is taken from the driver through the runtime's
// entry-point query, so the library does not link the driver library.
#pragma once

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <mutex>

#include "skr_common.h"

namespace skr {

// Describe the basis slab (nslots * NCOLS columns of ld elements of esz
// bytes, column-contiguous) as a 2D tensor: dim 0 = rows (ld), dim 1 =
// columns, with boxes of {RING_SEG_BYTES / esz rows x (16 >> i) columns} in
// maps[i], i < NBOX.  Boxes reaching past row ld read zeros.  Returns
// cudaErrorInvalidValue when the driver rejects a descriptor.
inline cudaError_t encode_basis_maps(void *basis, long long ld, int nslots, int esz, CUtensorMap *maps) {
    static std::once_flag once;
    static PFN_cuTensorMapEncodeTiled_v12000 enc = nullptr;
    static cudaError_t qerr = cudaSuccess;
    std::call_once(once, [] {
        cudaDriverEntryPointQueryResult qr;
        void *fn = nullptr;
        qerr = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &qr);
        if (qerr == cudaSuccess && qr != cudaDriverEntryPointSuccess) qerr = cudaErrorSymbolNotFound;
        enc = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    });
    if (qerr != cudaSuccess || enc == nullptr) return qerr != cudaSuccess ? qerr : cudaErrorSymbolNotFound;
    const CUtensorMapDataType dt = (esz == 8) ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    cuuint64_t dims[2] = {(cuuint64_t)ld, (cuuint64_t)nslots * (cuuint64_t)NCOLS};
    cuuint64_t strides[1] = {(cuuint64_t)ld * (cuuint64_t)esz};
    cuuint32_t estr[2] = {1, 1};
    for (int i = 0; i < NBOX; i++) {
        cuuint32_t box[2] = {(cuuint32_t)(RING_SEG_BYTES / esz), (cuuint32_t)(16 >> i)};
        const CUresult r = enc(maps + i, dt, 2, basis, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                               CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
    }
    return cudaSuccess;
}

}  // namespace skr
