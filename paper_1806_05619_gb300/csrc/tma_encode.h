// Host side of the TMA-fed kernels: 3D tiled tensor maps over the sample
// pools (FP32 arrays of per-sample blocks), encoded through the driver entry
// point looked up once.
#pragma once

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "fmg_device.cuh"

namespace mlqmc_tmap {

inline PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

// FP32 array of per-sample blocks: x extent w (row pitch `pitch` floats), h
// rows, B samples; boxes of bw x bh x 1, zeros outside the extent.
inline bool encode_3d(CUtensorMap* map, const mlqmc_dev::ArrDesc& a, uint64_t w, uint64_t pitch, uint64_t h,
                      uint64_t B, uint32_t bw, uint32_t bh)
{
    PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
    if (!fn || !a.base) return false;
    const cuuint64_t dims[3] = {w, h, B};
    const cuuint64_t strides[2] = {pitch * sizeof(float), static_cast<cuuint64_t>(a.stride)};
    const cuuint32_t box[3] = {bw, bh, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, a.base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
              CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace mlqmc_tmap
