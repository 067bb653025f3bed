// tma_host.cpp -- TMA tensor-map encoding through the driver entry point (no libcuda link).
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include "kernels.h"

namespace mmfd {

static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

int encode_field_map(CUtensorMap* m, void* field_base, int st, const Geom& g, int boxw, int boxh, int boxd, bool promote_l2) {
    auto fn = encode_fn();
    if (!fn) return -1;
    const CUtensorMapDataType dt = st == ST_F64   ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64
                                   : st == ST_F32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                                  : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    const cuuint64_t es = (cuuint64_t)g.es;
    const CUtensorMapL2promotion promo = promote_l2 ? CU_TENSOR_MAP_L2_PROMOTION_L2_256B : CU_TENSOR_MAP_L2_PROMOTION_NONE;
    if (g.dim == 2) {
        cuuint64_t dims[2] = {(cuuint64_t)g.py, (cuuint64_t)(g.ny + 2)};
        cuuint64_t strides[1] = {(cuuint64_t)g.py * es};
        cuuint32_t box[2] = {(cuuint32_t)boxw, (cuuint32_t)boxh};
        cuuint32_t estr[2] = {1, 1};
        CUresult r = fn(m, dt, 2, field_base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_NONE, promo,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        return r == CUDA_SUCCESS ? 0 : (int)r;
    }
    cuuint64_t dims[3] = {(cuuint64_t)g.py, (cuuint64_t)(g.ny + 2), (cuuint64_t)(g.nz + 2 * g.gz)};
    cuuint64_t strides[2] = {(cuuint64_t)g.py * es, (cuuint64_t)g.pz * es};
    cuuint32_t box[3] = {(cuuint32_t)boxw, (cuuint32_t)boxh, (cuuint32_t)boxd};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = fn(m, dt, 3, field_base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_NONE, promo, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? 0 : (int)r;
}

}  // namespace mmfd
