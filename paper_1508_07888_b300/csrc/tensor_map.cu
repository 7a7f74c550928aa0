// tensor_map.cu -- TMA tensor maps of a box's FP32 radiation state for the
// FP32 GLF transport (rt_kernels.cuh, k_transport_pm with TMA).
//
// U is [G][nz][ny][nx][4] floats: the maps see it as a 4-D tensor of dims
// (4 components, nx, ny, nz G), strides 16 B, 16 nx B, 16 nx ny B, so a copy
// at coordinates (0, x, y, z + nz g) takes whole cells and its innermost
// coordinate is always 0 (16-byte aligned).  Three boxes per tile shape:
// the tile with its halo, (TX + 2) x (TY + 2) cells of one plane; a halo
// column, 1 x TY cells; a halo row, TX x 1 cells.  Out-of-range cells of a
// box read as zeros.  The encoder is the driver's cuTensorMapEncodeTiled,
// reached through the runtime's entry-point query (no link against the
// driver library).
#include <cstdint>
#include <mutex>

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include "launch.h"

namespace {

static_assert(sizeof(CUtensorMap) == 128, "three maps of 128 bytes per box");

PFN_cuTensorMapEncodeTiled_v12000 encoder()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        else
            cudaGetLastError();
    });
    return fn;
}

bool encode(CUtensorMap *m, void *base, const rtd::BoxDev &B, int G, unsigned bx, unsigned by)
{
    PFN_cuTensorMapEncodeTiled_v12000 fn = encoder();
    if (!fn) return false;
    const cuuint64_t dims[4] = {4, (cuuint64_t)B.nx, (cuuint64_t)B.ny, (cuuint64_t)B.nz * (cuuint64_t)G};
    const cuuint64_t strides[3] = {16, 16ull * (cuuint64_t)B.nx, 16ull * (cuuint64_t)B.nx * (cuuint64_t)B.ny};
    const cuuint32_t box[4] = {4, bx, by, 1};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, base, dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

bool rtl::transport_tensor_maps(const rtd::BoxDev &B, int ngroups, int variant, void *out)
{
    if (!B.U || (reinterpret_cast<uintptr_t>(B.U) & 15u) || (reinterpret_cast<uintptr_t>(out) & 63u))
        return false;
    if (variant < 0 || variant >= kTileVariants) return false;
    const unsigned tx = (unsigned)kTileX[variant], ty = (unsigned)kTileY[variant];
    CUtensorMap *m = static_cast<CUtensorMap *>(out);
    return encode(&m[0], B.U, B, ngroups, tx + 2, ty + 2) && encode(&m[1], B.U, B, ngroups, 1, ty) &&
           encode(&m[2], B.U, B, ngroups, tx, 1);
}
