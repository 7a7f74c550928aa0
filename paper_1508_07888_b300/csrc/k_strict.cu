// k_strict.cu -- instantiations of the FP64 hot-path kernels compiled with
// --fmad=false: no contraction, IEEE division and square root, operations in
// the order the source writes them (RT_PREC_FP64_STRICT).
#define RTK_STRICT_TU 1   // the diagnostics kernel is defined once, in k_fast.cu
#include "launch.h"
#include "rt_kernels.cuh"

namespace rtl {

cudaError_t transport_strict(const Launch &L, int zc, const rtd::Phys &ph, rtd::Ctl *ctl)
{
    dim3 blk(RTD_TX, RTD_TY);
    rtk::k_transport<double, true><<<L.grid, blk, 0, L.stream>>>(L.boxes, L.nboxes, L.nitems, zc, ph, ctl);
    return cudaGetLastError();
}

cudaError_t chem_strict(int G, const Launch &L, const rtd::Phys &ph, rtd::Ctl *ctl, double *partials)
{
#define CHEM_G(g)                                                                          \
    rtk::k_chem<g, double, double, true><<<L.grid, RTD_CHEM_BLOCK, 0, L.stream>>>(          \
        L.boxes, L.nboxes, L.nitems, ph, ctl, partials)
    switch (G) {
    case 1: CHEM_G(1); break;
    case 2: CHEM_G(2); break;
    case 3: CHEM_G(3); break;
    case 4: CHEM_G(4); break;
    default: return cudaErrorInvalidValue;
    }
#undef CHEM_G
    return cudaGetLastError();
}

static int occ(const void *f, int threads)
{
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, f, threads, 0) != cudaSuccess) n = 1;
    return n > 0 ? n : 1;
}

int transport_occupancy_fast(bool fp64);
int chem_occupancy_fast(bool fp64, int G);

int transport_occupancy(bool fp64, bool strict)
{
    if (strict) return occ((const void *)rtk::k_transport<double, true>, RTD_TX * RTD_TY);
    return transport_occupancy_fast(fp64);
}

int chem_occupancy(bool fp64, bool strict, int G)
{
    if (!strict) return chem_occupancy_fast(fp64, G);
    switch (G) {
    case 1: return occ((const void *)rtk::k_chem<1, double, double, true>, RTD_CHEM_BLOCK);
    case 2: return occ((const void *)rtk::k_chem<2, double, double, true>, RTD_CHEM_BLOCK);
    case 3: return occ((const void *)rtk::k_chem<3, double, double, true>, RTD_CHEM_BLOCK);
    default: return occ((const void *)rtk::k_chem<4, double, double, true>, RTD_CHEM_BLOCK);
    }
}

}  // namespace rtl
