// k_fast.cu -- instantiations of the hot-path kernels with the compiler's
// default floating-point contraction (fused multiply-add): the FP32
// transport + FP64 chemistry form and the all-FP64 form.
#include "launch.h"
#include "rt_kernels.cuh"

namespace rtl {

cudaError_t transport_fast(bool fp64, const Launch &L, int zc, const rtd::Phys &ph, rtd::Ctl *ctl)
{
    dim3 blk(RTD_TX, RTD_TY);
    if (fp64)
        rtk::k_transport<double, false><<<L.grid, blk, 0, L.stream>>>(L.boxes, L.nboxes, L.nitems, zc, ph, ctl);
    else
        rtk::k_transport<float, false><<<L.grid, blk, 0, L.stream>>>(L.boxes, L.nboxes, L.nitems, zc, ph, ctl);
    return cudaGetLastError();
}

template <int G>
static void chem_g(bool fp64, const Launch &L, const rtd::Phys &ph, rtd::Ctl *ctl, double *partials)
{
    if (fp64)
        rtk::k_chem<G, double, double, false><<<L.grid, RTD_CHEM_BLOCK, 0, L.stream>>>(
            L.boxes, L.nboxes, L.nitems, ph, ctl, partials);
    else
        rtk::k_chem<G, float, float, false><<<L.grid, RTD_CHEM_BLOCK, 0, L.stream>>>(
            L.boxes, L.nboxes, L.nitems, ph, ctl, partials);
}

cudaError_t chem_fast(bool fp64, int G, const Launch &L, const rtd::Phys &ph, rtd::Ctl *ctl,
                      double *partials)
{
    switch (G) {
    case 1: chem_g<1>(fp64, L, ph, ctl, partials); break;
    case 2: chem_g<2>(fp64, L, ph, ctl, partials); break;
    case 3: chem_g<3>(fp64, L, ph, ctl, partials); break;
    case 4: chem_g<4>(fp64, L, ph, ctl, partials); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t finalize(const rtd::BoxDev *boxes, int nboxes, const double *partials, rtd::Ctl *ctl,
                     double *lastdiag, cudaStream_t stream)
{
    rtk::k_finalize<<<nboxes, RTD_CHEM_BLOCK, 0, stream>>>(boxes, partials, ctl, lastdiag);
    return cudaGetLastError();
}

static int occ(const void *f, int threads)
{
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, f, threads, 0) != cudaSuccess) n = 1;
    return n > 0 ? n : 1;
}

int transport_occupancy_fast(bool fp64)
{
    return fp64 ? occ((const void *)rtk::k_transport<double, false>, RTD_TX * RTD_TY)
                : occ((const void *)rtk::k_transport<float, false>, RTD_TX * RTD_TY);
}

int chem_occupancy_fast(bool fp64, int G)
{
#define OCC_G(g) \
    (fp64 ? occ((const void *)rtk::k_chem<g, double, double, false>, RTD_CHEM_BLOCK) \
          : occ((const void *)rtk::k_chem<g, float, float, false>, RTD_CHEM_BLOCK))
    switch (G) {
    case 1: return OCC_G(1);
    case 2: return OCC_G(2);
    case 3: return OCC_G(3);
    default: return OCC_G(4);
    }
#undef OCC_G
}

}  // namespace rtl
