// k_strict.cu -- instantiations of the FP64 hot-path kernels compiled with
// --fmad=false: no contraction, IEEE division and square root, operations in
// the order the source writes them (RT_PREC_FP64_STRICT).
#define RTK_SKIP_SINGLE_KERNELS 1   // the FP32-only kernels are defined once, in k_fast.cu
#include "launch.h"
#include "rt_kernels.cuh"

namespace rtl {

template <int FLUX>
static cudaError_t transport_attr_strict()
{
    static int done_dev = -1;
    int dev = 0;
    cudaGetDevice(&dev);
    if (done_dev == dev) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(rtk::k_transport<double, true, FLUX>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)rtk::transport_smem_bytes<double, FLUX>());
    if (e == cudaSuccess) done_dev = dev;
    return e;
}

template <int FLUX>
static cudaError_t transport_strict_f(const Launch &L, int zc, const rtd::Phys &ph, rtd::Ctl *ctl)
{
    cudaError_t e = transport_attr_strict<FLUX>();
    if (e != cudaSuccess) return e;
    rtk::k_transport<double, true, FLUX>
        <<<L.grid, dim3(RTD_TX, RTD_TY), rtk::transport_smem_bytes<double, FLUX>(), L.stream>>>(
            L.boxes, L.nboxes, L.nitems, zc, ph, ctl);
    return cudaGetLastError();
}

cudaError_t transport_strict(const Launch &L, int zc, const rtd::Phys &ph, rtd::Ctl *ctl)
{
    return ph.flux == RTD_FLUX_HLL ? transport_strict_f<RTD_FLUX_HLL>(L, zc, ph, ctl)
                                   : transport_strict_f<RTD_FLUX_GLF>(L, zc, ph, ctl);
}

cudaError_t chem_strict(int G, const Launch &L, const rtd::Phys &ph, rtd::Ctl *ctl, const rtd::DiagBuf &db)
{
#define CHEM_G(g)                                                                                \
    rtk::k_chem<g, double, double, true><<<L.grid, RTD_CHEM_BLOCK, 0, L.stream>>>(               \
        L.boxes, L.nboxes, L.nitems, ph, ctl, db, L.grab)
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

cudaError_t chem_fine_strict(int G, const Launch &L, const rtd::FineDev *fines, const rtd::Phys &ph,
                             rtd::Ctl *ctl)
{
#define FINE_G(g)                                                                                \
    rtk::k_chem_fine<g, double, double, true><<<L.grid, RTD_CHEM_BLOCK, 0, L.stream>>>(          \
        L.boxes, fines, L.nboxes, L.nitems, ph, ctl)
    switch (G) {
    case 1: FINE_G(1); break;
    case 2: FINE_G(2); break;
    case 3: FINE_G(3); break;
    case 4: FINE_G(4); break;
    default: return cudaErrorInvalidValue;
    }
#undef FINE_G
    return cudaGetLastError();
}

static int occ(const void *f, int threads, size_t smem = 0)
{
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, f, threads, smem) != cudaSuccess) n = 1;
    return n > 0 ? n : 1;
}

int transport_occupancy_fast(bool fp64, int variant, int flux, bool tma, int gpb);
int chem_occupancy_fast(bool fp64, int G);

int transport_occupancy(bool fp64, bool strict, int variant, int flux, bool tma, int gpb)
{
    if (strict) {
        if (flux == RTD_FLUX_HLL) {
            transport_attr_strict<RTD_FLUX_HLL>();
            return occ((const void *)rtk::k_transport<double, true, RTD_FLUX_HLL>, RTD_TX * RTD_TY,
                       rtk::transport_smem_bytes<double, RTD_FLUX_HLL>());
        }
        transport_attr_strict<RTD_FLUX_GLF>();
        return occ((const void *)rtk::k_transport<double, true, RTD_FLUX_GLF>, RTD_TX * RTD_TY,
                   rtk::transport_smem_bytes<double, RTD_FLUX_GLF>());
    }
    return transport_occupancy_fast(fp64, variant, flux, tma, gpb);
}

int chem_occupancy(bool fp64, bool strict, int G)
{
    if (!strict) return chem_occupancy_fast(fp64, G);
#define OCC_S(g) occ((const void *)rtk::k_chem<g, double, double, true>, RTD_CHEM_BLOCK, 0)
    switch (G) {
    case 1: return OCC_S(1);
    case 2: return OCC_S(2);
    case 3: return OCC_S(3);
    default: return OCC_S(4);
    }
#undef OCC_S
}

}  // namespace rtl
