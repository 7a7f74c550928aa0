// k_fast.cu -- instantiations of the hot-path kernels with the compiler's
// default floating-point contraction (fused multiply-add): the FP32
// transport + FP64 chemistry form (GLF and HLL transports) and the all-FP64
// form.
#include "launch.h"
#include "rt_kernels.cuh"

namespace rtl {

// dynamic shared memory of the transport pipeline (above the 48 KB default
// for FP64); set once per kernel and device before its first launch
template <typename R, bool STRICT, int FLUX>
static cudaError_t transport_attr()
{
    static int done_dev = -1;
    int dev = 0;
    cudaGetDevice(&dev);
    if (done_dev == dev) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(rtk::k_transport<R, STRICT, FLUX>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)rtk::transport_smem_bytes<R, FLUX>());
    if (e == cudaSuccess) done_dev = dev;
    return e;
}

// the canonical transport kernel (the FP64 forms, GLF and HLL)
template <typename R, int FLUX>
static cudaError_t transport_generic(const Launch &L, int zc, const rtd::Phys &ph, rtd::Ctl *ctl)
{
    cudaError_t e = transport_attr<R, false, FLUX>();
    if (e != cudaSuccess) return e;
    rtk::k_transport<R, false, FLUX>
        <<<L.grid, dim3(RTD_TX, RTD_TY), rtk::transport_smem_bytes<R, FLUX>(), L.stream>>>(
            L.boxes, L.nboxes, L.nitems, zc, ph, ctl);
    return cudaSuccess;
}

// the FP32 transport with a TX x TY tile: shared-memory attribute set once
// per device, then the launch (TMA: the boxes' tensor maps are set)
template <int TX, int TY, bool TMA>
static cudaError_t pm_attr()
{
    static int done_dev = -1;
    int dev = 0;
    cudaGetDevice(&dev);
    if (done_dev == dev) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(rtk::k_transport_pm<TX, TY, TMA>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)rtk::transport_pm_smem_bytes<TX, TY, TMA>());
    if (e == cudaSuccess) done_dev = dev;
    return e;
}

template <int TX, int TY, bool TMA>
static cudaError_t transport_pm_t(const Launch &L, int zc, const rtd::Phys &ph, rtd::Ctl *ctl)
{
    cudaError_t e = pm_attr<TX, TY, TMA>();
    if (e != cudaSuccess) return e;
    (void)zc;
    rtk::k_transport_pm<TX, TY, TMA><<<L.grid, rtk::transport_pm_threads<TX, TY>(),
                                       rtk::transport_pm_smem_bytes<TX, TY, TMA>(), L.stream>>>(
        L.boxes, L.nboxes, L.nitems, L.lockstep, ph, ctl);
    return cudaSuccess;
}

// groups per block (two photon groups of each tile in one block)
template <int TX, int TY, int NG>
static cudaError_t pmg_attr()
{
    static int done_dev = -1;
    int dev = 0;
    cudaGetDevice(&dev);
    if (done_dev == dev) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(rtk::k_transport_pmg<TX, TY, NG>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)rtk::transport_pmg_smem_bytes<TX, TY, NG>());
    if (e == cudaSuccess) done_dev = dev;
    return e;
}

template <int TX, int TY>
static cudaError_t transport_pm(const Launch &L, int zc, const rtd::Phys &ph, rtd::Ctl *ctl)
{
    if (L.gpb == 2 && !L.tma) {
        cudaError_t e = pmg_attr<TX, TY, 2>();
        if (e != cudaSuccess) return e;
        rtk::k_transport_pmg<TX, TY, 2><<<L.grid, rtk::transport_pm_threads<TX, TY>(),
                                          rtk::transport_pmg_smem_bytes<TX, TY, 2>(), L.stream>>>(
            L.boxes, L.nboxes, L.nitems, L.lockstep, ph, ctl);
        return cudaSuccess;
    }
    if (L.gpb != 1) return cudaErrorInvalidValue;
    return L.tma ? transport_pm_t<TX, TY, true>(L, zc, ph, ctl) : transport_pm_t<TX, TY, false>(L, zc, ph, ctl);
}

template <int TX, int TY>
static int pm_occupancy(bool tma, int gpb);
template <int TX, int TY>
static int hll_occupancy();

// the FP32 HLL transport with a TX x TY tile
template <int TX, int TY>
static cudaError_t hll_attr()
{
    static int done_dev = -1;
    int dev = 0;
    cudaGetDevice(&dev);
    if (done_dev == dev) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(rtk::k_transport_hll<TX, TY>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)rtk::transport_hll_smem_bytes<TX, TY>());
    if (e == cudaSuccess) done_dev = dev;
    return e;
}

template <int TX, int TY>
static cudaError_t transport_hll(const Launch &L, int zc, const rtd::Phys &ph, rtd::Ctl *ctl)
{
    cudaError_t e = hll_attr<TX, TY>();
    if (e != cudaSuccess) return e;
    rtk::k_transport_hll<TX, TY><<<L.grid, rtk::transport_pm_threads<TX, TY>(),
                                   rtk::transport_hll_smem_bytes<TX, TY>(), L.stream>>>(
        L.boxes, L.nboxes, L.nitems, zc, ph, ctl);
    return cudaSuccess;
}

cudaError_t transport_fast(bool fp64, const Launch &L, int zc, const rtd::Phys &ph, rtd::Ctl *ctl)
{
    cudaError_t e = cudaSuccess;
    if (ph.flux == RTD_FLUX_HLL && fp64) {
        e = transport_generic<double, RTD_FLUX_HLL>(L, zc, ph, ctl);
    } else if (ph.flux == RTD_FLUX_HLL) {
        switch (L.variant) {
        case 0: e = transport_hll<kTileX[0], kTileY[0]>(L, zc, ph, ctl); break;
        case 1: e = transport_hll<kTileX[1], kTileY[1]>(L, zc, ph, ctl); break;
        case 2: e = transport_hll<kTileX[2], kTileY[2]>(L, zc, ph, ctl); break;
        default: return cudaErrorInvalidValue;
        }
    } else if (fp64) {
        e = transport_generic<double, RTD_FLUX_GLF>(L, zc, ph, ctl);
    } else {
        switch (L.variant) {
        case 0: e = transport_pm<kTileX[0], kTileY[0]>(L, zc, ph, ctl); break;
        case 1: e = transport_pm<kTileX[1], kTileY[1]>(L, zc, ph, ctl); break;
        case 2: e = transport_pm<kTileX[2], kTileY[2]>(L, zc, ph, ctl); break;
        default: return cudaErrorInvalidValue;
        }
    }
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

// dynamic shared memory of the chemistry kernels (staged rows); the limit
// is raised once per process and device at set-up (chem_occupancy_fast),
// before any launch or capture
template <int G, typename T>
static void chem_attr()
{
    cudaFuncSetAttribute((const void *)rtk::k_chem<G, T, T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)rtk::chem_smem_bytes<G, T, T, false>());
}

template <int G>
static void chem_g(bool fp64, const Launch &L, const rtd::Phys &ph, rtd::Ctl *ctl, const rtd::DiagBuf &db)
{
    if (fp64) {
        auto k = rtk::k_chem<G, double, double, false>;
        k<<<L.grid, RTD_CHEM_BLOCK, rtk::chem_smem_bytes<G, double, double, false>(), L.stream>>>(
            L.boxes, L.nboxes, L.nitems, ph, ctl, db, L.grab);
    } else {
        auto k = rtk::k_chem<G, float, float, false>;
        k<<<L.grid, RTD_CHEM_BLOCK, rtk::chem_smem_bytes<G, float, float, false>(), L.stream>>>(
            L.boxes, L.nboxes, L.nitems, ph, ctl, db, L.grab);
    }
}

cudaError_t cconst_fast(bool fp64, const Launch &L, const rtd::Phys &ph, rtd::CellConst *cc)
{
    const int grid = (int)std::min<int64_t>((L.nitems + 7) / 8, 4096);
    if (fp64)
        rtk::k_cconst<double><<<grid, 256, 0, L.stream>>>(L.boxes, L.nboxes, L.nitems, ph, cc);
    else
        rtk::k_cconst<float><<<grid, 256, 0, L.stream>>>(L.boxes, L.nboxes, L.nitems, ph, cc);
    return cudaGetLastError();
}

cudaError_t chem_fast(bool fp64, int G, const Launch &L, const rtd::Phys &ph, rtd::Ctl *ctl,
                      const rtd::DiagBuf &db)
{
    switch (G) {
    case 1: chem_g<1>(fp64, L, ph, ctl, db); break;
    case 2: chem_g<2>(fp64, L, ph, ctl, db); break;
    case 3: chem_g<3>(fp64, L, ph, ctl, db); break;
    case 4: chem_g<4>(fp64, L, ph, ctl, db); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}



template <int G>
static void chem_fine_g(bool fp64, const Launch &L, const rtd::FineDev *fines, const rtd::Phys &ph,
                        rtd::Ctl *ctl)
{
    if (fp64)
        rtk::k_chem_fine<G, double, double, false><<<L.grid, RTD_CHEM_BLOCK, 0, L.stream>>>(
            L.boxes, fines, L.nboxes, L.nitems, ph, ctl);
    else
        rtk::k_chem_fine<G, float, float, false><<<L.grid, RTD_CHEM_BLOCK, 0, L.stream>>>(
            L.boxes, fines, L.nboxes, L.nitems, ph, ctl);
}

cudaError_t chem_fine_fast(bool fp64, int G, const Launch &L, const rtd::FineDev *fines,
                           const rtd::Phys &ph, rtd::Ctl *ctl)
{
    switch (G) {
    case 1: chem_fine_g<1>(fp64, L, fines, ph, ctl); break;
    case 2: chem_fine_g<2>(fp64, L, fines, ph, ctl); break;
    case 3: chem_fine_g<3>(fp64, L, fines, ph, ctl); break;
    case 4: chem_fine_g<4>(fp64, L, fines, ph, ctl); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

static int occ(const void *f, int threads, size_t smem = 0)
{
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, f, threads, smem) != cudaSuccess) n = 1;
    return n > 0 ? n : 1;
}

template <typename R, int FLUX>
static int generic_occupancy()
{
    transport_attr<R, false, FLUX>();
    return occ((const void *)rtk::k_transport<R, false, FLUX>, RTD_TX * RTD_TY,
               rtk::transport_smem_bytes<R, FLUX>());
}

int transport_occupancy_fast(bool fp64, int variant, int flux, bool tma, int gpb)
{
    if (flux == RTD_FLUX_HLL && fp64) return generic_occupancy<double, RTD_FLUX_HLL>();
    if (flux == RTD_FLUX_HLL) {
        switch (variant) {
        case 1: return hll_occupancy<kTileX[1], kTileY[1]>();
        case 2: return hll_occupancy<kTileX[2], kTileY[2]>();
        default: return hll_occupancy<kTileX[0], kTileY[0]>();
        }
    }
    if (fp64) return generic_occupancy<double, RTD_FLUX_GLF>();
    switch (variant) {
    case 1: return pm_occupancy<kTileX[1], kTileY[1]>(tma, gpb);
    case 2: return pm_occupancy<kTileX[2], kTileY[2]>(tma, gpb);
    default: return pm_occupancy<kTileX[0], kTileY[0]>(tma, gpb);
    }
}

template <int TX, int TY>
static int hll_occupancy()
{
    hll_attr<TX, TY>();
    return occ((const void *)rtk::k_transport_hll<TX, TY>, rtk::transport_pm_threads<TX, TY>(),
               rtk::transport_hll_smem_bytes<TX, TY>());
}

template <int TX, int TY>
static int pm_occupancy(bool tma, int gpb)
{
    if (gpb == 2 && !tma) {
        pmg_attr<TX, TY, 2>();
        return occ((const void *)rtk::k_transport_pmg<TX, TY, 2>, rtk::transport_pm_threads<TX, TY>(),
                   rtk::transport_pmg_smem_bytes<TX, TY, 2>());
    }
    if (tma) {
        pm_attr<TX, TY, true>();
        return occ((const void *)rtk::k_transport_pm<TX, TY, true>, rtk::transport_pm_threads<TX, TY>(),
                   rtk::transport_pm_smem_bytes<TX, TY, true>());
    }
    pm_attr<TX, TY, false>();
    return occ((const void *)rtk::k_transport_pm<TX, TY, false>, rtk::transport_pm_threads<TX, TY>(),
               rtk::transport_pm_smem_bytes<TX, TY, false>());
}

__global__ void k_fill_tune(float4 *U, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        U[i] = make_float4(1.0f, 0.3f, 0.2f, 0.1f);
}

cudaError_t fill_tune_state(void *U, int64_t n, cudaStream_t s)
{
    k_fill_tune<<<1024, 256, 0, s>>>(reinterpret_cast<float4 *>(U), n);
    return cudaGetLastError();
}

int chem_occupancy_fast(bool fp64, int G)
{
#define OCC_G(g)                                                                                \
    (fp64 ? (chem_attr<g, double>(),                                                            \
             occ((const void *)rtk::k_chem<g, double, double, false>, RTD_CHEM_BLOCK,           \
                 rtk::chem_smem_bytes<g, double, double, false>()))                             \
          : (chem_attr<g, float>(),                                                             \
             occ((const void *)rtk::k_chem<g, float, float, false>, RTD_CHEM_BLOCK,             \
                 rtk::chem_smem_bytes<g, float, float, false>())))
    switch (G) {
    case 1: return OCC_G(1);
    case 2: return OCC_G(2);
    case 3: return OCC_G(3);
    default: return OCC_G(4);
    }
#undef OCC_G
}

}  // namespace rtl
