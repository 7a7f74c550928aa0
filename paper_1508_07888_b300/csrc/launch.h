// launch.h -- host-side launchers of the kernels in rt_kernels.cuh
// (internal to librt_m1).  "fast" launchers live in k_fast.cu (default
// contraction), "strict" ones in k_strict.cu (compiled with --fmad=false).
#pragma once

#include <cstdint>

#include <cuda_runtime.h>

#include "rt_device.h"

namespace rtl {

// element types of a precision form: 0 = SPLIT (float U, float n0),
// 1 = FP64 (double U, double n0)
struct Launch {
    const rtd::BoxDev *boxes;
    int nboxes;
    int64_t nitems;
    int grid;
    cudaStream_t stream;
};

cudaError_t transport_fast(bool fp64, const Launch &L, int zc, const rtd::Phys &ph, rtd::Ctl *ctl);
cudaError_t transport_strict(const Launch &L, int zc, const rtd::Phys &ph, rtd::Ctl *ctl);
cudaError_t chem_fast(bool fp64, int G, const Launch &L, const rtd::Phys &ph, rtd::Ctl *ctl,
                      const rtd::DiagBuf &db);
cudaError_t chem_strict(int G, const Launch &L, const rtd::Phys &ph, rtd::Ctl *ctl,
                        const rtd::DiagBuf &db);

// transport tiling of a box: x/y tiles and the number of plane units
// (ngroups x tiles_x x tiles_y x nz) the transport kernel spreads over its grid
inline void transport_layout(rtd::BoxDev &B, int ngroups)
{
    B.tiles_x = (B.nx + RTD_TX - 1) / RTD_TX;
    B.tiles_y = (B.ny + RTD_TY - 1) / RTD_TY;
    B.zchunks = 1;
    B.ntitems = (int64_t)ngroups * B.tiles_x * B.tiles_y * B.nz;
}

// rate tables of the chemistry kernel (rate_table.cu); false = unusable
bool build_rate_table(bool ots, double *out);
constexpr size_t rate_table_doubles() { return (size_t)RTD_TAB_NF * RTD_TAB_NINT * RTD_TAB_NC; }

// reverse-mode kernels of one FP64 step on a periodic single box (adjoint.cu)
cudaError_t chem_adj(int G, const rtd::BoxDev *boxes, const rtd::Phys &ph, const double *Us,
                     const double *xk, const double *Tk, double *lamU, double *lamx, double *lamT,
                     double gx, double *dn0, double *dS, unsigned *err, int64_t ncell,
                     cudaStream_t s);
cudaError_t transport_adj(int G, const rtd::BoxDev *boxes, const double *U, const double *lamS,
                          double *lamU, int64_t ncell, cudaStream_t s);

// resident blocks per SM of each kernel (for persistent grid sizing)
int transport_occupancy(bool fp64, bool strict);
int chem_occupancy(bool fp64, bool strict, int G);

}  // namespace rtl
