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
    int variant = 0;                 // tile shape of the FP32 transport (kTileX/kTileY)
    bool tma = false;                // FP32 GLF transport: every box has its tensor maps
    int lockstep = 0;                // FP32 GLF transport: tile columns of the lockstep-rows
                                     // order (every box has that many; grid a multiple), 0 = off
    int grab = 1;                    // chemistry: work items a warp takes per draw
    int gpb = 1;                     // FP32 GLF transport: photon groups per block (1 or 2)
};

// the three TMA tensor maps of a box's FP32 radiation state U for tile shape
// `variant` (the tile with its halo, a halo column, a halo row), written to
// out (3 x 128 bytes, host memory); false when the map cannot be encoded
// (the transport then copies per thread)
bool transport_tensor_maps(const rtd::BoxDev &B, int ngroups, int variant, void *out);

// tile shapes (columns x rows, one thread per column) of the FP32 transport
// kernel; the FP64 kernels always use variant 0 (RTD_TX x RTD_TY)
constexpr int kTileVariants = 3;
constexpr int kTileX[kTileVariants] = {RTD_TX, 16, 64};
constexpr int kTileY[kTileVariants] = {RTD_TY, 16, 4};

cudaError_t transport_fast(bool fp64, const Launch &L, int zc, const rtd::Phys &ph, rtd::Ctl *ctl);
cudaError_t transport_strict(const Launch &L, int zc, const rtd::Phys &ph, rtd::Ctl *ctl);
cudaError_t chem_fast(bool fp64, int G, const Launch &L, const rtd::Phys &ph, rtd::Ctl *ctl,
                      const rtd::DiagBuf &db);
cudaError_t chem_strict(int G, const Launch &L, const rtd::Phys &ph, rtd::Ctl *ctl,
                        const rtd::DiagBuf &db);
// CRTA fine level: L.nitems work items of 32 refined cells over fines[nboxes]
cudaError_t chem_fine_fast(bool fp64, int G, const Launch &L, const rtd::FineDev *fines,
                           const rtd::Phys &ph, rtd::Ctl *ctl);
cudaError_t chem_fine_strict(int G, const Launch &L, const rtd::FineDev *fines, const rtd::Phys &ph,
                             rtd::Ctl *ctl);

// transport tiling of a box: x/y tiles, the z-chunk length of the unit order
// (zlen <= 0 or >= nz: whole columns; only the FP32 kernels take chunks) and
// the number of plane units (ngroups x tiles_x x tiles_y x nz) the transport
// kernel spreads over its grid
inline void transport_layout(rtd::BoxDev &B, int ngroups, int variant = 0, int zlen = 0, int gpb = 1)
{
    const int tx = kTileX[variant], ty = kTileY[variant];
    B.tiles_x = (B.nx + tx - 1) / tx;
    B.tiles_y = (B.ny + ty - 1) / ty;
    B.zlen = zlen <= 0 || zlen >= B.nz ? B.nz : zlen;
    const int gblocks = (ngroups + gpb - 1) / gpb;  // units count blocks of gpb groups
    B.ntitems = (int64_t)gblocks * B.tiles_x * B.tiles_y * B.nz;
}

// a realizable radiation state (N = 1, F = (0.3, 0.2, 0.1)) in n cells of
// FP32 U, the input of the launch-shape tuner
cudaError_t fill_tune_state(void *U, int64_t n, cudaStream_t s);

// rate tables of the chemistry kernel (rate_table.cu); false = unusable
bool build_rate_table(bool ots, rtd::RateCoef *out);
// 2^(j/64), j = 0..63, as pairs hi + lo of doubles (the fast forms' exp)
void build_exp2_table(double2 *out);
constexpr size_t rate_table_entries() { return (size_t)RTD_TAB_NF * RTD_TAB_NINT; }

// reverse-mode kernels of one FP64 step on a periodic single box (adjoint.cu)
cudaError_t chem_adj(int G, const rtd::BoxDev *boxes, const rtd::Phys &ph, const double *Us,
                     const double *xk, const double *Tk, double *lamU, double *lamx, double *lamT,
                     double gx, double *dn0, double *dS, unsigned *err, int64_t ncell,
                     cudaStream_t s);
cudaError_t transport_adj(int G, const rtd::BoxDev *boxes, const double *U, const double *lamS,
                          double *lamU, int64_t ncell, cudaStream_t s);

// message that rt_last_error(NULL) returns on the calling thread (rt_api.cu);
// entry points without a handle record their failures here
void set_thread_error(const char *msg);

// resident blocks per SM of each kernel (for persistent grid sizing)
// blocks per SM of the transport kernel a launch runs (tma: the FP32 GLF
// kernel's TMA form)
int transport_occupancy(bool fp64, bool strict, int variant = 0, int flux = RTD_FLUX_GLF, bool tma = false,
                        int gpb = 1);
int chem_occupancy(bool fp64, bool strict, int G);
// the fast forms' per-cell chemistry constants from n0 (before the steps of a call)
cudaError_t cconst_fast(bool fp64, const Launch &L, const rtd::Phys &ph, rtd::CellConst *cc);

}  // namespace rtl
