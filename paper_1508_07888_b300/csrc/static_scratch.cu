// static_scratch.cu -- rt_transport_static: radiative transport steps that
// allocate no device memory.
//
// Who needs this: code that cannot call cudaMalloc while it runs -- for
// instance a host framework whose caching allocator owns every device byte
// and forbids outside allocations, or a solver embedded in a larger code that
// must not grow its device footprint or synchronise the device mid-run (a
// cudaMalloc/cudaFree can do both).  rt_create allocates its scratch; this
// entry point does not: the post-transport radiation state and the two
// kernel descriptors live in one file-scope __device__ array of
// RT_STATIC_SCRATCH_BYTES bytes that every GPU loading this library holds
// until the process exits.
//
// The array's name is only a host-side stand-in in host code; its device
// address is fetched once per device, with that device current, through
// cudaGetSymbolAddress on the first call made while that device is current.
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <mutex>

#include <cuda_runtime.h>

#include "../../include/rt_m1.h"
#include "launch.h"
#include "rt_device.h"

namespace {

// layout: [0, 256) control block, [256, 512) and [512, 768) descriptors of the
// two ping-pong directions, [768, end) post-transport radiation state
constexpr size_t kCtlOff = 0, kDescOff0 = 256, kDescOff1 = 512, kStateOff = 768;
static_assert(sizeof(rtd::Ctl) <= 256 && sizeof(rtd::BoxDev) <= 256, "descriptor slots");

__device__ __align__(256) unsigned char g_static_scratch[RT_STATIC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
unsigned char *g_dev_addr[kMaxDevices] = {nullptr};
std::mutex g_setup_mutex;

// a failure returns its status and leaves its message for rt_last_error(NULL)
inline int err(int code, const char *msg)
{
    rtl::set_thread_error(msg);
    return code;
}

// device address of the scratch on the current device (set-up on first use)
int scratch_address(unsigned char **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return err(RT_ERR_CUDA, "rt_transport_static: no usable current CUDA device");
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_dev_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return err(RT_ERR_CUDA, "rt_transport_static: cudaGetSymbolAddress of the static "
                                    "scratch failed on the current device");
        }
        g_dev_addr[dev] = static_cast<unsigned char *>(p);
    }
    *out = g_dev_addr[dev];
    return RT_OK;
}

}  // namespace

extern "C" int rt_transport_static(const rt_params *p, const rt_box *box, int nsteps, void *stream)
{
    if (!p || !box) return err(RT_ERR_ARG, "rt_transport_static: NULL params or box");
    if (p->ngroups < 1 || p->ngroups > RT_MAX_GROUPS)
        return err(RT_ERR_ARG, "rt_transport_static: ngroups outside [1, RT_MAX_GROUPS]");
    if (!(p->c_red > 0) || !(p->cfl > 0 && p->cfl <= 1))
        return err(RT_ERR_ARG, "rt_transport_static: need c_red > 0 and cfl in (0, 1]");
    if (p->precision < RT_PREC_SPLIT || p->precision > RT_PREC_FP64_STRICT)
        return err(RT_ERR_ARG, "rt_transport_static: unknown precision");
    if (p->flux != RT_FLUX_GLF) return err(RT_ERR_ARG, "rt_transport_static: GLF flux only");
    if (p->cosmo) return err(RT_ERR_ARG, "rt_transport_static: no supercomoving units");
    for (int f = 0; f < 6; f++)
        if (p->bc[f] < RT_BC_PERIODIC || p->bc[f] > RT_BC_REFLECTIVE)
            return err(RT_ERR_ARG, "rt_transport_static: unknown boundary condition");
    for (int d = 0; d < 3; d++)
        if ((p->bc[2 * d] == RT_BC_PERIODIC) != (p->bc[2 * d + 1] == RT_BC_PERIODIC))
            return err(RT_ERR_ARG, "rt_transport_static: periodic on one face of an axis only");
    if (box->nx < 1 || box->ny < 1 || box->nz < 1 || !(box->dx > 0))
        return err(RT_ERR_ARG, "rt_transport_static: box sizes and dx must be positive");
    if (!box->U || ((uintptr_t)box->U % 16))
        return err(RT_ERR_ARG, "rt_transport_static: U must be a 16-byte aligned device pointer");
    if (nsteps < 0) return err(RT_ERR_ARG, "rt_transport_static: nsteps must be >= 0");
    const bool fp64 = p->precision != RT_PREC_SPLIT;
    const bool strict = p->precision == RT_PREC_FP64_STRICT;
    // capacity in cells, then the box against it one factor at a time, so that
    // no product of the sizes can overflow before it is compared
    const uint64_t cell_bytes = (uint64_t)p->ngroups * 4 * (fp64 ? 8 : 4);
    const uint64_t cap = (RT_STATIC_SCRATCH_BYTES - kStateOff) / cell_bytes;
    const uint64_t nxy_cap = cap / (uint64_t)box->nx;
    if ((uint64_t)box->ny > nxy_cap || (uint64_t)box->nz > nxy_cap / (uint64_t)box->ny)
        return err(RT_ERR_TOO_LARGE, "rt_transport_static: the box's radiation state does not fit the "
                               "static scratch (G*nx*ny*nz*4*element size must be at most "
                               "RT_STATIC_SCRATCH_BYTES - 768 bytes)");
    const int64_t ncell = (int64_t)box->nx * box->ny * box->nz;
    const size_t need = (size_t)cell_bytes * (size_t)ncell;
    if (nsteps == 0) return RT_OK;

    unsigned char *base = nullptr;
    int rc = scratch_address(&base);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;

    // the two directions: U -> scratch and scratch -> U
    rtd::BoxDev D[2];
    std::memset(D, 0, sizeof D);
    for (int k = 0; k < 2; k++) {
        rtd::BoxDev &B = D[k];
        B.nx = box->nx; B.ny = box->ny; B.nz = box->nz;
        B.ncell = ncell;
        B.dx = box->dx;
        B.nunit = box->nunit;
        B.inv_nunit = 1.0 / box->nunit;
        B.dt = p->cfl * box->dx / (3.0 * p->c_red);
        B.lam = p->c_red * B.dt / box->dx;
        rtl::transport_layout(B, p->ngroups);
        B.titem0 = 0;
        B.U = k == 0 ? box->U : (void *)(base + kStateOff);
        B.Us = k == 0 ? (void *)(base + kStateOff) : box->U;
    }
    rtd::Ctl ctl;
    std::memset(&ctl, 0, sizeof ctl);
    ctl.step = -1;
    ctl.nboxes = 1;
    rtd::Phys ph;
    std::memset(&ph, 0, sizeof ph);
    ph.G = p->ngroups;
    ph.c = p->c_red;
    for (int f = 0; f < 6; f++) ph.bc[f] = p->bc[f];

    // the scratch keeps the previous call's contents: rewrite the control
    // block and both descriptors before every call
    if (cudaMemcpyAsync(base + kCtlOff, &ctl, sizeof ctl, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(base + kDescOff0, &D[0], sizeof D[0], cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(base + kDescOff1, &D[1], sizeof D[1], cudaMemcpyHostToDevice, s) != cudaSuccess)
        return err(RT_ERR_CUDA, "rt_transport_static: copy of the descriptors failed");

    int dev = 0, nsm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int grid = (int)std::min<int64_t>(D[0].ntitems,
                                            (int64_t)rtl::transport_occupancy(fp64, strict) * nsm);
    rtd::Ctl *dctl = reinterpret_cast<rtd::Ctl *>(base + kCtlOff);
    for (int k = 0; k < nsteps; k++) {
        const rtd::BoxDev *dd = reinterpret_cast<const rtd::BoxDev *>(
            base + ((k & 1) ? kDescOff1 : kDescOff0));
        rtl::Launch L{dd, 1, D[0].ntitems, grid, s};
        cudaError_t e = strict ? rtl::transport_strict(L, 32, ph, dctl)
                               : rtl::transport_fast(fp64, L, 32, ph, dctl);
        if (e != cudaSuccess) {
            // drain what was queued before the failure, so that no step of this
            // call is still running on box->U when the caller gets the status
            cudaStreamSynchronize(s);
            return err(RT_ERR_CUDA, "rt_transport_static: kernel launch failed");
        }
    }
    if (nsteps & 1) {
        if (cudaMemcpyAsync(box->U, base + kStateOff, need, cudaMemcpyDeviceToDevice, s) != cudaSuccess) {
            cudaStreamSynchronize(s);
            return err(RT_ERR_CUDA, "rt_transport_static: copy of the result failed");
        }
    }
    if (cudaStreamSynchronize(s) != cudaSuccess)
        return err(RT_ERR_CUDA, "rt_transport_static: stream synchronisation failed");
    rtl::set_thread_error("");
    return RT_OK;
}
