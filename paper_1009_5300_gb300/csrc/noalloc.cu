// Allocation-free variant of the Eq. 10 preconditioner with its Krylov dot
// products, for callers that must not allocate device memory.
//
// The regular path keeps the per-CTA partial sums of r^T z and |r|^2 in the
// solve workspace.  This entry point keeps them instead in a fixed,
// file-scope device array that every GPU loading the library holds until the
// process exits, so a call allocates nothing: no cudaMalloc, no cudaFree, no
// allocating library routine.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "../../include/iobm.h"
#include "iobm_internal.cuh"

namespace iobm {
namespace {

// Maximum number of per-CTA partial slots (RHS x CTAs of one launch) = 1 MiB
// of double2 plus 512 KiB of double per device.
constexpr int kNoAllocSlots = 1 << 16;
constexpr int kNoAllocZChunk = 32;
constexpr int kMaxDevices = 64;
constexpr int kMaxGridZ = 65535;

static __device__ __align__(256) double2 g_dot_partials[kNoAllocSlots];
static __device__ __align__(256) double g_nrm_partials[kNoAllocSlots];

struct DeviceScratch {
    double2* dot = nullptr;
    double* nrm = nullptr;
};
DeviceScratch g_scratch[kMaxDevices];
std::mutex g_scratch_mutex;

// Device addresses of the two arrays on the current device (in host code the
// array names are only host-side stand-ins).  Looked up afresh on every call made
// while the stream is not being captured (cheap, and it follows a context that
// was destroyed and re-created, e.g. after cudaDeviceReset); during stream capture
// the address cached by the last such call is used.
cudaError_t scratch_for_current_device(cudaStream_t stream, DeviceScratch& out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing(stream, &cs);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    DeviceScratch& s = g_scratch[dev];
    if (cs == cudaStreamCaptureStatusNone || !s.dot) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_dot_partials);
        if (e != cudaSuccess) return e;
        void* q = nullptr;
        e = cudaGetSymbolAddress(&q, g_nrm_partials);
        if (e != cudaSuccess) return e;
        s.dot = static_cast<double2*>(p);
        s.nrm = static_cast<double*>(q);
    }
    out = s;
    return cudaSuccess;
}

// rho[i] = sum of the dot slots of RHS i, rr[i] = sum of its norm slots (fixed order)
__global__ void k_sum_slots(const double2* dot, const double* nrm, int nslots, int nrhs,
                            double2* rho, double* rr) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nrhs) return;
    double a = 0.0, b = 0.0, c = 0.0;
    for (int j = 0; j < nslots; ++j) {
        const double2 v = dot[(long long)i * nslots + j];
        a += v.x;
        b += v.y;
        c += nrm[(long long)i * nslots + j];
    }
    rho[i] = make_double2(a, b);
    rr[i] = c;
}

}  // namespace
}  // namespace iobm

using namespace iobm;

extern "C" int iobm_precond_dots_noalloc(const iobm_grid* grid, double alpha, const void* r,
                                         void* z, int nrhs, double* rho, double* rr,
                                         void* cuda_stream) {
    if (!grid || !r || !z || !rho || !rr || nrhs < 0 || !(alpha > 0)) return IOBM_E_ARG;
    const iobm_grid& g = *grid;
    if (g.nx < 1 || g.ny < 1 || g.nz < 1) return IOBM_E_ARG;
    if (nrhs == 0) return IOBM_OK;
    // the RHS index is the grid's z dimension (at most 65535), and every RHS needs at
    // least one partial slot
    if (nrhs > kMaxGridZ || nrhs > kNoAllocSlots) return IOBM_E_UNSUPPORTED;
    const int per_rhs = stencil_slots(g.nx, g.ny, g.nz, kNoAllocZChunk, 1);
    if ((long long)per_rhs * nrhs > kNoAllocSlots) return IOBM_E_UNSUPPORTED;
    // z = P r reads neighbours of r that other CTAs may already have overwritten
    // in z, so the two ranges must not overlap
    const unsigned long long bytes =
        (unsigned long long)nrhs * g.nx * g.ny * g.nz * sizeof(double2);
    const unsigned long long rb = reinterpret_cast<unsigned long long>(r);
    const unsigned long long zb = reinterpret_cast<unsigned long long>(z);
    if (rb < zb + bytes && zb < rb + bytes) return IOBM_E_ARG;
    cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
    DeviceScratch s;
    if (scratch_for_current_device(stream, s) != cudaSuccess) return IOBM_E_CUDA;

    StencilArgs<double> a{};
    a.x = static_cast<const double2*>(r);
    a.y = static_cast<double2*>(z);
    a.nx = g.nx;
    a.ny = g.ny;
    a.nz = g.nz;
    a.nf = 1;
    const double c1 = std::exp(-alpha);
    a.cx[1] = a.cy[1] = a.cz[1] = c1;
    a.c0 = 1.0 + 6.0 * c1;   // the stencil kernel applies its taps in difference form
    a.vsign = 0.0;
    a.mask = M_ALL;
    a.dot_mode = 1;
    a.dot_part = s.dot;
    a.nrm_part = s.nrm;
    a.slot_stride = per_rhs;
    a.slot_base = 0;
    a.zchunk = kNoAllocZChunk;
    a.npts = (long long)g.nx * g.ny * g.nz;
    if (launch_stencil<double>(a, nrhs, stream) != cudaSuccess) return IOBM_E_CUDA;
    k_sum_slots<<<(nrhs + 127) / 128, 128, 0, stream>>>(s.dot, s.nrm, per_rhs, nrhs,
                                                         reinterpret_cast<double2*>(rho), rr);
    if (cudaGetLastError() != cudaSuccess) return IOBM_E_CUDA;
    return IOBM_OK;
}
