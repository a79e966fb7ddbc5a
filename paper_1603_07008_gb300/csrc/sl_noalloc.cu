// sl_noalloc.cu -- the mass reduction for callers that cannot allocate device
// memory.
//
// sl_mass needs a small scratch buffer for its per-block partial sums, which
// sl_create allocates with cudaMalloc.  Some callers cannot let a library
// allocate: a host application that owns all device memory through its own
// pool or arena and forbids other cudaMalloc calls, or a latency-sensitive
// loop where cudaMalloc (which may synchronise the device) must not run.
// sl_mass_noalloc serves them: its scratch is a fixed file-scope __device__
// array, so it allocates nothing; the caller passes the input plane and the
// output location.
#include <mutex>

#include "../../include/sl.h"
#include "sl_internal.cuh"

namespace {

// Maximum number of per-block partial sums (mass_blocks never asks for more
// than 1024), 8 KB.  Every GPU that loads the library holds this array until
// the process exits.
constexpr int kNoallocPartials = 1024;
__device__ __align__(256) double g_mass_scratch[kNoallocPartials];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_scratch_addr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device, looked up once
// per device.  In host code the array's name is only a host-side stand-in,
// never a device address, so the address must come from the runtime.
cudaError_t scratch_for_current_device(double** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_mass_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = static_cast<double*>(p);
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" sl_status sl_mass_noalloc(const double* d_mean, int64_t cells, double cell_volume,
                                     double* d_out, void* cuda_stream)
{
    // Sizes beyond the maximum: the reduction indexes cells with 31 bits and
    // keeps at most kNoallocPartials partial sums.
    if (!d_mean || !d_out) return SL_EINVAL;
    if (cells < 1 || cells > int64_t(0x7fffffff)) return SL_EINVAL;
    if (cell_volume != cell_volume) return SL_ENAN;
    const int nblk = sl::mass_blocks(uint32_t(cells));
    if (nblk > kNoallocPartials) return SL_EINVAL;
    double* scratch = nullptr;
    cudaError_t e = scratch_for_current_device(&scratch);
    if (e != cudaSuccess) return SL_ECUDA;
    // Every partial slot in use is overwritten by the first kernel before the
    // second reads it, so nothing has to be cleared between calls.
    e = sl::launch_mass(d_mean, uint32_t(cells), scratch, nblk, cell_volume, d_out,
                        static_cast<cudaStream_t>(cuda_stream));
    return e == cudaSuccess ? SL_OK : SL_ECUDA;
}
