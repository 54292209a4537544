// resample_noalloc.cu -- systematic resampling for callers that cannot
// allocate device memory.
//
// mcl_resample keeps its integer CDF in the workspace that mcl_init_map
// allocates.  Some callers have no map and may not allocate at all: a
// real-time control loop that forbids allocation after start-up, code that
// runs while a CUDA stream is being captured into a graph (allocation calls
// are not allowed there), or a particle filter that only wants the
// resampling step.  mcl_resample_noalloc gives them the same kernel with its
// scratch in a fixed array that the library's image places on every device
// that loads it (declared below; it stays allocated until the process exits).
#include <mutex>

#include "internal.cuh"

// Scratch of the allocation-free entry point: the integer CDF of up to
// MCL_RESAMPLE_NOALLOC_MAX_IN weights (512 KB).  In host code this name is a
// host-side stand-in, not a device address; kernels get the device address
// from cudaGetSymbolAddress.  The kernel rewrites every entry it reads, so
// nothing has to be cleared between calls.
static __device__ __align__(256) unsigned long long g_noalloc_cdf[MCL_RESAMPLE_NOALLOC_MAX_IN];

namespace mcl {
namespace {

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned long long* g_cdf_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once
// per device with that device current and cached for the life of the
// process.  A cudaDeviceReset() would invalidate the cached address; callers
// that reset a device must not call this entry point on it afterwards.
int scratch_for_current_device(int* dev_out, unsigned long long** cdf) {
    int dev = -1;
    int rc;
    if ((rc = cuda_check(cudaGetDevice(&dev), "cudaGetDevice"))) return rc;
    if (dev < 0 || dev >= kMaxDevices) return fail(MCL_ERR_UNSUPPORTED, "device ordinal %d", dev);
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_cdf_ptr[dev]) {
        void* a = nullptr;
        if ((rc = cuda_check(cudaGetSymbolAddress(&a, g_noalloc_cdf), "cudaGetSymbolAddress(cdf)")))
            return rc;
        g_cdf_ptr[dev] = (unsigned long long*)a;
    }
    *dev_out = dev;
    *cdf = g_cdf_ptr[dev];
    return MCL_OK;
}

// A caller pointer must be device (or managed) memory of device `dev`: a
// pointer of another device would make the kernel read or write the wrong
// GPU's memory.
int check_on_device(const void* p, int dev, const char* name) {
    cudaPointerAttributes at;
    const cudaError_t e = cudaPointerGetAttributes(&at, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(MCL_ERR_ARG, "mcl_resample_noalloc: %s is not a CUDA pointer", name);
    }
    if ((at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged) || at.device != dev)
        return fail(MCL_ERR_ARG, "mcl_resample_noalloc: %s is not device memory of the current device %d",
                    name, dev);
    return MCL_OK;
}

}  // namespace
}  // namespace mcl

using namespace mcl;

extern "C" int mcl_resample_noalloc(const double* d_w, int N_in, int N_out, double u0,
                                    int32_t* d_idx, void* stream) {
    clear_error();
    if (!d_w || !d_idx) return fail(MCL_ERR_ARG, "mcl_resample_noalloc: NULL argument");
    if (N_in < 1 || N_in > MCL_RESAMPLE_NOALLOC_MAX_IN)
        return fail(MCL_ERR_ARG,
                    "mcl_resample_noalloc: N_in %d outside [1, %d] (the fixed scratch holds %d "
                    "weights; use mcl_resample with a map for more)",
                    N_in, MCL_RESAMPLE_NOALLOC_MAX_IN, MCL_RESAMPLE_NOALLOC_MAX_IN);
    if (N_out < 1 || N_out > 65536)
        return fail(MCL_ERR_ARG, "mcl_resample_noalloc: N_out %d outside [1, 65536]", N_out);
    if (!(u0 >= 0.0 && u0 < 1.0)) return fail(MCL_ERR_ARG, "mcl_resample_noalloc: u0 must be in [0, 1)");
    unsigned long long* cdf = nullptr;
    int dev = -1;
    int rc;
    if ((rc = scratch_for_current_device(&dev, &cdf))) return rc;
    if ((rc = check_on_device(d_w, dev, "d_w")) || (rc = check_on_device(d_idx, dev, "d_idx")))
        return rc;
    // no status word: degenerate weights show as d_idx[k] = -1
    return cuda_check(launch_resample(d_w, N_in, N_out, u0, d_idx, cdf, nullptr, (cudaStream_t)stream),
                      "resample (no-alloc)");
}
