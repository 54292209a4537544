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
// MCL_RESAMPLE_NOALLOC_MAX_IN weights (512 KB) and a status word.  In host
// code these names are host-side stand-ins, not device addresses; kernels get
// the device address from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned long long g_noalloc_cdf[MCL_RESAMPLE_NOALLOC_MAX_IN];
static __device__ __align__(256) mcl::Status g_noalloc_status;

namespace mcl {
namespace {

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned long long* g_cdf_ptr[kMaxDevices] = {};
Status* g_status_ptr[kMaxDevices] = {};

// Device addresses of the scratch arrays on the current device (looked up
// once per device, with that device current).
int scratch_for_current_device(unsigned long long** cdf, Status** status) {
    int dev = -1;
    int rc;
    if ((rc = cuda_check(cudaGetDevice(&dev), "cudaGetDevice"))) return rc;
    if (dev < 0 || dev >= kMaxDevices) return fail(MCL_ERR_UNSUPPORTED, "device ordinal %d", dev);
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_cdf_ptr[dev]) {
        void* a = nullptr;
        void* b = nullptr;
        if ((rc = cuda_check(cudaGetSymbolAddress(&a, g_noalloc_cdf), "cudaGetSymbolAddress(cdf)")))
            return rc;
        if ((rc = cuda_check(cudaGetSymbolAddress(&b, g_noalloc_status),
                             "cudaGetSymbolAddress(status)")))
            return rc;
        g_status_ptr[dev] = (Status*)b;
        g_cdf_ptr[dev] = (unsigned long long*)a;
    }
    *cdf = g_cdf_ptr[dev];
    *status = g_status_ptr[dev];
    return MCL_OK;
}

}  // namespace
}  // namespace mcl

using namespace mcl;

extern "C" int mcl_resample_noalloc(const double* d_w, int N_in, int N_out, double u0,
                                    int32_t* d_idx, void* stream) {
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
    Status* status = nullptr;
    int rc;
    if ((rc = scratch_for_current_device(&cdf, &status))) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    // the status word must start at zero; the CDF is fully rewritten
    if ((rc = cuda_check(cudaMemsetAsync(status, 0, sizeof(Status), s), "clear scratch status")))
        return rc;
    return cuda_check(launch_resample(d_w, N_in, N_out, u0, d_idx, cdf, status, s),
                      "resample (no-alloc)");
}
