// probe.cu -- a diagnostic of the tensor-core issue path behind the NeRF MLP
// kernel's schedule: the throughput of back-to-back tcgen05 MMAs (BF16,
// M = 128, N = 256, K = 16, both operands in shared memory, FP32 accumulators
// in TMEM) issued by one thread of each CTA (one CTA per SM), in groups of
// G MMAs separated by a dependent chain of D integer multiply-adds in the
// issuing thread.  With D = 0 it measures the per-SM MMA rate; with D > 0 it
// shows how far the issuing thread runs ahead of the tensor pipe, i.e. how
// much work a group leaves queued while the thread does something else.
// The operands are zero (their values do not affect the timing).
#include <algorithm>
#include <vector>

#include "internal.cuh"
#include "tc_ptx.cuh"

namespace mcl {

namespace {

using namespace tc;

constexpr int kProbeSmem = 128 * 1024 + 1024;   // A: 4 K-blocks x 16 KB, B: 4 blocks x 16 KB

__global__ void __launch_bounds__(128, 1)
    k_probe_mma(int group, int gap, int n_groups, long long* cycles, long long* gap_cycles,
                int* status) {
    extern __shared__ uint8_t smem_raw[];
    __shared__ uint64_t bar;
    __shared__ uint32_t tbase;
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int tid = threadIdx.x;
    for (int i = tid; i < 128 * 1024 / 16; i += blockDim.x)
        reinterpret_cast<uint4*>(smem)[i] = make_uint4(0u, 0u, 0u, 0u);
    if (tid == 0) {
        mbar_init(smem_u32(&bar), 1);
        fence_mbar_init();
    }
    if (tid < 32) {
        tmem_alloc(smem_u32(&tbase), 512);
        tmem_relinquish();
    }
    fence_proxy_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tbase;
    if (tid == 0) {
        const uint32_t sA = smem_u32(smem), sB = sA + 65536;
        // A: K-blocks of 128 rows x 128 bytes (128-byte swizzle); B: blocks of
        // 256 rows x 64 bytes (64-byte swizzle), the layouts of the MLP kernel
        const uint64_t dA = smem_desc(sA, 1024, kLayoutSw128);
        const uint64_t dB = smem_desc(sB, 512, kLayoutSw64);
        const uint32_t idesc = idesc_bf16(128, 256);
        uint32_t x = (uint32_t)clock();
        const long long tg = clock64();
#pragma unroll 1
        for (int k = 0; k < gap; ++k) asm volatile("mad.lo.u32 %0, %0, 1664525, 1013904223;" : "+r"(x));
        const long long t_gap = clock64() - tg;
        const long long t0 = clock64();
#pragma unroll 1
        for (int b = 0; b < n_groups; ++b) {
#pragma unroll 1
            for (int j = 0; j < group; ++j) {
                const int i = b * group + j;
                mma_bf16(tmem + (uint32_t)(i & 1) * 256u, dA + (uint64_t)((i & 3) * 1024),
                         dB + (uint64_t)((i & 3) * 1024), idesc, 1u);
            }
#pragma unroll 1
            for (int k = 0; k < gap; ++k) asm volatile("mad.lo.u32 %0, %0, 1664525, 1013904223;" : "+r"(x));
        }
        mma_commit(smem_u32(&bar));
        const bool ok = mbar_wait(smem_u32(&bar), 0, nullptr);
        cycles[blockIdx.x] = ok ? clock64() - t0 : -1;
        if (blockIdx.x == 0) gap_cycles[0] = t_gap + (x == 0x9e3779b9u ? 1 : 0);
        if (!ok) atomicExch(status, MCL_ERR_TIMEOUT);
    }
    tc_fence_before();
    __syncthreads();
    if (tid < 32) {
        tc_fence_after();
        tmem_dealloc(tmem, 512);
    }
}

}  // namespace

}  // namespace mcl

using namespace mcl;

extern "C" int mcl_probe_mma_rate(int group, int gap, int n_groups, double* clk_per_group,
                                  double* gap_clk) {
    clear_error();
    if (group < 1 || group > 64 || gap < 0 || gap > 4096 || n_groups < 1 || n_groups > 100000 ||
        !clk_per_group)
        return fail(MCL_ERR_ARG, "mcl_probe_mma_rate: 1 <= group <= 64, 0 <= gap <= 4096, "
                                 "1 <= n_groups <= 100000, clk_per_group not NULL");
    int dev = 0, major = 0, minor = 0, n_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
    cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    if (major != 10 || minor != 3)
        return fail(MCL_ERR_UNSUPPORTED, "mcl_probe_mma_rate: needs sm_103 (found sm_%d%d)", major, minor);
    long long *cyc = nullptr, *gcyc = nullptr;
    int* status = nullptr;
    int rc = MCL_OK;
    if ((rc = cuda_check(cudaMalloc(&cyc, sizeof(long long) * n_sm), "probe buffers")) ||
        (rc = cuda_check(cudaMalloc(&gcyc, sizeof(long long)), "probe buffers")) ||
        (rc = cuda_check(cudaMalloc(&status, sizeof(int)), "probe buffers")) ||
        (rc = cuda_check(cudaMemset(status, 0, sizeof(int)), "probe status")) ||
        (rc = cuda_check(cudaFuncSetAttribute(k_probe_mma, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              kProbeSmem),
                         "probe smem"))) {
        cudaFree(cyc);
        cudaFree(gcyc);
        cudaFree(status);
        return rc;
    }
    std::vector<long long> h(n_sm);
    long long g = 0;
    int st = 0;
    for (int rep = 0; rep < 2 && !rc; ++rep) {   // the first launch warms up
        note_launch();
        k_probe_mma<<<n_sm, 128, kProbeSmem>>>(group, gap, n_groups, cyc, gcyc, status);
        rc = cuda_check(cudaDeviceSynchronize(), "probe launch");
    }
    if (!rc) rc = cuda_check(cudaMemcpy(h.data(), cyc, sizeof(long long) * n_sm, cudaMemcpyDeviceToHost), "probe read");
    if (!rc) rc = cuda_check(cudaMemcpy(&g, gcyc, sizeof(long long), cudaMemcpyDeviceToHost), "probe read");
    if (!rc) rc = cuda_check(cudaMemcpy(&st, status, sizeof(int), cudaMemcpyDeviceToHost), "probe read");
    cudaFree(cyc);
    cudaFree(gcyc);
    cudaFree(status);
    if (rc) return rc;
    if (st) return fail(st, "mcl_probe_mma_rate: a wait ran out");
    std::sort(h.begin(), h.end());
    *clk_per_group = (double)h[n_sm / 2] / n_groups;   // median over SMs
    if (gap_clk) *gap_clk = (double)g;
    return MCL_OK;
}
