// proposal_tc.cu -- inference of the learned proposal sampler on the
// tensor cores (tcgen05, BF16 operands, FP32 accumulation in TMEM), used by
// the BF16 and FP8 forms of the update (the FP32 form keeps the FP32 kernel
// of proposal.cu).
//
// The network (gamma(x) with 6 frequencies, 39 -> 64, three 64 -> 64 ReLU
// layers, linear density head) is small enough to stay resident: the four
// 64 x 64 weight matrices (the first K-padded from 39) live in shared memory
// as BF16 in the 128-byte-swizzled K-major layout for the whole kernel.
// Each CTA runs four warpgroups, each owning 128-row tiles, 64 TMEM columns
// and a 16 KB activation tile; per tile and layer one thread of the group
// issues four 128 x 64 x 16 MMAs, the group reads the accumulators back,
// applies bias + ReLU and writes the next layer's BF16 operand.  The four
// groups interleave, so one group's epilogue overlaps the others' MMAs.
// Every wait is bounded (tc_ptx.cuh).
#include <math.h>

#include "internal.cuh"
#include "tc_ptx.cuh"

namespace mcl {

using namespace tc;

namespace {

constexpr int kPL = 6, kPIn = 39, kPW = 64;
constexpr int kGroups = 4;                         // warpgroups (tile slots) per CTA
constexpr int kThreadsTc = 128 * kGroups;
constexpr uint32_t kLayerBytes = 64 * 128;         // one 64 x 64 BF16 matrix, 128-byte rows
constexpr uint32_t kTileBytes = 128 * 128;         // one 128-row activation tile (64 BF16 per row)
constexpr uint32_t kSmemTc = 1024 + 4 * kLayerBytes + kGroups * kTileBytes;
// blob offsets (proposal.cu): P1 W[64][39] b[64], P2..P4 W[64][64] b[64], head w[64] b[1]
__host__ __device__ constexpr int poff(int l) {
    return l == 0 ? 0 : kPW * kPIn + kPW + (l - 1) * (kPW * kPW + kPW);
}
constexpr int kPOffHead = kPW * kPIn + kPW + 3 * (kPW * kPW + kPW);

struct __align__(8) PBars {
    uint64_t a_ready[kGroups];
    uint64_t mma_done[kGroups];
    uint64_t drain[kGroups];
    uint32_t tmem_base;
};

// gamma(x) with 6 frequencies as 64 BF16 values (39, then zeros), packed in
// pairs: sin / cos of 2^k x by angle doubling from an accurate sincos of x.
__device__ __forceinline__ void prop_pe_bf16(const float x[3], uint32_t (&pk)[32]) {
    float v[64];
#pragma unroll
    for (int i = 0; i < 64; ++i) v[i] = 0.0f;
    v[0] = x[0]; v[1] = x[1]; v[2] = x[2];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        float s, cs;
        sincosf(x[c], &s, &cs);
#pragma unroll
        for (int k = 0; k < kPL; ++k) {
            v[3 + 6 * k + c] = s;
            v[6 + 6 * k + c] = cs;
            const float s2 = 2.0f * s * cs;
            const float c2 = (cs - s) * (cs + s);
            s = s2;
            cs = c2;
        }
    }
#pragma unroll
    for (int i = 0; i < 32; ++i) pk[i] = pack_bf16x2(v[2 * i], v[2 * i + 1]);
}

}  // namespace

// FP32 blob -> BF16 weight matrices [4][64 rows][64 k] in the 128-byte
// swizzled layout (copied verbatim into shared memory by k_prop_tc).
__global__ void k_prop_pack(const float* __restrict__ W, uint16_t* __restrict__ out) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 4 * 64 * 64) return;
    const int l = t >> 12, n = (t >> 6) & 63, k = t & 63;
    const int fin = l == 0 ? kPIn : kPW;
    const float w = k < fin ? W[poff(l) + n * fin + k] : 0.0f;
    const uint32_t off = l * kLayerBytes + sw128_offset((uint32_t)n, (uint32_t)(k >> 3)) + (k & 7) * 2;
    out[off >> 1] = (uint16_t)(pack_bf16x2(w, 0.0f) & 0xFFFFu);
}

__global__ void __launch_bounds__(kThreadsTc, 1)
    k_prop_tc(const float* __restrict__ W, const uint16_t* __restrict__ packed,
              const Ray* __restrict__ rays, const float* __restrict__ z, int n_p, long long rows_max,
              const int* __restrict__ n_rays_dev, float4* __restrict__ out,
              int* __restrict__ abort_flag, int* __restrict__ status_code) {
    extern __shared__ uint8_t smem_raw[];
    __shared__ PBars bars;
    __shared__ float s_bias[4 * kPW + kPW + 1];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const uint32_t s_w = smem_u32(smem);
    const uint32_t s_a = s_w + 4 * kLayerBytes;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int grp = tid >> 7, quad = warp & 3;
    const long long rows = n_rays_dev ? min(rows_max, (long long)*n_rays_dev * n_p) : rows_max;
    const long long n_tiles = (rows + 127) / 128;
    volatile int* err = abort_flag;

    // resident weights and biases
    for (int i = tid; i < (int)(4 * kLayerBytes / 16); i += blockDim.x)
        reinterpret_cast<uint4*>(smem)[i] = reinterpret_cast<const uint4*>(packed)[i];
    for (int i = tid; i < 4 * kPW; i += blockDim.x) {
        const int l = i / kPW, o = i % kPW;
        s_bias[i] = W[poff(l) + kPW * (l == 0 ? kPIn : kPW) + o];
    }
    for (int i = tid; i < kPW + 1; i += blockDim.x) s_bias[4 * kPW + i] = W[kPOffHead + i];
    if (tid == 0) {
        for (int g = 0; g < kGroups; ++g) {
            mbar_init(smem_u32(&bars.a_ready[g]), 128);
            mbar_init(smem_u32(&bars.mma_done[g]), 1);
            mbar_init(smem_u32(&bars.drain[g]), 1);
        }
        fence_mbar_init();
    }
    if (warp == 0) {
        tmem_alloc(smem_u32(&bars.tmem_base), 32 * 2 * kGroups);   // 64 columns per group
        tmem_relinquish();
    }
    fence_proxy_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = bars.tmem_base;

    const uint32_t r = quad * 32 + lane;                            // row within the tile
    const uint32_t t_lane = tmem + ((uint32_t)(quad * 32) << 16) + grp * 64;
    const uint32_t t_mma = tmem + grp * 64;
    const uint32_t a_tile = s_a + grp * kTileBytes;
    const bool issuer = (tid & 127) == 0;
    const uint32_t bar_ready = smem_u32(&bars.a_ready[grp]);
    const uint32_t bar_done = smem_u32(&bars.mma_done[grp]);
    const uint32_t idesc = idesc_bf16(128, 64);
    uint32_t ph_ready = 0, ph_done = 0;
    bool ok = true;
    for (long long tile = (long long)blockIdx.x * kGroups + grp; tile < n_tiles && ok;
         tile += (long long)gridDim.x * kGroups) {
        const long long row = tile * 128 + r;
        const bool valid = row < rows;
        {
            uint32_t pk[32];
            if (valid) {
                const Ray R = rays[row / n_p];
                const float zz = z[row];
                const float x[3] = {fmaf(zz, R.dx, R.ox), fmaf(zz, R.dy, R.oy), fmaf(zz, R.dz, R.oz)};
                prop_pe_bf16(x, pk);
            } else {
#pragma unroll
                for (int i = 0; i < 32; ++i) pk[i] = 0u;
            }
#pragma unroll
            for (int j = 0; j < 8; ++j)
                st_shared_v4(a_tile + sw128_offset(r, j), pk[4 * j], pk[4 * j + 1], pk[4 * j + 2],
                             pk[4 * j + 3]);
            fence_proxy_async_smem();
            tc_fence_before();
            mbar_arrive(bar_ready);
        }
        float sigma = 0.0f;
        for (int l = 0; l < 4 && ok; ++l) {
            if (issuer) {
                if (!mbar_wait(bar_ready, ph_ready, err)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
#pragma unroll
                for (int kk = 0; kk < 4; ++kk) {
                    const uint64_t ad = smem_desc(a_tile + kk * 32, 1024, kLayoutSw128);
                    const uint64_t bd = smem_desc(s_w + l * kLayerBytes + kk * 32, 1024, kLayoutSw128);
                    mma_bf16(t_mma, ad, bd, idesc, kk ? 1u : 0u);
                }
                mma_commit(bar_done);
            }
            ph_ready ^= 1u;
            if (!mbar_wait(bar_done, ph_done, err)) {
                ok = false;
                break;
            }
            ph_done ^= 1u;
            tc_fence_after();
            uint32_t va[32], vb[32];
            tmem_ld32(t_lane, va);
            tmem_ld32(t_lane + 32, vb);
            tmem_ld_wait();
            const float* b = s_bias + l * kPW;
            if (l < 3) {
                uint32_t pk[32];
#pragma unroll
                for (int i = 0; i < 16; ++i)
                    pk[i] = pack_bf16x2(fmaxf(__uint_as_float(va[2 * i]) + b[2 * i], 0.0f),
                                        fmaxf(__uint_as_float(va[2 * i + 1]) + b[2 * i + 1], 0.0f));
#pragma unroll
                for (int i = 0; i < 16; ++i)
                    pk[16 + i] = pack_bf16x2(fmaxf(__uint_as_float(vb[2 * i]) + b[32 + 2 * i], 0.0f),
                                             fmaxf(__uint_as_float(vb[2 * i + 1]) + b[33 + 2 * i], 0.0f));
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    st_shared_v4(a_tile + sw128_offset(r, j), pk[4 * j], pk[4 * j + 1], pk[4 * j + 2],
                                 pk[4 * j + 3]);
                fence_proxy_async_smem();
                tc_fence_before();
                mbar_arrive(bar_ready);
            } else {
                const float* hw = s_bias + 4 * kPW;
                float s = hw[kPW];
#pragma unroll
                for (int i = 0; i < 32; ++i) s = fmaf(fmaxf(__uint_as_float(va[i]) + b[i], 0.0f), hw[i], s);
#pragma unroll
                for (int i = 0; i < 32; ++i)
                    s = fmaf(fmaxf(__uint_as_float(vb[i]) + b[32 + i], 0.0f), hw[32 + i], s);
                sigma = s;
                tc_fence_before();
            }
        }
        if (ok && valid) out[row] = make_float4(sigma, 0.0f, 0.0f, 0.0f);
    }
    if (!ok) atomicCAS(status_code, 0, MCL_ERR_TIMEOUT);
    if (issuer) {
        // every MMA of this group completes before TMEM is released
        mma_commit(smem_u32(&bars.drain[grp]));
        mbar_wait(smem_u32(&bars.drain[grp]), 0, nullptr);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, 32 * 2 * kGroups);
    }
}

cudaError_t prop_tc_pack(mcl_map* m, cudaStream_t s) {
    note_launch();
    k_prop_pack<<<(4 * 64 * 64 + 255) / 256, 256, 0, s>>>(m->prop_w, m->prop_packed);
    return cudaGetLastError();
}

cudaError_t prop_tc_prepare() {
    return cudaFuncSetAttribute(k_prop_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemTc);
}

cudaError_t launch_prop_infer_tc(mcl_map* m, const Ray* rays, const float* z, int n_p, int n_rays,
                                 const int* n_rays_dev, float4* out, int n_sm, cudaStream_t s) {
    const long long rows = (long long)n_rays * n_p;
    const long long tiles = (rows + 127) / 128;
    long long grid = (tiles + kGroups - 1) / kGroups;
    if (grid > n_sm) grid = n_sm;
    if (grid < 1) grid = 1;
    cudaError_t e = cudaMemsetAsync(m->prop_abort, 0, sizeof(int), s);
    if (e) return e;
    note_launch();
    k_prop_tc<<<(unsigned)grid, kThreadsTc, kSmemTc, s>>>(m->prop_w, m->prop_packed, rays, z, n_p, rows,
                                                         n_rays_dev, out, m->prop_abort,
                                                         &m->status->code);
    return cudaGetLastError();
}

}  // namespace mcl
