// mlp_tc.cu -- the NeRF MLP on the 5th-generation tensor cores (tcgen05,
// BF16 operands, FP32 accumulation in TMEM), fused across all layers.
//
// One persistent CTA per SM walks over pairs of 128-row tiles (rows are the
// samples of the pass, row = ray * S + k).  Per pair:
//   prologue   x = o + z d, gamma(x) (63 -> 64, BF16) into shared memory;
//   9 layers   trunk 1..8 (ReLU; gamma(x) re-enters layer 6 through the skip),
//              then the RGB hidden layer with the feature layer folded in
//              (W' = W_rgb_hidden[:, :256] W_feature, computed in FP64 when
//              the map is loaded: the feature layer has no activation);
//   epilogues  TMEM -> registers, bias + ReLU, BF16 back into the same
//              shared-memory tile as the next layer's A operand; the density
//              head (256 -> 1) as a per-row dot product after trunk layer 8;
//              the RGB output layer (128 -> 3, sigmoid) after the last MMA,
//              with gamma(d)'s contribution added as a per-ray bias.
// Warp roles: warp 0 streams weight blocks [256 x 32] (64-byte swizzle) by
// TMA through a 4-stage ring; warp 1 allocates TMEM and issues the MMAs for
// both tiles from the same weight block (M = 128, N = 256, K = 16 per
// instruction); warps 2-5 and 6-9 run prologue and epilogues of tile 0 and
// tile 1 (one warp per TMEM lane quadrant, one thread per row).  Every wait
// is bounded (see tc_ptx.cuh).
#include <cuda.h>
#include <cudaTypedefs.h>
#include <math.h>
#include <string.h>

#include <vector>

#include "internal.cuh"
#include "tc_ptx.cuh"

#ifdef MCL_TC_TRACE
// Timeline instrumentation of CTA 0 (compiled only with -DMCL_TC_TRACE):
// globaltimer stamps of the MMA issuer, the first row of each tile's
// epilogue and the TMA producer for the first two tile pairs.
constexpr int kTraceSlots = 16, kTraceLen = 128;
__device__ unsigned long long g_tc_trace[kTraceSlots * kTraceLen];
#define TC_TRACE(slot, idx)                                                           \
    do {                                                                              \
        if (blockIdx.x == 0 && (slot) < kTraceSlots && (idx) < kTraceLen)             \
            g_tc_trace[(slot) * kTraceLen + (idx)] = mcl::tc::globaltimer();          \
    } while (0)
extern "C" int mcl_tc_trace_read(unsigned long long* out, int n) {
    const int m = n < kTraceSlots * kTraceLen ? n : kTraceSlots * kTraceLen;
    return (int)cudaMemcpyFromSymbol(out, g_tc_trace, sizeof(unsigned long long) * m);
}
#else
#define TC_TRACE(slot, idx) \
    do {                    \
    } while (0)
#endif

namespace mcl {

using namespace tc;

namespace {

constexpr int kEpiThreads = 128;                // 4 warps per 128-row tile
constexpr int kThreads = 64 + 2 * kEpiThreads;   // + TMA warp + MMA warp
constexpr int kStages = 4;
constexpr uint32_t kStageBytes = 256 * 32 * 2;  // one weight block [256 rows x 32 k] bf16
constexpr uint32_t kActBytes = 128 * 256 * 2;   // one tile's activations (4 K-blocks of 64)
constexpr uint32_t kGxBytes = 128 * 64 * 2;     // one tile's gamma(x)
constexpr int kLayers = 9;
constexpr int kBlocksPerPair = 68;              // weight blocks streamed per tile pair
constexpr uint32_t kSmemBytes = 1024 + 2 * kActBytes + 2 * kGxBytes + kStages * kStageBytes;
// 32-wide K chunks (one weight block each) per layer: trunk1 reads gamma(x)
// (64), trunk6 reads [h (256), gamma(x) (64)], the others h (256).  The last
// layer has N = 144: rows 0..127 are the RGB hidden layer (feature layer
// folded in), row 128 the density head, so sigma_raw arrives as accumulator
// column 128 of the last MMA.
__constant__ int c_chunks[kLayers] = {2, 8, 8, 8, 8, 10, 8, 8, 8};

struct Params {
    const Ray* rays;
    const float* z;
    int S;
    long long M;            // rows of the pass (upper bound when M_dev is set)
    long long n_pairs;
    const int* M_dev;       // optional: rows of the pass from device memory
    const uint32_t* bias2;  // [8][128] trunk biases as BF16 pairs
    float b_sigma;
    const float* ray_bias;  // [n_rays][128]
    const float* w_out;     // [3][128]
    float b_out0, b_out1, b_out2;
    float4* out;
    int* abort_flag;        // per-launch: set on a timed-out wait
    int* status_code;       // map status word
};

struct __align__(8) Bars {
    uint64_t full[kStages];
    uint64_t empty[kStages];
    uint64_t acc_full[2];
    uint64_t a_ready[2];
    uint64_t drain;
    uint32_t tmem_base;
};

__device__ __forceinline__ void record_abort(const Params& p) {
    atomicCAS(p.status_code, 0, MCL_ERR_TIMEOUT);
}

// gamma(x) of one row as 32 packed BF16 pairs; sin / cos of 2^k x by angle
// doubling from an accurate sincos of x (error ~2^k ulp, far below BF16).
__device__ __forceinline__ void pe_row_bf16(const float x[3], uint32_t (&pk)[32]) {
    float v[64];
    v[0] = x[0]; v[1] = x[1]; v[2] = x[2];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        float s, cs;
        sincosf(x[c], &s, &cs);
#pragma unroll
        for (int k = 0; k < kLxyz; ++k) {
            v[3 + 6 * k + c] = s;
            v[6 + 6 * k + c] = cs;
            const float s2 = 2.0f * s * cs;
            const float c2 = (cs - s) * (cs + s);
            s = s2;
            cs = c2;
        }
    }
    v[63] = 0.0f;
#pragma unroll
    for (int i = 0; i < 32; ++i) pk[i] = pack_bf16x2(v[2 * i], v[2 * i + 1]);
}

// 32 accumulator columns of one row -> relu(acc + bias) as BF16 -> four
// 16-byte chunks (j0 .. j0+3) of the row in a 128-byte-swizzled K-block.
__device__ __forceinline__ void epi_chunk_store(const uint32_t (&v)[32], const uint4* b4,
                                                uint32_t blk, uint32_t r, uint32_t j0) {
    const uint32_t one2 = 0x3F803F80u;  // (1.0, 1.0) in BF16
    uint32_t pk[16];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const uint4 b = __ldg(b4 + q);
        const uint32_t bb[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int i = 4 * q + e;
            const uint32_t a = pack_bf16x2(__uint_as_float(v[2 * i]), __uint_as_float(v[2 * i + 1]));
            uint32_t h;
            asm("fma.rn.relu.bf16x2 %0, %1, %2, %3;" : "=r"(h) : "r"(a), "r"(one2), "r"(bb[e]));
            pk[i] = h;
        }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q)
        st_shared_v4(blk + sw128_offset(r, j0 + q), pk[4 * q], pk[4 * q + 1], pk[4 * q + 2],
                     pk[4 * q + 3]);
}

__global__ void __launch_bounds__(kThreads, 1)
    k_mlp_tc(const __grid_constant__ CUtensorMap tmap, const Params p) {
    extern __shared__ uint8_t smem_raw[];
    __shared__ Bars bars;
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const uint32_t s_act = smem_u32(smem);                    // 2 x 64 KB
    const uint32_t s_gx = s_act + 2 * kActBytes;              // 2 x 16 KB
    const uint32_t s_ring = s_gx + 2 * kGxBytes;              // kStages x 16 KB
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    volatile int* abort_flag = p.abort_flag;
    // rows of this pass: fixed, or decided on the device by an earlier kernel
    const long long M = p.M_dev ? min(p.M, (long long)*p.M_dev) : p.M;
    const long long n_pairs = (M + 255) / 256;

    if (tid == 0) {
        for (int i = 0; i < kStages; ++i) {
            mbar_init(smem_u32(&bars.full[i]), 1);
            mbar_init(smem_u32(&bars.empty[i]), 1);
        }
        for (int s = 0; s < 2; ++s) {
            mbar_init(smem_u32(&bars.acc_full[s]), 1);
            mbar_init(smem_u32(&bars.a_ready[s]), kEpiThreads);
        }
        mbar_init(smem_u32(&bars.drain), 1);
        fence_mbar_init();
        tma_prefetch_desc(&tmap);
    }
    if (warp == 1) {
        tmem_alloc(smem_u32(&bars.tmem_base), 512);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = bars.tmem_base;

    if (warp == 0) {
        // ------------------------------------------------ TMA producer
        if (lane == 0) {
            uint32_t issued[kStages] = {0, 0, 0, 0};
            uint32_t g = 0;
            bool ok = true;
            for (long long pr = blockIdx.x; pr < n_pairs && ok; pr += gridDim.x) {
                for (int b = 0; b < kBlocksPerPair; ++b, ++g) {
                    const uint32_t st = g % kStages, ph = (g / kStages) & 1u;
                    TC_TRACE(0, g);
                    if (!mbar_wait(smem_u32(&bars.empty[st]), ph ^ 1u, abort_flag)) {
                        ok = false;
                        break;
                    }
                    TC_TRACE(1, g);
                    mbar_arrive_expect_tx(smem_u32(&bars.full[st]), kStageBytes);
                    tma_load_2d(s_ring + st * kStageBytes, &tmap, 0, b * 256,
                                smem_u32(&bars.full[st]));
                    ++issued[st];
                }
            }
            if (!ok) record_abort(p);
            // every issued copy lands before the CTA may exit
            for (int st = 0; st < kStages; ++st)
                if (issued[st])
                    mbar_wait(smem_u32(&bars.full[st]), (issued[st] - 1) & 1u, nullptr);
        }
    } else if (warp == 1) {
        // ------------------------------------------------ MMA issuer
        if (lane == 0) {
            uint32_t g = 0;
            uint32_t rdy_ph[2] = {0, 0};
            bool ok = true;
            const uint32_t id256 = idesc_bf16(128, 256), id144 = idesc_bf16(128, 144);
            int tl = 0;
            for (long long pr = blockIdx.x; pr < n_pairs && ok; pr += gridDim.x) {
                for (int l = 0; l < kLayers && ok; ++l, ++tl) {
                    const int nch = c_chunks[l];
                    const uint32_t idesc = (l == 8) ? id144 : id256;
                    TC_TRACE(2, tl);
                    for (int c = 0; c < nch && ok; ++c) {
                        const uint32_t st = g % kStages, ph = (g / kStages) & 1u;
                        if (!mbar_wait(smem_u32(&bars.full[st]), ph, abort_flag)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        for (int s = 0; s < 2; ++s) {
                            if (c == 0) {
                                if (!mbar_wait(smem_u32(&bars.a_ready[s]), rdy_ph[s], abort_flag)) {
                                    ok = false;
                                    break;
                                }
                                TC_TRACE(3 + s, tl);
                                rdy_ph[s] ^= 1u;
                                tc_fence_after();
                            }
#pragma unroll
                            for (int kk = 0; kk < 2; ++kk) {
                                uint32_t a_addr;
                                if (l == 0) {
                                    a_addr = s_gx + s * kGxBytes + (c * 2 + kk) * 32;
                                } else if (l == 5 && c >= 8) {
                                    a_addr = s_gx + s * kGxBytes + ((c - 8) * 2 + kk) * 32;
                                } else {
                                    const int ks = c * 2 + kk;
                                    a_addr = s_act + s * kActBytes + (ks >> 2) * 16384 + (ks & 3) * 32;
                                }
                                const uint64_t ad = smem_desc(a_addr, 1024, kLayoutSw128);
                                const uint64_t bd =
                                    smem_desc(s_ring + st * kStageBytes + kk * 32, 512, kLayoutSw64);
                                mma_bf16(tmem + s * 256, ad, bd, idesc, (c | kk) ? 1u : 0u);
                            }
                            if (c == nch - 1) mma_commit(smem_u32(&bars.acc_full[s]));
                        }
                        if (!ok) break;
                        mma_commit(smem_u32(&bars.empty[st]));
                        ++g;
                    }
                    TC_TRACE(5, tl);
                }
            }
            if (!ok) record_abort(p);
            // all issued MMAs complete before TMEM is released
            mma_commit(smem_u32(&bars.drain));
            mbar_wait(smem_u32(&bars.drain), 0, nullptr);
        }
    } else {
        // ------------------------------------------------ prologue / epilogues
        // 4 warps per tile: warp w covers TMEM lane quadrant (w % 4), i.e. rows
        // 32 (w % 4) .. +31, all columns; one thread owns one row.
        const int slot = (warp - 2) >> 2;
        const int quad = warp & 3;
        const uint32_t r = quad * 32 + lane;              // row within the tile
        const uint32_t t_acc = tmem + ((uint32_t)(quad * 32) << 16) + slot * 256;
        const uint32_t a_base = s_act + slot * kActBytes;
        const uint32_t g_base = s_gx + slot * kGxBytes;
        const uint32_t bar_ready = smem_u32(&bars.a_ready[slot]);
        const uint32_t bar_acc = smem_u32(&bars.acc_full[slot]);
        uint32_t acc_ph = 0;
        bool ok = true;
        const bool tracer = (r == 0);
        int tl = 0;
        for (long long pr = blockIdx.x; pr < n_pairs && ok; pr += gridDim.x) {
            const long long grow = pr * 256 + slot * 128 + r;
            const bool valid = grow < M;
            const long long ray = valid ? grow / p.S : 0;
            // ---- prologue: gamma(x) of this row into the tile's gamma(x) buffer
            {
                uint32_t pk[32];
                if (valid) {
                    const Ray R = p.rays[ray];
                    const float zz = p.z[grow];
                    const float x[3] = {fmaf(zz, R.dx, R.ox), fmaf(zz, R.dy, R.oy),
                                        fmaf(zz, R.dz, R.oz)};
                    pe_row_bf16(x, pk);
                } else {
#pragma unroll
                    for (int i = 0; i < 32; ++i) pk[i] = 0u;
                }
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    st_shared_v4(g_base + sw128_offset(r, j), pk[4 * j], pk[4 * j + 1],
                                 pk[4 * j + 2], pk[4 * j + 3]);
                fence_proxy_async_smem();
                tc_fence_before();
                mbar_arrive(bar_ready);
            }
            float sigma = 0.0f;
            for (int l = 0; l < kLayers && ok; ++l, ++tl) {
                if (!mbar_wait(bar_acc, acc_ph, abort_flag)) {
                    ok = false;
                    break;
                }
                if (tracer) TC_TRACE(6 + 2 * slot, tl);
                acc_ph ^= 1u;
                tc_fence_after();
                if (l < 8) {
                    // h = relu(acc + b): accumulators rounded to BF16 pairs,
                    // bias added and ReLU applied in packed BF16 arithmetic
                    const uint4* b4 = reinterpret_cast<const uint4*>(p.bias2 + l * 128);
                    uint32_t va[32], vb[32];
                    tmem_ld32(t_acc, va);
#pragma unroll 1
                    for (int c32 = 0; c32 < 8; c32 += 2) {
                        tmem_ld_wait();
                        if (tracer && slot == 0 && tl < 16) TC_TRACE(10 + (c32 >> 1), tl);
                        tmem_ld32(t_acc + (c32 + 1) * 32, vb);
                        const uint32_t blk = a_base + (c32 >> 1) * 16384;
                        epi_chunk_store(va, b4 + c32 * 4, blk, r, 0);
                        tmem_ld_wait();
                        if (c32 + 2 < 8) tmem_ld32(t_acc + (c32 + 2) * 32, va);
                        epi_chunk_store(vb, b4 + (c32 + 1) * 4, blk, r, 4);
                    }
                    if (tracer && slot == 0 && tl < 16) TC_TRACE(14, tl);
                    fence_proxy_async_smem();
                    tc_fence_before();
                    if (tracer) TC_TRACE(7 + 2 * slot, tl);
                    mbar_arrive(bar_ready);
                } else {
                    const float4* rb4 = reinterpret_cast<const float4*>(p.ray_bias + ray * 128);
                    const float4* wo4 = reinterpret_cast<const float4*>(p.w_out);
                    float o0 = 0.f, o1 = 0.f, o2 = 0.f;
                    uint32_t va[32], vb[32];
                    tmem_ld32(t_acc, va);
#pragma unroll 1
                    for (int c32 = 0; c32 < 4; c32 += 2) {
                        tmem_ld_wait();
                        tmem_ld32(t_acc + (c32 + 1) * 32, vb);
#pragma unroll
                        for (int q = 0; q < 8; ++q) {
                            const float4 b = __ldg(rb4 + c32 * 8 + q);
                            const float4 w0 = __ldg(wo4 + c32 * 8 + q);
                            const float4 w1 = __ldg(wo4 + 32 + c32 * 8 + q);
                            const float4 w2 = __ldg(wo4 + 64 + c32 * 8 + q);
                            const float h0 = fmaxf(__uint_as_float(va[4 * q + 0]) + b.x, 0.0f);
                            const float h1 = fmaxf(__uint_as_float(va[4 * q + 1]) + b.y, 0.0f);
                            const float h2 = fmaxf(__uint_as_float(va[4 * q + 2]) + b.z, 0.0f);
                            const float h3 = fmaxf(__uint_as_float(va[4 * q + 3]) + b.w, 0.0f);
                            o0 = fmaf(h0, w0.x, fmaf(h1, w0.y, fmaf(h2, w0.z, fmaf(h3, w0.w, o0))));
                            o1 = fmaf(h0, w1.x, fmaf(h1, w1.y, fmaf(h2, w1.z, fmaf(h3, w1.w, o1))));
                            o2 = fmaf(h0, w2.x, fmaf(h1, w2.y, fmaf(h2, w2.z, fmaf(h3, w2.w, o2))));
                        }
                        tmem_ld_wait();
                        if (c32 + 2 < 4) tmem_ld32(t_acc + (c32 + 2) * 32, va);
#pragma unroll
                        for (int q = 0; q < 8; ++q) {
                            const float4 b = __ldg(rb4 + (c32 + 1) * 8 + q);
                            const float4 w0 = __ldg(wo4 + (c32 + 1) * 8 + q);
                            const float4 w1 = __ldg(wo4 + 32 + (c32 + 1) * 8 + q);
                            const float4 w2 = __ldg(wo4 + 64 + (c32 + 1) * 8 + q);
                            const float h0 = fmaxf(__uint_as_float(vb[4 * q + 0]) + b.x, 0.0f);
                            const float h1 = fmaxf(__uint_as_float(vb[4 * q + 1]) + b.y, 0.0f);
                            const float h2 = fmaxf(__uint_as_float(vb[4 * q + 2]) + b.z, 0.0f);
                            const float h3 = fmaxf(__uint_as_float(vb[4 * q + 3]) + b.w, 0.0f);
                            o0 = fmaf(h0, w0.x, fmaf(h1, w0.y, fmaf(h2, w0.z, fmaf(h3, w0.w, o0))));
                            o1 = fmaf(h0, w1.x, fmaf(h1, w1.y, fmaf(h2, w1.z, fmaf(h3, w1.w, o1))));
                            o2 = fmaf(h0, w2.x, fmaf(h1, w2.y, fmaf(h2, w2.z, fmaf(h3, w2.w, o2))));
                        }
                    }
                    {
                        // density head: accumulator column 128 of the last MMA
                        uint32_t vs[32];
                        tmem_ld32(t_acc + 128, vs);
                        tmem_ld_wait();
                        sigma = __uint_as_float(vs[0]);
                    }
                    tc_fence_before();
                    if (valid) {
                        float4 res;
                        res.x = sigma + p.b_sigma;
                        res.y = 1.0f / (1.0f + __expf(-(o0 + p.b_out0)));
                        res.z = 1.0f / (1.0f + __expf(-(o1 + p.b_out1)));
                        res.w = 1.0f / (1.0f + __expf(-(o2 + p.b_out2)));
                        p.out[grow] = res;
                    }
                }
            }
        }
        if (!ok) record_abort(p);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, 512);
    }
}

// Per-ray bias of the RGB hidden layer: b'_ray = b' + W_rgb_hidden[:, 256:283] gamma(d).
__global__ void k_ray_bias(const float* __restrict__ gd, int n_rays, const int* __restrict__ n_dev,
                           const float* __restrict__ Wd, const float* __restrict__ bprime,
                           float* __restrict__ out) {
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    const int n = n_dev ? min(n_rays, *n_dev) : n_rays;
    if (t >= (long)n * 128) return;
    const long ray = t >> 7;
    const int o = (int)(t & 127);
    const float* g = gd + ray * kGdPad;
    float s = bprime[o];
#pragma unroll
    for (int i = 0; i < kGd; ++i) s = fmaf(Wd[o * kGd + i], g[i], s);
    out[t] = s;
}

struct TcState {
    CUtensorMap tmap;
    void* wblocks = nullptr;   // bf16 weight blocks
    float* aux = nullptr;      // fp32 biases and small heads
    float* ray_bias = nullptr; // [max_rays][128]
    int* abort_flag = nullptr;
    const uint32_t* bias2 = nullptr;
    const float* w_out = nullptr;
    const float* Wd = nullptr;
    const float* bprime = nullptr;
    float b_sigma = 0.f, b_out[3] = {0.f, 0.f, 0.f};
    int n_sm = 0;
    bool ready = false;
};

inline uint16_t f2bf(float f) {
    uint32_t u;
    memcpy(&u, &f, 4);
    if ((u & 0x7fffffffu) > 0x7f800000u) return 0x7fc0;  // NaN
    const uint32_t lsb = (u >> 16) & 1u;
    u += 0x7fffu + lsb;                                   // round to nearest even
    return (uint16_t)(u >> 16);
}

}  // namespace

int mlp_tc_prepare(mcl_map* m, const float* blob) {
    TcState* st = new TcState();
    m->tc_aux = st;
    // ---- layer views of the FP32 blob
    int fin[12], fout[12];
    for (int l = 0; l < kDepth; ++l) {
        fin[l] = (l == 0) ? kGx : (l == kSkip ? kWidth + kGx : kWidth);
        fout[l] = kWidth;
    }
    fin[8] = kWidth; fout[8] = 1;
    fin[9] = kWidth; fout[9] = kWidth;
    fin[10] = kWidth + kGd; fout[10] = kRgbW;
    fin[11] = kRgbW; fout[11] = 3;
    const float* Wp[12];
    const float* bp[12];
    const float* q = blob;
    for (int l = 0; l < 12; ++l) {
        Wp[l] = q;
        q += (size_t)fin[l] * fout[l];
        bp[l] = q;
        q += fout[l];
    }
    // ---- fold the linear feature layer into the RGB hidden layer (FP64)
    std::vector<double> Wfold((size_t)kRgbW * kWidth, 0.0), bfold(kRgbW, 0.0);
    for (int o = 0; o < kRgbW; ++o) {
        const float* wr = Wp[10] + (size_t)o * fin[10];
        double bb = bp[10][o];
        for (int j = 0; j < kWidth; ++j) bb += (double)wr[j] * bp[9][j];
        bfold[o] = bb;
        for (int i = 0; i < kWidth; ++i) {
            double s = 0.0;
            for (int j = 0; j < kWidth; ++j) s += (double)wr[j] * Wp[9][(size_t)j * kWidth + i];
            Wfold[(size_t)o * kWidth + i] = s;
        }
    }
    // ---- weight blocks [256 rows][32 k] in consumption order
    std::vector<uint16_t> blk((size_t)kBlocksPerPair * 256 * 32, 0);
    int b = 0;
    auto put_chunk = [&](int block, int row0, int nrows, auto getter, int k0) {
        for (int n = 0; n < nrows; ++n)
            for (int k = 0; k < 32; ++k)
                blk[((size_t)block * 256 + row0 + n) * 32 + k] = f2bf((float)getter(n, k0 + k));
    };
    // trunk layers: K padded (gamma(x) 63 -> 64); layer 6 = [h | gamma(x)]
    for (int l = 0; l < kDepth; ++l) {
        const int K = (l == 0) ? kGxPad : (l == kSkip ? kWidth + kGxPad : kWidth);
        for (int k0 = 0; k0 < K; k0 += 32, ++b) {
            // column k of the padded layer is column k of the blob layer
            // ([h, gamma(x)] order for the skip layer); padding columns are 0
            auto get = [&](int n, int k) -> double {
                if (k >= fin[l]) return 0.0;
                return (double)Wp[l][(size_t)n * fin[l] + k];
            };
            put_chunk(b, 0, 256, get, k0);
        }
    }
    // last layer, N = 144: rows 0..127 RGB hidden (folded), row 128 density head
    for (int k0 = 0; k0 < kWidth; k0 += 32, ++b) {
        auto get = [&](int n, int k) -> double { return Wfold[(size_t)n * kWidth + k]; };
        put_chunk(b, 0, 128, get, k0);
        auto gets = [&](int n, int k) -> double { (void)n; return (double)Wp[8][k]; };
        put_chunk(b, 128, 1, gets, k0);
    }
    if (b != kBlocksPerPair) return fail(MCL_ERR_UNSUPPORTED, "internal: weight block count %d", b);
    // ---- aux: trunk biases as BF16 pairs [8][128] (bit patterns stored in
    //      floats), w_out [3][128], W_d [128][27], b' [128]
    std::vector<float> aux;
    const size_t o_bias = aux.size();
    for (int l = 0; l < kDepth; ++l)
        for (int j = 0; j < kWidth / 2; ++j) {
            const uint32_t pr = (uint32_t)f2bf(bp[l][2 * j]) | ((uint32_t)f2bf(bp[l][2 * j + 1]) << 16);
            float f;
            memcpy(&f, &pr, 4);
            aux.push_back(f);
        }
    const size_t o_wout = aux.size();
    aux.insert(aux.end(), Wp[11], Wp[11] + 3 * kRgbW);
    const size_t o_wd = aux.size();
    for (int o = 0; o < kRgbW; ++o)
        for (int i = 0; i < kGd; ++i) aux.push_back(Wp[10][(size_t)o * fin[10] + kWidth + i]);
    const size_t o_bp = aux.size();
    for (int o = 0; o < kRgbW; ++o) aux.push_back((float)bfold[o]);
    st->b_sigma = bp[8][0];
    for (int c = 0; c < 3; ++c) st->b_out[c] = bp[11][c];

    int rc;
    if ((rc = cuda_check(cudaMalloc(&st->wblocks, blk.size() * 2), "cudaMalloc(tc weights)"))) return rc;
    if ((rc = cuda_check(cudaMemcpy(st->wblocks, blk.data(), blk.size() * 2, cudaMemcpyHostToDevice),
                         "upload tc weights")))
        return rc;
    if ((rc = cuda_check(cudaMalloc(&st->aux, aux.size() * 4), "cudaMalloc(tc aux)"))) return rc;
    if ((rc = cuda_check(cudaMemcpy(st->aux, aux.data(), aux.size() * 4, cudaMemcpyHostToDevice),
                         "upload tc aux")))
        return rc;
    if ((rc = cuda_check(cudaMalloc(&st->ray_bias, (size_t)m->cfg.max_rays * 128 * 4), "ray bias")))
        return rc;
    if ((rc = cuda_check(cudaMalloc(&st->abort_flag, sizeof(int)), "abort flag"))) return rc;
    st->bias2 = reinterpret_cast<const uint32_t*>(st->aux + o_bias);
    st->w_out = st->aux + o_wout;
    st->Wd = st->aux + o_wd;
    st->bprime = st->aux + o_bp;

    // ---- tensor map over the weight blocks: [64*256 rows][32] bf16, box 32 x 256
    PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    cudaDriverEntryPointQueryResult qr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", (void**)&encode, 12000,
                                         cudaEnableDefault, &qr) != cudaSuccess ||
        qr != cudaDriverEntryPointSuccess || !encode) {
        cudaGetLastError();
        // no driver (CPU-only machine): the tensor-core form stays unavailable
        return MCL_OK;
    }
    cuuint64_t dims[2] = {32, (cuuint64_t)kBlocksPerPair * 256};
    cuuint64_t strides[1] = {64};
    cuuint32_t box[2] = {32, 256};
    cuuint32_t es[2] = {1, 1};
    CUresult r = encode(&st->tmap, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, st->wblocks, dims, strides,
                        box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(MCL_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&st->n_sm, cudaDevAttrMultiProcessorCount, dev);
    int major = 0, minor = 0;
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
    cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
    if (major != 10 || minor != 3) return MCL_OK;  // kernels are built for sm_103a only
    if ((rc = cuda_check(cudaFuncSetAttribute(k_mlp_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)kSmemBytes),
                         "smem attribute")))
        return rc;
    st->ready = true;
    return MCL_OK;
}

void mlp_tc_free(mcl_map* m) {
    TcState* st = (TcState*)m->tc_aux;
    if (!st) return;
    if (st->wblocks) cudaFree(st->wblocks);
    if (st->aux) cudaFree(st->aux);
    if (st->ray_bias) cudaFree(st->ray_bias);
    if (st->abort_flag) cudaFree(st->abort_flag);
    delete st;
    m->tc_aux = nullptr;
}

bool mlp_tc_available(const mcl_map* m) {
    const TcState* st = (const TcState*)m->tc_aux;
    return st && st->ready;
}

cudaError_t mlp_tc_ray_bias(mcl_map* m, const float* gd, int n_rays, const int* n_rays_dev,
                            cudaStream_t s) {
    TcState* st = (TcState*)m->tc_aux;
    const long n = (long)n_rays * 128;
    note_launch();
    k_ray_bias<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(gd, n_rays, n_rays_dev, st->Wd,
                                                           st->bprime, st->ray_bias);
    return cudaGetLastError();
}

cudaError_t mlp_tc(mcl_map* m, int precision, const Ray* rays, const float* gd, const float* z,
                   int S, int n_rays, const int* rows_dev, float4* out, cudaStream_t s) {
    (void)gd;
    TcState* st = (TcState*)m->tc_aux;
    if (!st || !st->ready || precision != MCL_PREC_BF16) return cudaErrorNotSupported;
    Params p;
    p.rays = rays;
    p.z = z;
    p.S = S;
    p.M = (long long)n_rays * S;
    p.n_pairs = (p.M + 255) / 256;
    p.M_dev = rows_dev;
    p.bias2 = st->bias2;
    p.b_sigma = st->b_sigma;
    p.ray_bias = st->ray_bias;
    p.w_out = st->w_out;
    p.b_out0 = st->b_out[0];
    p.b_out1 = st->b_out[1];
    p.b_out2 = st->b_out[2];
    p.out = out;
    p.abort_flag = st->abort_flag;
    p.status_code = &m->status->code;
    cudaError_t e = cudaMemsetAsync(st->abort_flag, 0, sizeof(int), s);
    if (e) return e;
    const long long grid = p.n_pairs < st->n_sm ? p.n_pairs : st->n_sm;
    note_launch();
    k_mlp_tc<<<(unsigned)grid, kThreads, kSmemBytes, s>>>(st->tmap, p);
    return cudaGetLastError();
}

}  // namespace mcl
