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
// tile 1.  Every wait is bounded (see tc_ptx.cuh).
#include <cuda.h>
#include <cudaTypedefs.h>
#include <math.h>
#include <string.h>

#include <vector>

#include "internal.cuh"
#include "tc_ptx.cuh"

namespace mcl {

using namespace tc;

namespace {

constexpr int kThreads = 320;
constexpr int kStages = 4;
constexpr uint32_t kStageBytes = 256 * 32 * 2;  // one weight block [256 rows x 32 k] bf16
constexpr uint32_t kActBytes = 128 * 256 * 2;   // one tile's activations (4 K-blocks of 64)
constexpr uint32_t kGxBytes = 128 * 64 * 2;     // one tile's gamma(x)
constexpr int kLayers = 9;
constexpr int kBlocksPerPair = 64;              // weight blocks streamed per tile pair
constexpr uint32_t kSmemBytes = 1024 + 2 * kActBytes + 2 * kGxBytes + kStages * kStageBytes;
// 32-wide K chunks per layer: trunk1 reads gamma(x) (64), trunk6 reads
// [h (256), gamma(x) (64)], the others h (256).
__constant__ int c_chunks[kLayers] = {2, 8, 8, 8, 8, 10, 8, 8, 8};

struct Params {
    const Ray* rays;
    const float* z;
    int S;
    long long M;            // rows of the pass
    long long n_pairs;
    const float* bias;      // [8][256] trunk biases
    const float* w_sigma;   // [256]
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

    if (tid == 0) {
        for (int i = 0; i < kStages; ++i) {
            mbar_init(smem_u32(&bars.full[i]), 1);
            mbar_init(smem_u32(&bars.empty[i]), 1);
        }
        for (int s = 0; s < 2; ++s) {
            mbar_init(smem_u32(&bars.acc_full[s]), 1);
            mbar_init(smem_u32(&bars.a_ready[s]), 128);
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
            for (long long pr = blockIdx.x; pr < p.n_pairs && ok; pr += gridDim.x) {
                for (int b = 0; b < kBlocksPerPair; ++b, ++g) {
                    const uint32_t st = g % kStages, ph = (g / kStages) & 1u;
                    if (!mbar_wait(smem_u32(&bars.empty[st]), ph ^ 1u, abort_flag)) {
                        ok = false;
                        break;
                    }
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
            const uint32_t id256 = idesc_bf16(128, 256), id128 = idesc_bf16(128, 128);
            for (long long pr = blockIdx.x; pr < p.n_pairs && ok; pr += gridDim.x) {
                for (int l = 0; l < kLayers && ok; ++l) {
                    const int nch = c_chunks[l];
                    const uint32_t idesc = (l == 8) ? id128 : id256;
                    for (int c = 0; c < nch && ok; ++c) {
                        const uint32_t st = g % kStages, ph = (g / kStages) & 1u;
                        const bool new_block = (l < 8) || ((c & 1) == 0);
                        if (new_block) {
                            if (!mbar_wait(smem_u32(&bars.full[st]), ph, abort_flag)) {
                                ok = false;
                                break;
                            }
                            tc_fence_after();
                        }
                        const uint32_t boff = (l == 8 && (c & 1)) ? 8192u : 0u;
                        for (int s = 0; s < 2; ++s) {
                            if (c == 0) {
                                if (!mbar_wait(smem_u32(&bars.a_ready[s]), rdy_ph[s], abort_flag)) {
                                    ok = false;
                                    break;
                                }
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
                                    smem_desc(s_ring + st * kStageBytes + boff + kk * 32, 512, kLayoutSw64);
                                mma_bf16(tmem + s * 256, ad, bd, idesc, (c | kk) ? 1u : 0u);
                            }
                            if (c == nch - 1) mma_commit(smem_u32(&bars.acc_full[s]));
                        }
                        if (!ok) break;
                        const bool block_done = (l < 8) || ((c & 1) == 1);
                        if (block_done) {
                            mma_commit(smem_u32(&bars.empty[st]));
                            ++g;
                        }
                    }
                }
            }
            if (!ok) record_abort(p);
            // all issued MMAs complete before TMEM is released
            mma_commit(smem_u32(&bars.drain));
            mbar_wait(smem_u32(&bars.drain), 0, nullptr);
        }
    } else {
        // ------------------------------------------------ prologue / epilogues
        const int slot = (warp - 2) >> 2;                 // warps 2-5 -> 0, 6-9 -> 1
        const int quad = warp & 3;                        // TMEM lane quadrant of this warp
        const uint32_t r = quad * 32 + lane;              // row within the tile
        const uint32_t t_acc = tmem + ((uint32_t)(quad * 32) << 16) + slot * 256;
        const uint32_t a_base = s_act + slot * kActBytes;
        const uint32_t g_base = s_gx + slot * kGxBytes;
        const uint32_t bar_ready = smem_u32(&bars.a_ready[slot]);
        const uint32_t bar_acc = smem_u32(&bars.acc_full[slot]);
        uint32_t acc_ph = 0;
        bool ok = true;
        for (long long pr = blockIdx.x; pr < p.n_pairs && ok; pr += gridDim.x) {
            const long long grow = pr * 256 + slot * 128 + r;
            const bool valid = grow < p.M;
            const long long ray = valid ? grow / p.S : 0;
            // ---- prologue: gamma(x) of this row
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
            for (int l = 0; l < kLayers && ok; ++l) {
                if (!mbar_wait(bar_acc, acc_ph, abort_flag)) {
                    ok = false;
                    break;
                }
                acc_ph ^= 1u;
                tc_fence_after();
                if (l < 8) {
                    const float* bias = p.bias + l * 256;
#pragma unroll 1
                    for (int c32 = 0; c32 < 8; ++c32) {
                        uint32_t v[32];
                        tmem_ld32(t_acc + c32 * 32, v);
                        tmem_ld_wait();
                        float h[32];
#pragma unroll
                        for (int i = 0; i < 32; ++i)
                            h[i] = fmaxf(__uint_as_float(v[i]) + __ldg(bias + c32 * 32 + i), 0.0f);
                        if (l == 7) {
#pragma unroll
                            for (int i = 0; i < 32; ++i)
                                sigma = fmaf(h[i], __ldg(p.w_sigma + c32 * 32 + i), sigma);
                        }
                        uint32_t pk[16];
#pragma unroll
                        for (int i = 0; i < 16; ++i) pk[i] = pack_bf16x2(h[2 * i], h[2 * i + 1]);
                        const uint32_t blk = a_base + (c32 >> 1) * 16384;
                        const uint32_t j0 = (c32 & 1) * 4;
#pragma unroll
                        for (int q = 0; q < 4; ++q)
                            st_shared_v4(blk + sw128_offset(r, j0 + q), pk[4 * q], pk[4 * q + 1],
                                         pk[4 * q + 2], pk[4 * q + 3]);
                    }
                    fence_proxy_async_smem();
                    tc_fence_before();
                    mbar_arrive(bar_ready);
                } else {
                    const float* rb = p.ray_bias + ray * 128;
                    float o0 = 0.f, o1 = 0.f, o2 = 0.f;
#pragma unroll 1
                    for (int c32 = 0; c32 < 4; ++c32) {
                        uint32_t v[32];
                        tmem_ld32(t_acc + c32 * 32, v);
                        tmem_ld_wait();
#pragma unroll
                        for (int i = 0; i < 32; ++i) {
                            const int col = c32 * 32 + i;
                            const float hr = fmaxf(__uint_as_float(v[i]) + __ldg(rb + col), 0.0f);
                            o0 = fmaf(hr, __ldg(p.w_out + col), o0);
                            o1 = fmaf(hr, __ldg(p.w_out + 128 + col), o1);
                            o2 = fmaf(hr, __ldg(p.w_out + 256 + col), o2);
                        }
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
__global__ void k_ray_bias(const float* __restrict__ gd, int n_rays, const float* __restrict__ Wd,
                           const float* __restrict__ bprime, float* __restrict__ out) {
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long)n_rays * 128) return;
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
    const float* bias = nullptr;
    const float* w_sigma = nullptr;
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
    // RGB hidden (folded), N = 128: two K chunks per block (rows 0..127, 128..255)
    for (int k0 = 0; k0 < kWidth; k0 += 64, ++b) {
        auto get = [&](int n, int k) -> double { return Wfold[(size_t)n * kWidth + k]; };
        put_chunk(b, 0, 128, get, k0);
        put_chunk(b, 128, 128, get, k0 + 32);
    }
    if (b != kBlocksPerPair) return fail(MCL_ERR_UNSUPPORTED, "internal: weight block count %d", b);
    // ---- fp32 aux: trunk biases [8][256], w_sigma [256], w_out [3][128],
    //      W_d [128][27], b' [128]
    std::vector<float> aux;
    const size_t o_bias = aux.size();
    for (int l = 0; l < kDepth; ++l) aux.insert(aux.end(), bp[l], bp[l] + kWidth);
    const size_t o_wsig = aux.size();
    aux.insert(aux.end(), Wp[8], Wp[8] + kWidth);
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
    st->bias = st->aux + o_bias;
    st->w_sigma = st->aux + o_wsig;
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

cudaError_t mlp_tc_ray_bias(mcl_map* m, const float* gd, int n_rays, cudaStream_t s) {
    TcState* st = (TcState*)m->tc_aux;
    const long n = (long)n_rays * 128;
    note_launch();
    k_ray_bias<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(gd, n_rays, st->Wd, st->bprime,
                                                           st->ray_bias);
    return cudaGetLastError();
}

cudaError_t mlp_tc(mcl_map* m, int precision, const Ray* rays, const float* gd, const float* z,
                   int S, int n_rays, float4* out, cudaStream_t s) {
    (void)gd;
    TcState* st = (TcState*)m->tc_aux;
    if (!st || !st->ready || precision != MCL_PREC_BF16) return cudaErrorNotSupported;
    Params p;
    p.rays = rays;
    p.z = z;
    p.S = S;
    p.M = (long long)n_rays * S;
    p.n_pairs = (p.M + 255) / 256;
    p.bias = st->bias;
    p.w_sigma = st->w_sigma;
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
