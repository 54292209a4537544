// mlp_tc.cu -- the NeRF MLP on the 5th-generation tensor cores (tcgen05,
// FP32 accumulation in TMEM), fused across all layers, in two operand
// forms: BF16, and FP8 (E4M3 with calibrated scales).
//
// One persistent CTA per SM walks over pairs of 128-row tiles (rows are the
// samples of the pass, row = ray * S + k).  Per pair:
//   prologue   x = o + z d, gamma(x) (63 -> 64) into shared memory;
//   9 layers   trunk 1..8 (ReLU; gamma(x) re-enters layer 6 through the skip),
//              then the RGB hidden layer with the feature layer folded in
//              (W' = W_rgb_hidden[:, :256] W_feature, computed in FP64 when
//              the map is loaded: the feature layer has no activation) and
//              the density head as its row 128;
//   epilogues  TMEM -> registers, bias + ReLU (and the FP8 scales), back
//              into the same shared-memory tile as the next layer's A
//              operand; after the last MMA the RGB output layer (128 -> 3,
//              sigmoid) with gamma(d)'s contribution added as a per-ray bias.
// Warp roles: warp 0 streams weight blocks (256 rows x 64 bytes, stored in
// global memory already in the 64-byte-swizzled shared-memory layout) with
// contiguous bulk copies through a ring; warp 1 allocates TMEM and issues
// the MMAs (M = 128, N = 256, 32 bytes of K per instruction); warp 2 (the
// gate) waits on the ring and activation barriers and releases warp 1
// through a named barrier, so that the issuing thread makes no shared-memory
// access between MMAs; the other warps run prologue and epilogues, 4 or 8
// per tile, one warp per TMEM lane quadrant and column half, one thread per
// row.  The two tiles run staggered: each part of a layer's weight blocks
// that the ring holds (the whole layer in FP8, half of it in BF16) is run
// by tile 0 and then by tile 1 on the resident blocks, so each tile's
// epilogue overlaps the other's MMAs (a lockstep schedule, each block
// serving both tiles at once, is the alternative the autotuner measures).
// The next work unit's gamma(x) is written while the last layers run, and
// the last accumulator is read out of TMEM first, so that the next unit's
// first MMAs overlap the RGB head.  Every wait is bounded (see tc_ptx.cuh).
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_fp8.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "internal.cuh"
#include "tc_ptx.cuh"


namespace mcl {

using namespace tc;

namespace {

constexpr uint32_t kStageBytes = 256 * 64;      // one weight block: 256 rows x 64 bytes
constexpr uint32_t kGxBytes = 128 * 128;        // one tile's gamma(x): 128-byte rows
constexpr int kLayers = 9;
constexpr int kMaxStages = 8;

// Operand form of the MMAs.  BF16: weight blocks [256 rows x 32 k], 4-stage
// ring, activations 128 x 256 BF16 (64 KB per tile).  FP8 (E4M3 with
// per-layer activation scales and per-layer weight scales): weight blocks
// [256 rows x 64 k], 8-stage ring, activations 128 x 256 bytes (32 KB).
// Both fill 225 KB of shared memory.
template <bool F8>
struct Form {
    static constexpr uint32_t kActBytes = F8 ? 128 * 256 : 128 * 256 * 2;
    static constexpr int kStages = F8 ? 8 : 4;
    static constexpr int kBlocks = F8 ? 34 : 68;     // weight blocks per tile pair
    static constexpr int kActChunks = F8 ? 4 : 8;    // K chunks of a 256-wide activation
    static constexpr uint32_t kSmemBytes = 1024 + 2 * kActBytes + 2 * kGxBytes + kStages * kStageBytes;
};
static_assert(Form<false>::kSmemBytes <= 232448 && Form<true>::kSmemBytes <= 232448, "smem");

// Kernel variant: operand form, epilogue warps per tile (4: one per TMEM lane
// quadrant, each thread a whole row; 8: two per quadrant, each thread half a
// row), and the tile schedule (lockstep: each weight block serves both
// tiles at once; staggered: tile 1 runs each part of a layer -- as many
// blocks as the ring holds: the whole layer in FP8's 8-stage ring, four of
// BF16's 8 or 10 -- after tile 0 on the same resident blocks, so each tile's
// epilogue overlaps the other's MMAs).  The autotuner picks among them.
template <bool F8, int EPIW, bool STAG>
struct Variant {
    static_assert(EPIW == 4 || EPIW == 8, "epilogue warps");
    static constexpr int kEpiThreads = 32 * EPIW;
    static constexpr int kThreads = 96 + 2 * kEpiThreads;   // + TMA, MMA and gate warps
};

// K chunks (one weight block each) per layer: trunk1 reads gamma(x) (64),
// trunk6 reads [h (256), gamma(x) (64)], the others h (256).  The last
// layer has N = 144: rows 0..127 are the RGB hidden layer (feature layer
// folded in), row 128 the density head, so sigma_raw arrives as accumulator
// column 128 of the last MMA.
__host__ __device__ constexpr int layer_chunks(bool f8, int l) {
    return (l == 0 ? 2 : l == 5 ? 10 : 8) >> (f8 ? 1 : 0);
}

struct EpiConsts {
    uint32_t bias2[8][128];   // BF16: trunk biases as BF16 pairs
    float beta[8][256];       // FP8: epilogue offset per column
    float alpha_last[128];    // FP8: dequantisation of the RGB hidden layer
    float w_out[3][128];      // RGB output layer
};

struct Params {
    const uint8_t* wblocks; // weight blocks of the form, pre-swizzled, in consumption order
    const Ray* rays;
    const float* z;
    int S;
    long long M;            // rows of the pass (upper bound when M_dev is set)
    long long n_pairs;
    const int* M_dev;       // optional: rows of the pass from device memory
    float alpha[8];         // FP8: epilogue scale per trunk layer
    const float* beta_g;    // FP8: [8][256] epilogue offset per column (global copy)
    float alpha_sigma;      // FP8: dequantisation of the density head
    float s_gx;             // FP8: scale of gamma(x)
    float b_sigma;
    const float* ray_bias;  // [n_rays][128]
    float b_out0, b_out1, b_out2;
    float4* out;
    int* abort_flag;        // per-launch: set on a timed-out wait
    int* status_code;       // map status word
    unsigned long long wait_ns;  // limit of the bounded waits of k_mlp_tc
    int hold_weights;       // failure-injection hook (k_mlp_tc): the weight
                            // stream issues no copies, so the waits expire
    // Fused ray epilogues (tiles hold whole rays: 128 % S == 0).
    //   fuse 0: write (sigma_raw, rgb) of every row to out;
    //   fuse 1: also the first pass of the hierarchical sampler: Eq. 1
    //           weights of each ray's S samples -> nf_out inverse-CDF samples
    //           into z_out [rays, nf_out];
    //   fuse 2: the last pass: merge each ray's S samples with the S1 samples
    //           of the first pass (z_first, out_first [rays, S1]; S1 = 0: this
    //           pass only), Eq. 1 composite, Eq. 5 / F and E against obs; out
    //           is not written.
    int fuse;
    int nf_out;
    float* z_out;
    const float* z_first;
    const float4* out_first;
    int S1;
    float eq5_alpha, tau;   // Eq. 5 threshold, lower bound of F
    int use_rej;
    const float4* obs;      // [rays] observed level-image colour (NaN: none), or NULL
    float* e_ray;           // [rays] E * F (with obs)
    float* rgb_out;         // [rays, 3] (optional)
    float* E_out;           // [rays] (optional)
    float* F_out;
    float* zt_out;
    float* zo_out;
    // Per-column constants of the epilogues, carried in the parameter block
    // (the constant bank): every thread of a warp reads the same column's
    // value, and a constant-bank read does not go through the L1 that the
    // 225 KB shared-memory carve-out leaves nearly empty.
    EpiConsts ec;
};

struct __align__(8) Bars {
    uint64_t full[kMaxStages];
    uint64_t empty[kMaxStages];
    uint64_t acc_full[2];
    uint64_t a_ready[2];
    uint64_t epi[2];        // the 128 row threads of a tile meet in the fused ray epilogues
    uint64_t drain;
    uint32_t tmem_base;
};

__device__ __forceinline__ void record_abort(const Params& p) {
    atomicCAS(p.status_code, 0, MCL_ERR_TIMEOUT);
}

// Half H of gamma(x) of one row: values 32 H .. 32 H + 31 of [x, sin(2^k x),
// cos(2^k x) (k = 0..9, each on the 3 axes), 0].  sin / cos of 2^k x by angle
// doubling from an accurate sincos of 2^k0 x (k0 = 0, or 4 for the upper
// half; error ~2^(k - k0) ulp, far below the operand precision).
template <int H>
__device__ __forceinline__ void pe_half(const float x[3], float (&v)[32]) {
    constexpr int k0 = H ? 4 : 0;
    if (H == 0) { v[0] = x[0]; v[1] = x[1]; v[2] = x[2]; }
    if (H == 1) v[31] = 0.0f;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        float s, cs;
        sincosf(H ? 16.0f * x[c] : x[c], &s, &cs);
#pragma unroll
        for (int k = k0; k < kLxyz; ++k) {
            const int is = 3 + 6 * k + c - 32 * H, ic = 6 + 6 * k + c - 32 * H;
            if (is >= 0 && is < 32) v[is] = s;
            if (ic >= 0 && ic < 32) v[ic] = cs;
            const float s2 = 2.0f * s * cs;
            const float c2 = (cs - s) * (cs + s);
            s = s2;
            cs = c2;
        }
    }
}

// 32 accumulator columns of one row -> relu(acc + bias) as BF16 -> four
// 16-byte chunks (j0 .. j0+3) of the row in a 128-byte-swizzled K-block.
// bias: 16 BF16 pairs in the parameter block.
__device__ __forceinline__ void epi_chunk_store(const uint32_t (&v)[32], const uint32_t* bias,
                                                uint32_t blk, uint32_t r, uint32_t j0) {
    const uint32_t one2 = 0x3F803F80u;  // (1.0, 1.0) in BF16
    uint32_t pk[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        const uint32_t a = pack_bf16x2(__uint_as_float(v[2 * i]), __uint_as_float(v[2 * i + 1]));
        uint32_t h;
        asm("fma.rn.relu.bf16x2 %0, %1, %2, %3;" : "=r"(h) : "r"(a), "r"(one2), "r"(bias[i]));
        pk[i] = h;
    }
#pragma unroll
    for (int q = 0; q < 4; ++q)
        st_shared_v4(blk + sw128_offset(r, j0 + q), pk[4 * q], pk[4 * q + 1], pk[4 * q + 2],
                     pk[4 * q + 3]);
}

// FP8 form: 32 accumulator columns -> relu(acc alpha + beta) (the next
// layer's activation scale folded into alpha, beta: 32 values, in global
// memory (kGlobal: eight 16-byte loads) or in the parameter block) as E4M3
// -> two 16-byte chunks (j0, j0+1) of the row in a 128-byte-swizzled K-block.
template <bool kGlobal>
__device__ __forceinline__ void epi_chunk_store_f8(const uint32_t (&v)[32], float alpha,
                                                   const float* beta, uint32_t blk, uint32_t r,
                                                   uint32_t j0) {
    uint32_t pk[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        float4 b;
        if constexpr (kGlobal) b = __ldg(reinterpret_cast<const float4*>(beta) + q);
        else b = make_float4(beta[4 * q], beta[4 * q + 1], beta[4 * q + 2], beta[4 * q + 3]);
        pk[q] = pack_e4m3x4_relu(fmaf(__uint_as_float(v[4 * q + 0]), alpha, b.x),
                                 fmaf(__uint_as_float(v[4 * q + 1]), alpha, b.y),
                                 fmaf(__uint_as_float(v[4 * q + 2]), alpha, b.z),
                                 fmaf(__uint_as_float(v[4 * q + 3]), alpha, b.w));
    }
    st_shared_v4(blk + sw128_offset(r, j0), pk[0], pk[1], pk[2], pk[3]);
    st_shared_v4(blk + sw128_offset(r, j0 + 1), pk[4], pk[5], pk[6], pk[7]);
}

// One 32-column group of the last layer: h = relu(acc (* alpha) + b_ray),
// then the 128 -> 3 output layer as running dot products (wo [3][128] and
// al [128]: the parameter block; rb4: the ray's bias in global memory).
template <bool F8>
__device__ __forceinline__ void rgb_group(const uint32_t (&v)[32], const float4* rb4,
                                          const float* wo, const float* al, int c32,
                                          float& o0, float& o1, float& o2) {
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const float4 b = __ldg(rb4 + c32 * 8 + q);
        const int c = c32 * 32 + 4 * q;
        float a0 = __uint_as_float(v[4 * q + 0]), a1 = __uint_as_float(v[4 * q + 1]);
        float a2 = __uint_as_float(v[4 * q + 2]), a3 = __uint_as_float(v[4 * q + 3]);
        if constexpr (F8) {
            a0 *= al[c]; a1 *= al[c + 1]; a2 *= al[c + 2]; a3 *= al[c + 3];
        }
        const float h0 = fmaxf(a0 + b.x, 0.0f);
        const float h1 = fmaxf(a1 + b.y, 0.0f);
        const float h2 = fmaxf(a2 + b.z, 0.0f);
        const float h3 = fmaxf(a3 + b.w, 0.0f);
        o0 = fmaf(h0, wo[c], fmaf(h1, wo[c + 1], fmaf(h2, wo[c + 2], fmaf(h3, wo[c + 3], o0))));
        o1 = fmaf(h0, wo[128 + c], fmaf(h1, wo[129 + c], fmaf(h2, wo[130 + c], fmaf(h3, wo[131 + c], o1))));
        o2 = fmaf(h0, wo[256 + c], fmaf(h1, wo[257 + c], fmaf(h2, wo[258 + c], fmaf(h3, wo[259 + c], o2))));
    }
}


// ---------------------------------------------------------------------------
// Fused ray epilogues.  After the last layer, the 128 threads that own the
// rows of a tile (one row each) work on the tile's R = 128 / S whole rays:
// they stage samples in shared memory (the first 16 KB of the tile's
// activation buffer, free between the last layer's MMA and the next work
// unit's first epilogue), meet at the tile's `epi` mbarrier (EpiSync), and
// one warp per ray runs the
// sequential parts of Eq. 1 as warp-shuffle scans: each lane takes a
// contiguous chunk of the ray's samples, the transmittance entering a chunk
// is the exclusive product scan of the chunks' transmittances, and running
// weight sums are exclusive sum scans.
// ---------------------------------------------------------------------------

// The tile's 128 row threads meet at the tile's `epi` mbarrier: every thread
// arrives, then waits for the phase with the kernel's bounded wait, so a
// launch that aborts cannot leave the others waiting.
struct EpiSync {
    uint32_t bar;
    uint32_t ph;
    volatile int* err;
    unsigned long long limit;
    // returns false if the wait gave up (abort or time limit)
    __device__ __forceinline__ bool sync() {
        mbar_arrive(bar);
        const bool r = mbar_wait(bar, ph, err, limit);
        ph ^= 1u;
        return r;
    }
};

__device__ __forceinline__ float warp_excl_prod(float v, int lane) {
    float x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const float t = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x *= t;
    }
    const float e = __shfl_up_sync(0xffffffffu, x, 1);
    return lane == 0 ? 1.0f : e;
}

__device__ __forceinline__ float warp_incl_sum(float v, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const float t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// cnt[t] += the number of the warp's values <= uu[t], the values being
// vals[0 .. C-1] of every lane: each lane's values are broadcast in turn.
template <int C>
__device__ __forceinline__ void warp_count_le(const float (&vals)[5], const float (&uu)[4],
                                              int (&cnt)[4]) {
#pragma unroll 4
    for (int src = 0; src < 32; ++src) {
#pragma unroll
        for (int i = 0; i < C; ++i) {
            const float e = __shfl_sync(0xffffffffu, vals[i], src);
#pragma unroll
            for (int t = 0; t < 4; ++t) cnt[t] += e <= uu[t] ? 1 : 0;
        }
    }
}

// Staging in the tile's activation buffer.  Warp q (the warp of TMEM lane
// quadrant q) rewrites only its own rows in the next unit's first epilogue:
// bytes [q 4096, +4096) of each 16 KB K-block.  Ray g of a tile (at most 4)
// is composited by warp g, and its samples are staged in that warp's part of
// K-block 0, so the other warps never wait for the compositing warp: once
// the staging is complete they go on to the next layer.  Data that every
// thread reads (this pass's z of the whole tile, the first pass's z) sits in
// K-block 1 and is dead after the second barrier.
__device__ __forceinline__ float* warp_part(float* scr, int q) {
    return scr + q * 1024;   // 4096 bytes
}

// First pass of the hierarchical sampler, fused: Eq. 1 weights w_k of each
// ray's S samples, pdf over the interior bins (between midpoints of
// consecutive samples) proportional to w_1 .. w_{S-2} + 1e-5, inverse CDF at
// u_j = j / (nf - 1) (bin: first CDF entry strictly greater than u_j, linear
// interpolation inside it).  In two steps, so that the arithmetic runs off
// the tensor pipe's critical path:
//   tail_importance_stage (every row thread, right after the last layer):
//     the rows' (z, sigma_raw) meet in shared memory at one barrier and the
//     compositing warp of each ray copies its contiguous chunk of the ray
//     (lane l: samples l c .. l c + c - 1, c = S / 32, and the next z) into
//     registers; the staging area may then be overwritten;
//   tail_importance_finish (the compositing warps, once the next unit's
//     first-layer epilogue has been signalled): the rest, from registers
//     and warp shuffles.
struct TailImp {
    float zc[5];      // z of the chunk's samples and of the sample after it
    float sc[4];      // sigma_raw of the chunk's samples
    float dn;         // |d| of the ray
    long long ray;    // -1: this warp composites no ray
};

// Row thread r holds (z, sigma_raw) of row r.  R = 128 / S <= 4 rays per
// tile; one barrier.  Returns false if the barrier's wait gave up.
__device__ __forceinline__ bool tail_importance_stage(const Params& p, EpiSync& es, float* scr, int r,
                                                      int lane, int quad, long long ray0,
                                                      long long n_rays, float z, float sg, float dn_row,
                                                      TailImp& ti) {
    const int S = p.S, R = 128 / S;
    {
        // ray g's part: z [S], sigma [S], |d|
        const int g = r / S, k = r - g * S;
        float* part = warp_part(scr, g);
        part[k] = z;
        part[S + k] = sg;
        if (k == 0) part[2 * S] = dn_row;
    }
    ti.ray = -1;
    if (!es.sync()) return false;
    if (quad >= R || ray0 + quad >= n_rays) return true;
    const float* part = warp_part(scr, quad);
    const int c = S >> 5;   // S = 32, 64, 128
    const int k0 = lane * c;
#pragma unroll
    for (int i = 0; i < 5; ++i) ti.zc[i] = (i <= c && k0 + i < S) ? part[k0 + i] : 0.0f;
#pragma unroll
    for (int i = 0; i < 4; ++i) ti.sc[i] = i < c ? part[S + k0 + i] : 0.0f;
    ti.dn = part[2 * S];
    ti.ray = ray0 + quad;
    // the loads above are complete before any lane of this warp rewrites
    // its rows of the buffer (the next unit's first epilogue)
    __syncwarp();
    return true;
}

// Entry k of values held c per lane (entry k in lane k / c, element k % c);
// every lane takes part, each with its own k.
__device__ __forceinline__ float warp_entry(const float (&v)[5], int c, int k) {
    const int lc = c == 4 ? 2 : c - 1;
    const int src = k >> lc, e = k & (c - 1);
    float x = __shfl_sync(0xffffffffu, v[0], src);
    if (c >= 2) {
        const float x1 = __shfl_sync(0xffffffffu, v[1], src);
        if (e == 1) x = x1;
    }
    if (c == 4) {
        const float x2 = __shfl_sync(0xffffffffu, v[2], src);
        const float x3 = __shfl_sync(0xffffffffu, v[3], src);
        if (e == 2) x = x2;
        if (e == 3) x = x3;
    }
    return x;
}

// The compositing warp of a ray (ti.ray >= 0), all 32 lanes.  part: the
// ray's staged part, still intact (the tail finishes right after the stage):
// the CDF goes there too and the interpolation reads it and z from shared
// memory; NULL (deferred: the part may have been overwritten): they come
// from the lanes' registers through warp shuffles.
__device__ __forceinline__ void tail_importance_finish(const Params& p, const TailImp& ti, int lane,
                                                       float* part) {
    const int S = p.S, nf = p.nf_out, ne = S - 1;
    const int c = S >> 5;
    const int k0 = lane * c;
    const float dn = ti.dn;
    float wl[4];
    float Tl = 1.0f;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int k = k0 + i;
        wl[i] = 0.0f;
        if (i < c) {
            const float delta = (k < S - 1) ? (ti.zc[i + 1] - ti.zc[i]) * dn : 1e10f;
            const float a = 1.0f - expf(-fmaxf(ti.sc[i], 0.0f) * delta);
            wl[i] = Tl * a;
            Tl *= 1.0f - a;
        }
    }
    const float T0 = warp_excl_prod(Tl, lane);
    float pl[4];
    float psum = 0.0f;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int k = k0 + i;
        pl[i] = (i < c && k >= 1 && k <= S - 2) ? T0 * wl[i] + 1e-5f : 0.0f;
        psum += pl[i];
    }
    const float incl = warp_incl_sum(psum, lane);
    const float tot = __shfl_sync(0xffffffffu, incl, 31);
    float run = incl - psum;
    // CDF entries 0 .. ne - 1 (entry 0 is 0), c per lane; +inf past the last
    float ce[5];
#pragma unroll
    for (int i = 0; i < 5; ++i) ce[i] = __int_as_float(0x7f800000);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int k = k0 + i;
        if (i < c && k >= 1 && k <= S - 2) {
            run += pl[i];
            ce[i] = run / tot;
        } else if (i < c && k == 0) {
            ce[i] = 0.0f;
        }
    }
    // Lane l: outputs j = d l .. d l + d - 1.  The bin of u_j, the first
    // entry with cdf > u_j, is the number of entries <= u_j (the CDF does
    // not decrease): each lane's entries are broadcast in turn and every
    // lane counts them against its own u_j.
    const int d = (nf + 31) >> 5;   // <= 4 (the launch checks nf <= 128)
    float uu[4];
    int cnt[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        const int j = lane * d + t;
        uu[t] = (nf > 1 && j < nf) ? (float)j / (float)(nf - 1) : 0.0f;
        cnt[t] = 0;
    }
    if (c == 1) warp_count_le<1>(ce, uu, cnt);
    else if (c == 2) warp_count_le<2>(ce, uu, cnt);
    else warp_count_le<4>(ce, uu, cnt);
    float* cdf = part ? part + 2 * S + 1 : nullptr;   // [ne] after z, sigma, |d|
    if (part) {
#pragma unroll
        for (int i = 0; i < 4; ++i)
            if (i < c && k0 + i < ne) cdf[k0 + i] = ce[i];
        __syncwarp();
    }
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        if (t >= d) break;   // (d is the same in every lane)
        const int j = lane * d + t;
        const float u = uu[t];
        const int idx = cnt[t];
        const int below = idx - 1 < 0 ? 0 : idx - 1;
        const int above = idx > ne - 1 ? ne - 1 : idx;
        float cb, ca, zb0, zb1, za0, za1;
        if (part) {
            cb = cdf[below]; ca = cdf[above];
            zb0 = part[below]; zb1 = part[below + 1];
            za0 = part[above]; za1 = part[above + 1];
        } else {
            cb = warp_entry(ce, c, below); ca = warp_entry(ce, c, above);
            zb0 = warp_entry(ti.zc, c, below); zb1 = warp_entry(ti.zc, c, below + 1);
            za0 = warp_entry(ti.zc, c, above); za1 = warp_entry(ti.zc, c, above + 1);
        }
        float denom = ca - cb;
        if (denom < 1e-5f) denom = 1.0f;
        const float tt = (u - cb) / denom;
        const float eb = 0.5f * (zb0 + zb1);
        const float ea = 0.5f * (za0 + za1);
        if (j < nf) p.z_out[ti.ray * nf + j] = eb + tt * (ea - eb);
    }
}

// Last pass, fused: merge each ray's S samples of this pass with the S1
// samples of the first pass (both sorted; equal z take the first pass's
// sample first), Eq. 1 composite over the merged samples (delta_last =
// 1e10), Eq. 5 on the running weight sum, F of Eq. 6 and the photometric E
// against the ray's observed colour.  Row thread r holds (z, sigma_raw, rgb)
// of row r and has prefetched first-pass samples q = r and r + 128 of the
// tile (fz / fo) and, in warp g, the observed colour of ray g (ob).  R =
// 128 / S <= 4 rays per tile, at most 204 merged samples per ray; two
// barriers.
__device__ __forceinline__ bool tail_final(const Params& p, EpiSync& es, float* scr, int r,
                                           int lane, int quad, long long ray0, long long n_rays,
                                           float z, float4 v, float dn_row, const float (&fz)[2],
                                           const float4 (&fo)[2], const float4& ob) {
    const int S = p.S, S1 = p.S1, R = 128 / S, n = S + S1;
    float* shared_z = scr + 4096;       // K-block 1: read by every thread
    float* zB = shared_z;               // [128] this pass
    float* dns = shared_z + 128;        // [4] |d| of each ray
    float* zA = shared_z + 132;         // [R * S1] first pass
    zB[r] = z;
    if (r % S == 0) dns[r / S] = dn_row;
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const int q = r + 128 * i;
        if (q < R * S1) zA[q] = fz[i];
    }
    if (!es.sync()) return false;
    {
        // this pass's sample j of ray g: j + (first-pass samples with z <= it)
        const int g = r / S, j = r - g * S;
        const float* a = zA + g * S1;
        int lo = 0, hi = S1;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (a[mid] <= z) lo = mid + 1;
            else hi = mid;
        }
        float* m = warp_part(scr, g);   // merged [n] z, sigma (then alpha), r, g, b
        const int k = j + lo;
        m[k] = z; m[n + k] = v.x; m[2 * n + k] = v.y; m[3 * n + k] = v.z; m[4 * n + k] = v.w;
    }
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        // first-pass sample q of ray g: i + (this pass's samples with z < it)
        const int q = r + 128 * i;
        if (q < R * S1) {
            const int g = q / S1, ii = q - g * S1;
            const float* b = zB + g * S;
            const float zq = fz[i];
            int lo = 0, hi = S;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (b[mid] < zq) lo = mid + 1;
                else hi = mid;
            }
            float* m = warp_part(scr, g);
            const int k = ii + lo;
            m[k] = zq; m[n + k] = fo[i].x; m[2 * n + k] = fo[i].y; m[3 * n + k] = fo[i].z;
            m[4 * n + k] = fo[i].w;
        }
    }
    const float dn = dns[quad < R ? quad : 0];
    if (!es.sync()) return false;
    if (quad >= R) return true;
    const long long ray = ray0 + quad;
    if (ray >= n_rays) return true;
    float* m = warp_part(scr, quad);
    const float* z_ = m;
    float* s_ = m + n;
    const float* r_ = m + 2 * n;
    const float* g_ = m + 3 * n;
    const float* b_ = m + 4 * n;
    const int c = (n + 31) >> 5;
    const int k0 = min(lane * c, n), k1 = min(k0 + c, n);
    // chunk pass 1: alpha (stored over sigma), local transmittance, colour
    // and weight sums of the chunk
    float Tl = 1.0f, cr = 0.0f, cg = 0.0f, cb = 0.0f, wsum = 0.0f;
    for (int k = k0; k < k1; ++k) {
        const float delta = (k < n - 1) ? (z_[k + 1] - z_[k]) * dn : 1e10f;
        const float a = 1.0f - expf(-fmaxf(s_[k], 0.0f) * delta);
        const float w = Tl * a;
        cr += w * r_[k]; cg += w * g_[k]; cb += w * b_[k];
        wsum += w;
        Tl *= 1.0f - a;
        s_[k] = a;
    }
    const float T0 = warp_excl_prod(Tl, lane);
    const float Cr = warp_sum(T0 * cr), Cg = warp_sum(T0 * cg), Cb = warp_sum(T0 * cb);
    const float incl = warp_incl_sum(T0 * wsum, lane);
    const float W0 = incl - T0 * wsum;
    // chunk pass 2: running weight sum W_k, Eq. 5 decisions
    int kt = n, ko = -1;
    float Tl2 = 1.0f, wc = 0.0f;
    for (int k = k0; k < k1; ++k) {
        const float w = Tl2 * s_[k];
        wc += w;
        Tl2 *= 1.0f - s_[k];
        const float Wk = W0 + T0 * wc;
        if (kt == n && Wk >= p.eq5_alpha) kt = k;
        if (Wk <= 1.0f - p.eq5_alpha) ko = k;
    }
    kt = __reduce_min_sync(0xffffffffu, kt);
    ko = __reduce_max_sync(0xffffffffu, ko);
    if (lane == 0) {
        const float zt = kt < n ? z_[kt] : z_[0];
        const float zo = ko >= 0 ? z_[ko] : z_[0];
        const float F = p.use_rej ? fmaxf(zo - zt, p.tau) : 1.0f;
        if (p.rgb_out) {
            p.rgb_out[3 * ray] = Cr; p.rgb_out[3 * ray + 1] = Cg; p.rgb_out[3 * ray + 2] = Cb;
        }
        if (p.F_out) p.F_out[ray] = F;
        if (p.zt_out) p.zt_out[ray] = zt;
        if (p.zo_out) p.zo_out[ray] = zo;
        if (p.obs) {
            const float e0 = ob.x - Cr, e1 = ob.y - Cg, e2 = ob.z - Cb;
            const float E = isfinite(dn) ? e0 * e0 + e1 * e1 + e2 * e2 : __int_as_float(0x7fc00000);
            if (p.E_out) p.E_out[ray] = E;
            p.e_ray[ray] = E * F;
        }
    }
    __syncwarp();
    return true;
}

// Operand writes of one thread (activations or gamma(x)) and its TMEM reads
// are done: make the writes visible to the tensor core and signal the MMA
// issuer.  Single CTA: every epilogue thread arrives on the local barrier.
// CTA pair: the MMAs are issued by the even CTA, whose barrier counts one
// arrival per epilogue warp of both CTAs (cluster scope).
template <bool PAIR>
__device__ __forceinline__ void signal_ready(uint32_t bar, int lane) {
    fence_proxy_async_smem();
    tc_fence_before();
    if constexpr (PAIR) {
        __syncwarp();
        if (lane == 0) mbar_arrive_cluster(bar);
    } else {
        mbar_arrive(bar);
    }
}

// Prologue and epilogues of the epilogue warps (warps warp0 .. warp0 + 2 EPIW - 1)
// over the CTA's work units: unit u holds rows u unit_rows + row_base ..
// +255 of the pass, tile slot s its rows + 128 s .. +127.  Per unit: gamma(x)
// into the slot's buffer, then per layer TMEM -> bias + ReLU (and the FP8
// scales) -> the next layer's A operand, and after the last layer the RGB
// output layer and the density.  PAIR: bar_ready* are shared::cluster
// addresses of the even CTA's barriers.  FUSE (0, 1, 2): the fused ray
// epilogue of the pass (Params::fuse); instantiations without it carry no
// code or registers for it.
template <bool F8, int EPIW, bool PAIR, int FUSE = 0>
__device__ __forceinline__ void epilogue_warps(const Params& p, int warp, int warp0, int lane, uint32_t tmem,
                                               uint32_t s_act, uint32_t s_gx, uint32_t bar_ready0,
                                               uint32_t bar_ready1, uint32_t bar_acc0,
                                               uint32_t bar_acc1, long long M, long long u0,
                                               long long du, long long n_units, long long unit_rows,
                                               long long row_base, uint8_t* act_ptr,
                                               uint32_t bar_epi0 = 0, uint32_t bar_epi1 = 0) {
    volatile int* abort_flag = p.abort_flag;
    // EPIW warps per tile: warp w covers TMEM lane quadrant (w % 4), i.e.
    // rows 32 (w % 4) .. +31; with 8 warps the first four take accumulator
    // columns 0..127 and the other four 128..255 (column halves h0 .. h1 - 1
    // of 128); one thread owns one row.
    constexpr int kH = EPIW / 4;
    constexpr uint32_t kActBytes = Form<F8>::kActBytes;
    const int slot = (warp - warp0) / EPIW;
    const int h0 = kH == 2 ? (((warp - warp0) >> 2) & 1) : 0;
    const int h1 = h0 + 3 - kH;                       // one half, or both
    const int quad = warp & 3;
    const uint32_t r = quad * 32 + lane;              // row within the tile
    const uint32_t t_row = tmem + ((uint32_t)(quad * 32) << 16) + slot * 256;
    const uint32_t a_base = s_act + slot * kActBytes;
    const uint32_t g_base = s_gx + slot * kGxBytes;
    const uint32_t bar_ready = slot ? bar_ready1 : bar_ready0;
    const uint32_t bar_acc = slot ? bar_acc1 : bar_acc0;
    uint32_t acc_ph = 0;
    bool ok = true;
    // fused ray epilogue of a finished unit, run by the row-owning warps
    // (h0 == 0) after the next unit's prologue, while its first MMAs run
    EpiSync es{slot ? bar_epi1 : bar_epi0, 0u, abort_flag, p.wait_ns};
    float* scr = reinterpret_cast<float*>(act_ptr + slot * kActBytes);
    const long long n_rays = M / p.S;
    float fz[2] = {0.f, 0.f};
    float4 fo[2] = {make_float4(0.f, 0.f, 0.f, 0.f), make_float4(0.f, 0.f, 0.f, 0.f)};
    float4 ob = make_float4(0.f, 0.f, 0.f, 0.f);
    // Prologue of unit pu: this thread's halves of gamma(x) of its row into
    // the tile's gamma(x) buffer; returns the row's z and its ray's |d|.
    auto prologue = [&](long long pu, float& z_out, float& dn_out) {
        const long long gr = pu * unit_rows + row_base + slot * 128 + r;
        const bool vr = gr < M;
        float x[3] = {0.f, 0.f, 0.f};
        z_out = 0.f;
        dn_out = 0.f;
        if (vr) {
            const Ray R = p.rays[gr / p.S];
            const float zz = p.z[gr];
            z_out = zz;
            dn_out = R.dnorm;
            x[0] = fmaf(zz, R.dx, R.ox);
            x[1] = fmaf(zz, R.dy, R.oy);
            x[2] = fmaf(zz, R.dz, R.oz);
        }
        for (int half = h0; half < h1; ++half) {
            float v[32];
            if (vr) {
                if (half == 0) pe_half<0>(x, v);
                else pe_half<1>(x, v);
            } else {
#pragma unroll
                for (int i = 0; i < 32; ++i) v[i] = 0.0f;
            }
            if constexpr (F8) {
                const float sg = p.s_gx;
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    uint32_t w[4];
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const int i = 16 * j + 4 * e;
                        w[e] = pack_e4m3x4(v[i] * sg, v[i + 1] * sg, v[i + 2] * sg, v[i + 3] * sg);
                    }
                    st_shared_v4(g_base + sw128_offset(r, 2 * half + j), w[0], w[1], w[2], w[3]);
                }
            } else {
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    st_shared_v4(g_base + sw128_offset(r, 4 * half + j), pack_bf16x2(v[8 * j], v[8 * j + 1]),
                                 pack_bf16x2(v[8 * j + 2], v[8 * j + 3]),
                                 pack_bf16x2(v[8 * j + 4], v[8 * j + 5]),
                                 pack_bf16x2(v[8 * j + 6], v[8 * j + 7]));
            }
        }
    };
    // The first unit's gamma(x) is written and signalled up front.  Every
    // later unit's is written during the previous unit, after the epilogue
    // of the skip layer (l = 5: gamma(x) is last read by its MMAs, which have
    // completed when its accumulator is signalled), and
    // signalled once the previous unit's last accumulator has been read out
    // of TMEM: the next unit's first MMAs then run while this unit's RGB
    // head and ray epilogue are computed.
    float nz = 0.f, ndn = 0.f;
    // FUSE == 1: a unit's staged ray tail, finished during the next unit
    TailImp tail_in;
    tail_in.ray = -1;
    if (u0 < n_units) {
        prologue(u0, nz, ndn);
        signal_ready<PAIR>(bar_ready, lane);
    }
    for (long long pr = u0; pr < n_units && ok; pr += du) {
        const long long grow = pr * unit_rows + row_base + slot * 128 + r;
        const bool valid = grow < M;
        const long long ray = valid ? grow / p.S : 0;
        const bool has_next = pr + du < n_units;
        const float zrow = nz, dnrow = ndn;
        float4 res = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int l = 0; l < kLayers && ok; ++l) {
            const bool got = PAIR ? mbar_wait_cluster<true>(bar_acc, acc_ph, abort_flag)
                                  : mbar_wait_sleep(bar_acc, acc_ph, abort_flag, p.wait_ns);
            if (!got) {
                if constexpr (FUSE != 0) {
                    record_abort(p);
                    return;
                }
                ok = false;
                break;
            }
            acc_ph ^= 1u;
            tc_fence_after();
            if (l < 8) {
                // this thread's columns, 32 at a time, the next TMEM load
                // in flight while the current group is stored
                for (int half = h0; half < h1; ++half) {
                    const uint32_t t_acc = t_row + half * 128;
                    uint32_t va[32], vb[32];
                    tmem_ld32(t_acc, va);
                    if constexpr (F8) {
                        // h = relu(acc alpha + beta) in FP32, stored as E4M3:
                        // columns 128 half .. +127 are K-block `half`, chunks 0..7;
                        // beta: with 4 warps per tile (a whole row per
                        // thread) from global memory, with 8 from the
                        // parameter block (the faster of the two measured
                        // for each)
                        constexpr bool kBg = EPIW == 4;
                        const float alpha = p.alpha[l];
                        const float* bc = (kBg ? p.beta_g + l * 256 : p.ec.beta[l]) + half * 128;
                        const uint32_t blk = a_base + half * 16384;
#pragma unroll 1
                        for (int c32 = 0; c32 < 4; c32 += 2) {
                            tmem_ld_wait();
                            tmem_ld32(t_acc + (c32 + 1) * 32, vb);
                            epi_chunk_store_f8<kBg>(va, alpha, bc + c32 * 32, blk, r, c32 * 2);
                            tmem_ld_wait();
                            if (c32 + 2 < 4) tmem_ld32(t_acc + (c32 + 2) * 32, va);
                            epi_chunk_store_f8<kBg>(vb, alpha, bc + (c32 + 1) * 32, blk, r,
                                                    (c32 + 1) * 2);
                        }
                    } else {
                        // h = relu(acc + b): accumulators rounded to BF16 pairs,
                        // bias added and ReLU applied in packed BF16 arithmetic;
                        // columns 128 half .. +127 are K-blocks 2 half, 2 half + 1
                        const uint32_t* bb = p.ec.bias2[l] + half * 64;
#pragma unroll 1
                        for (int c32 = 0; c32 < 4; c32 += 2) {
                            tmem_ld_wait();
                            tmem_ld32(t_acc + (c32 + 1) * 32, vb);
                            const uint32_t blk = a_base + (2 * half + (c32 >> 1)) * 16384;
                            epi_chunk_store(va, bb + c32 * 16, blk, r, 0);
                            tmem_ld_wait();
                            if (c32 + 2 < 4) tmem_ld32(t_acc + (c32 + 2) * 32, va);
                            epi_chunk_store(vb, bb + (c32 + 1) * 16, blk, r, 4);
                        }
                    }
                }
                signal_ready<PAIR>(bar_ready, lane);
                if constexpr (FUSE == 1 && !F8) {
                    // the previous unit's deferred ray tail (its warp's
                    // rows: the pending state is the same in all lanes)
                    if (l == 0 && tail_in.ray >= 0) {
                        tail_importance_finish(p, tail_in, lane, nullptr);
                        tail_in.ray = -1;
                    }
                }
                if (l == 5 && has_next) prologue(pr + du, nz, ndn);
            } else {
                if (h0 == 0) {
                    // the RGB hidden layer (128 columns) and the density
                    // (column 128) read out of TMEM in two bursts, so that
                    // the accumulator is soon free for the next unit's
                    // first layer
                    const float4* rb4 = reinterpret_cast<const float4*>(p.ray_bias + ray * 128);
                    const float* wo = &p.ec.w_out[0][0];
                    float o0 = 0.f, o1 = 0.f, o2 = 0.f;
                    uint32_t va[32], vb[32];
                    uint32_t vs;
                    tmem_ld32(t_row, va);
                    tmem_ld32(t_row + 32, vb);
                    if constexpr (FUSE == 2) {
                        // the ray tail's global inputs, in flight during the
                        // RGB head: first-pass samples q = r, r + 128 of this
                        // tile's rays and the observed colour of the ray this
                        // warp composites
                        const long long ray0 = (pr * unit_rows + row_base + slot * 128) / p.S;
                        const int R1 = (128 / p.S) * p.S1;
#pragma unroll
                        for (int i = 0; i < 2; ++i) {
                            const int q = (int)r + 128 * i;
                            if (q < R1 && ray0 + q / p.S1 < n_rays) {
                                const long long idx = (ray0 + q / p.S1) * p.S1 + q % p.S1;
                                fz[i] = p.z_first[idx];
                                fo[i] = p.out_first[idx];
                            }
                        }
                        if (p.obs && quad < 128 / p.S && ray0 + quad < n_rays) ob = p.obs[ray0 + quad];
                    }
                    tmem_ld_wait();
                    rgb_group<F8>(va, rb4, wo, p.ec.alpha_last, 0, o0, o1, o2);
                    rgb_group<F8>(vb, rb4, wo, p.ec.alpha_last, 1, o0, o1, o2);
                    tmem_ld32(t_row + 64, va);
                    tmem_ld32(t_row + 96, vb);
                    tmem_ld1(t_row + 128, vs);
                    tmem_ld_wait();
                    if (has_next) signal_ready<PAIR>(bar_ready, lane);
                    rgb_group<F8>(va, rb4, wo, p.ec.alpha_last, 2, o0, o1, o2);
                    rgb_group<F8>(vb, rb4, wo, p.ec.alpha_last, 3, o0, o1, o2);
                    float sigma = __uint_as_float(vs);
                    if constexpr (F8) sigma *= p.alpha_sigma;
                    res.x = sigma + p.b_sigma;
                    res.y = 1.0f / (1.0f + __expf(-(o0 + p.b_out0)));
                    res.z = 1.0f / (1.0f + __expf(-(o1 + p.b_out1)));
                    res.w = 1.0f / (1.0f + __expf(-(o2 + p.b_out2)));
                    if (valid && FUSE != 2) p.out[grow] = res;
                } else if (has_next) {
                    // (8 warps per tile: the second column half reads no
                    // TMEM in the last layer)
                    signal_ready<PAIR>(bar_ready, lane);
                }
            }
        }
        if constexpr (FUSE != 0) {
            // the unit's ray epilogue, under the next unit's first MMAs
            if (ok) {
                const long long ray0 = (pr * unit_rows + row_base + slot * 128) / p.S;
                bool good;
                if constexpr (FUSE == 1) {
                    // staged now; BF16: computed once the next unit's
                    // first epilogue is signalled (at once after the last
                    // unit), in the epilogue warps' idle time between
                    // layers; FP8, whose epilogues bound the tensor pipe,
                    // computes it at once (measured faster for each)
                    good = tail_importance_stage(p, es, scr, (int)r, lane, quad, ray0, n_rays, zrow,
                                                 valid ? res.x : 0.f, dnrow, tail_in);
                    if (good && tail_in.ray >= 0 && (F8 || !has_next)) {
                        tail_importance_finish(p, tail_in, lane, F8 ? warp_part(scr, quad) : nullptr);
                        tail_in.ray = -1;
                    }
                } else {
                    good = tail_final(p, es, scr, (int)r, lane, quad, ray0, n_rays, zrow,
                                      valid ? res : make_float4(0.f, 0.f, 0.f, 0.f), dnrow, fz, fo, ob);
                }
                if (!good) {
                    record_abort(p);
                    return;
                }
            }
        }
    }
    if (!ok) record_abort(p);
}

template <bool F8, int EPIW, bool STAG, int FUSE = 0>
__global__ void __launch_bounds__(Variant<F8, EPIW, STAG>::kThreads, 1)
    k_mlp_tc(const __grid_constant__ Params p) {
    using Fm = Form<F8>;
    using Vt = Variant<F8, EPIW, STAG>;
    constexpr int kStages = Fm::kStages;
    constexpr uint32_t kActBytes = Fm::kActBytes;
    extern __shared__ uint8_t smem_raw[];
    __shared__ Bars bars;
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const uint32_t s_act = smem_u32(smem);                    // 2 activation tiles
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
            mbar_init(smem_u32(&bars.a_ready[s]), Vt::kEpiThreads);
            mbar_init(smem_u32(&bars.epi[s]), 128);
        }
        mbar_init(smem_u32(&bars.drain), 1);
        fence_mbar_init();
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
        // (hold_weights: issues nothing, so that the gate's first wait runs
        // out; a failure-detection test hook)
        if (lane == 0 && !p.hold_weights) {
            uint32_t g = 0;
            bool ok = true;
            auto stream = [&](int b) -> bool {
                const uint32_t st = g % kStages, ph = (g / kStages) & 1u;
                if (!mbar_wait(smem_u32(&bars.empty[st]), ph ^ 1u, abort_flag, p.wait_ns)) return false;
                mbar_arrive_expect_tx(smem_u32(&bars.full[st]), kStageBytes);
                bulk_load(s_ring + st * kStageBytes, p.wblocks + (size_t)b * kStageBytes, kStageBytes,
                          smem_u32(&bars.full[st]));
                ++g;
                return true;
            };
            for (long long pr = blockIdx.x; pr < n_pairs && ok; pr += gridDim.x)
                for (int b = 0; b < Fm::kBlocks && ok; ++b) ok = stream(b);
            if (!ok) record_abort(p);
            // every issued copy lands before the CTA may exit: the last copy
            // of each stage (earlier ones were consumed before it was issued)
            for (uint32_t k = 0; k < (uint32_t)kStages && k < g; ++k) {
                const uint32_t gl = g - 1 - k;
                mbar_wait(smem_u32(&bars.full[gl % kStages]), (gl / kStages) & 1u, nullptr);
            }
        }
    } else if (warp == 1) {
        // ------------------------------------------------ MMA issuer
        // The whole warp walks the schedule; before each group of MMAs it
        // meets the gate warp at named barrier 1 (which has waited for the
        // group's weight block and activations); lane 0 issues.
        uint32_t g = 0;
        bool ok = true;
        const uint32_t id256 = F8 ? idesc_e4m3(128, 256) : idesc_bf16(128, 256);
        const uint32_t id144 = F8 ? idesc_e4m3(128, 144) : idesc_bf16(128, 144);
        // Operand descriptors: the bases are built once; an operand at byte
        // offset o from a base is base + o / 16 (the 14-bit start-address
        // field does not overflow: all of shared memory is below 256 KB), so
        // the issuing lane does one add per operand between MMAs.  Nothing
        // here is indexed at run time: a local-memory load in the issuing
        // thread would wait behind its queued MMAs.
        const uint64_t d_act = smem_desc(s_act, 1024, kLayoutSw128);
        const uint64_t d_gx = smem_desc(s_gx, 1024, kLayoutSw128);
        const uint64_t d_ring = smem_desc(s_ring, 512, kLayoutSw64);
        // A operand of tile s, chunk c (two 32-byte K steps) of layer l:
        // gamma(x) for layer 1 and the skip layer's last chunks, else the
        // activation tile (K-blocks of 128-byte rows, 16 KB apart)
        auto a_desc = [&](int l, int s, int c) -> uint64_t {
            if (l == 0) return d_gx + (uint64_t)(s * (kGxBytes >> 4) + c * 4);
            if (l == 5 && c >= Fm::kActChunks)
                return d_gx + (uint64_t)(s * (kGxBytes >> 4) + (c - Fm::kActChunks) * 4);
            return d_act + (uint64_t)(s * (kActBytes >> 4) + (c >> 1) * 1024 + (c & 1) * 4);
        };
        auto issue = [&](int l, int s, int c, uint32_t st, uint32_t idesc) {
            const uint64_t ad = a_desc(l, s, c);
            const uint64_t bd = d_ring + (uint64_t)(st * (kStageBytes >> 4));
            const uint32_t d = tmem + s * 256;
            if constexpr (F8) {
                mma_f8(d, ad, bd, idesc, c ? 1u : 0u);
                mma_f8(d, ad + 2, bd + 2, idesc, 1u);
            } else {
                mma_bf16(d, ad, bd, idesc, c ? 1u : 0u);
                mma_bf16(d, ad + 2, bd + 2, idesc, 1u);
            }
        };
        auto gate = [&]() -> bool { return !named_bar_or(1, 64, false); };
        for (long long pr = blockIdx.x; pr < n_pairs && ok; pr += gridDim.x) {
            for (int l = 0; l < kLayers && ok; ++l) {
                const int nch = layer_chunks(F8, l);
                const uint32_t idesc = (l == 8) ? id144 : id256;
                if constexpr (STAG) {
                    // Staggered tiles: the layer's blocks in parts of at most
                    // kStages (the ring holds a whole part; the last parts are
                    // full), each part run by tile 0 and then by tile 1 on
                    // the same resident blocks, so that tile 0's epilogue
                    // runs under tile 1's last part and tile 1's under tile
                    // 0's first part of the next layer.  A stage is released
                    // after tile 1's MMAs.  (FP8: a layer is at most 5 of the
                    // 8 stages, one part; BF16: 4-block parts.)  Tile 0 takes
                    // the part's blocks in runs: each release of the gate
                    // carries the number of consecutive blocks that have
                    // landed (FP8; one block for BF16), all issued at once,
                    // so that the MMA queue stays ahead of the release round
                    // trip (a group of G MMAs leaves only a third to a half
                    // of them queued when the issuing thread moves on).
                    for (int c0 = 0; c0 < nch && ok;) {
                        const int np = (c0 == 0 && nch % kStages) ? nch % kStages : kStages;
                        for (int c = c0; c < c0 + np;) {
                            if constexpr (!F8) {
                                // one block per release: its operands and
                                // flags computed before the wait, so that
                                // only the MMAs follow the release
                                const uint64_t ad = a_desc(l, 0, c);
                                const uint64_t bd = d_ring + (uint64_t)(((g + c) % kStages) * (kStageBytes >> 4));
                                const uint32_t accum = c ? 1u : 0u;
                                const bool last = c == nch - 1;
                                if (!gate()) { ok = false; break; }
                                if (lane == 0) {
                                    tc_fence_after();
                                    mma_bf16(tmem, ad, bd, idesc, accum);
                                    mma_bf16(tmem, ad + 2, bd + 2, idesc, 1u);
                                    if (last) mma_commit(smem_u32(&bars.acc_full[0]));
                                }
                                __syncwarp();
                                ++c;
                            } else {
                                // (the run's first operands computed before the wait)
                                const uint64_t ad0 = a_desc(l, 0, c);
                                const uint64_t bd0 = d_ring + (uint64_t)(((g + c) % kStages) * (kStageBytes >> 4));
                                const int k = (int)named_bar_popc(1, 64, false);
                                if (k < 1 || k > c0 + np - c) { ok = false; break; }
                                if (lane == 0) {
                                    tc_fence_after();
                                    mma_f8(tmem, ad0, bd0, idesc, c ? 1u : 0u);
                                    mma_f8(tmem, ad0 + 2, bd0 + 2, idesc, 1u);
                                    if (c == nch - 1) mma_commit(smem_u32(&bars.acc_full[0]));
                                    for (int j = 1; j < k; ++j) {
                                        issue(l, 0, c + j, (g + c + j) % kStages, idesc);
                                        if (c + j == nch - 1) mma_commit(smem_u32(&bars.acc_full[0]));
                                    }
                                }
                                __syncwarp();
                                c += k;
                            }
                        }
                        if (!ok) break;
                        const uint64_t ad1 = a_desc(l, 1, c0);
                        const uint64_t bd1 = d_ring + (uint64_t)(((g + c0) % kStages) * (kStageBytes >> 4));
                        if (!gate()) { ok = false; break; }
                        if (lane == 0) {
                            tc_fence_after();
                            if constexpr (F8) {
                                mma_f8(tmem + 256, ad1, bd1, idesc, c0 ? 1u : 0u);
                                mma_f8(tmem + 256, ad1 + 2, bd1 + 2, idesc, 1u);
                            } else {
                                mma_bf16(tmem + 256, ad1, bd1, idesc, c0 ? 1u : 0u);
                                mma_bf16(tmem + 256, ad1 + 2, bd1 + 2, idesc, 1u);
                            }
                            mma_commit(smem_u32(&bars.empty[(g + c0) % kStages]));
                            for (int c = c0 + 1; c < c0 + np; ++c) {
                                const uint32_t st = (g + c) % kStages;
                                issue(l, 1, c, st, idesc);
                                mma_commit(smem_u32(&bars.empty[st]));
                            }
                            if (c0 + np == nch) mma_commit(smem_u32(&bars.acc_full[1]));
                        }
                        __syncwarp();
                        c0 += np;
                    }
                    g += nch;
                } else {
                    // Lockstep tiles: each weight block serves both tiles at
                    // once; the first block of a layer waits for each tile's
                    // activations separately, later blocks come in runs of
                    // landed blocks (as tile 0's in the staggered schedule).
                    for (int c = 0; c < nch;) {
                        const int k = (int)named_bar_popc(1, 64, false);
                        if (k < 1 || k > nch - c) { ok = false; break; }
                        if (lane == 0) {
                            tc_fence_after();
                            for (int j = 0; j < k; ++j) {
                                const int cc = c + j;
                                const uint32_t st = (g + cc) % kStages;
                                issue(l, 0, cc, st, idesc);
                                if (cc == nch - 1) mma_commit(smem_u32(&bars.acc_full[0]));
                                if (cc > 0) {
                                    issue(l, 1, cc, st, idesc);
                                    if (cc == nch - 1) mma_commit(smem_u32(&bars.acc_full[1]));
                                    mma_commit(smem_u32(&bars.empty[st]));
                                }
                            }
                        }
                        __syncwarp();
                        if (c == 0) {
                            if (!gate()) { ok = false; break; }
                            if (lane == 0) {
                                tc_fence_after();
                                const uint32_t st = g % kStages;
                                issue(l, 1, 0, st, idesc);
                                if (nch == 1) mma_commit(smem_u32(&bars.acc_full[1]));
                                mma_commit(smem_u32(&bars.empty[st]));
                            }
                            __syncwarp();
                        }
                        c += k;
                    }
                    g += nch;
                }
            }
        }
        if (lane == 0) {
            if (!ok) record_abort(p);
            // all issued MMAs complete before TMEM is released
            mma_commit(smem_u32(&bars.drain));
            mbar_wait(smem_u32(&bars.drain), 0, nullptr);
        }
        __syncwarp();
    } else if (warp == 2) {
        // ------------------------------------------------ gate
        // Waits (all lanes) for what each MMA group of the schedule needs,
        // then releases the MMA warp at named barrier 1, or stops it.
        uint32_t g = 0;
        uint32_t rdy_ph = 0;   // bit s: phase parity of a_ready[s]
        bool ok = true;
        auto wait_ready = [&](int s) -> bool {
            const bool r = mbar_wait(smem_u32(&bars.a_ready[s]), (rdy_ph >> s) & 1u, abort_flag, p.wait_ns);
            rdy_ph ^= 1u << s;
            return r;
        };
        auto wait_block = [&](uint32_t gi) -> bool {
            const bool r = mbar_wait(smem_u32(&bars.full[gi % kStages]), (gi / kStages) & 1u, abort_flag,
                                     p.wait_ns);
            return r;
        };
        auto release = [&](bool good) -> bool {
            __syncwarp();
            return !named_bar_or(1, 64, !good);
        };
        for (long long pr = blockIdx.x; pr < n_pairs && ok; pr += gridDim.x) {
            for (int l = 0; l < kLayers && ok; ++l) {
                const int nch = layer_chunks(F8, l);
                if constexpr (STAG) {
                    for (int c0 = 0; c0 < nch && ok;) {
                        const int np = (c0 == 0 && nch % kStages) ? nch % kStages : kStages;
                        for (int c = c0; c < c0 + np;) {
                            // wait for block c (and, for a layer's first
                            // block, tile 0's activations); lane j > 0 tests
                            // block c + j of the part without waiting; the
                            // release counts the run of landed blocks from c
                            // (0 on failure, which stops the MMA warp).
                            // BF16: one block per release, the faster
                            // measured (its blocks land just in time: the
                            // 4-stage ring holds only the current part).
                            bool good = true;
                            if (c == 0) good = wait_ready(0);
                            good = good && wait_block(g + c);
                            if constexpr (!F8) {
                                if (!release(good)) { ok = false; break; }
                                ++c;
                            } else {
                                const int rem = c0 + np - c;
                                bool landed = lane == 0;
                                if (lane > 0 && lane < rem) {
                                    const uint32_t gi = g + c + lane;
                                    landed = mbar_try_wait(smem_u32(&bars.full[gi % kStages]), (gi / kStages) & 1u);
                                }
                                const uint32_t m = __ballot_sync(0xffffffffu, landed);
                                const int k = good ? __ffs(~m) - 1 : 0;
                                __syncwarp();
                                named_bar_popc(1, 64, lane < k);
                                if (!good) { ok = false; break; }
                                c += k;
                            }
                        }
                        if (!ok) break;
                        if (!release(c0 == 0 ? wait_ready(1) : true)) { ok = false; break; }
                        c0 += np;
                    }
                    g += nch;
                } else {
                    for (int c = 0; c < nch;) {
                        // block c (and, for the first, tile 0's activations);
                        // after the first, the run of landed blocks from c,
                        // probed without waiting by lanes 1 .. (a probe stays
                        // within the ring: block c + kStages would share
                        // block c's stage)
                        bool good = wait_block(g + c);
                        if (c == 0) good = good && wait_ready(0);
                        const int rem = c == 0 ? 1 : min(nch - c, kStages);
                        bool landed = lane == 0;
                        if (lane > 0 && lane < rem) {
                            const uint32_t gi = g + c + lane;
                            landed = mbar_try_wait(smem_u32(&bars.full[gi % kStages]), (gi / kStages) & 1u);
                        }
                        const uint32_t m = __ballot_sync(0xffffffffu, landed);
                        const int k = good ? __ffs(~m) - 1 : 0;
                        __syncwarp();
                        named_bar_popc(1, 64, lane < k);
                        if (!good) { ok = false; break; }
                        if (c == 0 && !release(wait_ready(1))) { ok = false; break; }
                        c += k;
                    }
                    g += nch;
                }
            }
        }
        if (!ok && lane == 0) record_abort(p);
    } else {
        epilogue_warps<F8, EPIW, false, FUSE>(p, warp, 3, lane, tmem, s_act, s_gx,
                                        smem_u32(&bars.a_ready[0]), smem_u32(&bars.a_ready[1]),
                                        smem_u32(&bars.acc_full[0]), smem_u32(&bars.acc_full[1]),
                                        M, blockIdx.x, gridDim.x, n_pairs, 256, 0, smem,
                                        smem_u32(&bars.epi[0]), smem_u32(&bars.epi[1]));
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, 512);
    }
}

// ---------------------------------------------------------------------------
// CTA-pair form (cluster of 2 CTAs on the two SMs of a TPC, tcgen05
// cta_group::2).  Work unit: 512 rows; CTA rank r holds rows 256 r .. +255 as
// its two 128-row tiles, exactly as the single-CTA kernel holds a tile pair.
// Each MMA is M = 256 (tile s of both CTAs), N = 256 (144 for the last
// layer), so each CTA stores and streams only its half of every weight block
// (output rows N/2 r .. +N/2 - 1: 8 KB, or 4,608 bytes of the last layer's
// 144 rows): twice the ring depth in blocks, half the weight bytes per SM.
// The even CTA's warp 1 issues all MMAs, released by its gate warp once its
// own copy of a block has landed (full[]) and the odd CTA's warp 1 has
// relayed that the odd CTA's copy has (the even CTA's pfull[]); the
// epilogue warps (3 .. 10) of both CTAs signal
// the even CTA's a_ready[] barriers; the MMA commits arrive on the barriers
// of both CTAs (multicast).  Same arithmetic per row as the single-CTA
// kernel.
template <bool F8>
struct PairForm {
    static constexpr int kStages = 2 * Form<F8>::kStages;     // half-blocks
    static constexpr uint32_t kHalf = kStageBytes / 2;       // 128 rows x 64 bytes
    static constexpr uint32_t kHalfLast = 72 * 64;           // 144 / 2 rows
    static constexpr uint32_t kSmemBytes = 1024 + 2 * Form<F8>::kActBytes + 2 * kGxBytes + kStages * kHalf;
};
static_assert(PairForm<false>::kSmemBytes <= 232448 && PairForm<true>::kSmemBytes <= 232448, "smem");
constexpr int kPairMaxStages = 16;
constexpr int kPairThreads = 96 + 2 * 128;

struct __align__(8) PairBars {
    uint64_t full[kPairMaxStages];
    uint64_t pfull[kPairMaxStages];   // even CTA: the odd CTA's copy has landed
    uint64_t empty[kPairMaxStages];
    uint64_t acc_full[2];
    uint64_t a_ready[2];
    uint64_t drain;
    uint32_t tmem_base;
};

template <bool F8, bool STAG>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kPairThreads, 1)
    k_mlp_tc2(const __grid_constant__ Params p) {
    using Fm = Form<F8>;
    using Pf = PairForm<F8>;
    constexpr int kStages = Pf::kStages;
    constexpr uint32_t kActBytes = Fm::kActBytes;
    constexpr int kLastBlock0 = F8 ? 30 : 60;                 // first block of layer 9
    extern __shared__ uint8_t smem_raw[];
    __shared__ PairBars bars;
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const uint32_t s_act = smem_u32(smem);
    const uint32_t s_gx = s_act + 2 * kActBytes;
    const uint32_t s_ring = s_gx + 2 * kGxBytes;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t rank = cluster_ctarank();
    volatile int* abort_flag = p.abort_flag;
    const long long M = p.M_dev ? min(p.M, (long long)*p.M_dev) : p.M;
    const long long n_units = (M + 511) / 512;
    const long long u0 = blockIdx.x >> 1, du = gridDim.x >> 1;

    if (tid == 0) {
        for (int i = 0; i < kStages; ++i) {
            mbar_init(smem_u32(&bars.full[i]), 1);
            mbar_init(smem_u32(&bars.pfull[i]), 1);
            mbar_init(smem_u32(&bars.empty[i]), 1);
        }
        for (int s = 0; s < 2; ++s) {
            mbar_init(smem_u32(&bars.acc_full[s]), 1);
            mbar_init(smem_u32(&bars.a_ready[s]), 8);   // 4 epilogue warps x 2 CTAs
        }
        mbar_init(smem_u32(&bars.drain), 1);
        fence_mbar_init();
    }
    if (warp == 1) {
        tmem_alloc2(smem_u32(&bars.tmem_base), 512);
        tmem_relinquish2();
    }
    tc_fence_before();
    cluster_sync_all();
    tc_fence_after();
    const uint32_t tmem = bars.tmem_base;

    if (warp == 0) {
        // ------------------------------------------------ weight stream (both CTAs)
        if (lane == 0) {
            uint32_t g = 0;
            bool ok = true;
            for (long long u = u0; u < n_units && ok; u += du) {
                for (int b = 0; b < Fm::kBlocks; ++b, ++g) {
                    const uint32_t st = g % kStages, ph = (g / kStages) & 1u;
                    if (!mbar_wait_cluster<false>(smem_u32(&bars.empty[st]), ph ^ 1u, abort_flag)) {
                        ok = false;
                        break;
                    }
                    const uint32_t bytes = b >= kLastBlock0 ? Pf::kHalfLast : Pf::kHalf;
                    mbar_arrive_expect_tx(smem_u32(&bars.full[st]), bytes);
                    bulk_load(s_ring + st * Pf::kHalf, p.wblocks + (size_t)b * kStageBytes + rank * bytes,
                              bytes, smem_u32(&bars.full[st]));
                }
            }
            if (!ok) record_abort(p);
            // every issued copy lands before the CTA may exit: the last copy
            // of each stage (earlier ones were consumed before it was issued)
            for (uint32_t k = 0; k < (uint32_t)kStages && k < g; ++k) {
                const uint32_t gl = g - 1 - k;
                mbar_wait(smem_u32(&bars.full[gl % kStages]), (gl / kStages) & 1u, nullptr);
            }
        }
    } else if (warp == 1 && rank == 1) {
        // ------------------------------------------------ relay (odd CTA)
        if (lane == 0) {
            uint32_t g = 0;
            bool ok = true;
            for (long long u = u0; u < n_units && ok; u += du)
                for (int b = 0; b < Fm::kBlocks; ++b, ++g) {
                    const uint32_t st = g % kStages, ph = (g / kStages) & 1u;
                    if (!mbar_wait(smem_u32(&bars.full[st]), ph, abort_flag)) {
                        ok = false;
                        break;
                    }
                    mbar_arrive_cluster(mapa_shared(smem_u32(&bars.pfull[st]), 0));
                }
            if (!ok) record_abort(p);
        }
    } else if (warp == 1) {
        // ------------------------------------------------ MMA issuer (even CTA)
        // As in the single-CTA kernel: the whole warp walks the schedule and
        // meets the gate warp at named barrier 1 before each group; lane 0
        // issues the pair's MMAs and commits to the barriers of both CTAs.
        uint32_t g = 0;
        bool ok = true;
        const uint32_t id256 = F8 ? idesc_e4m3(256, 256) : idesc_bf16(256, 256);
        const uint32_t id144 = F8 ? idesc_e4m3(256, 144) : idesc_bf16(256, 144);
        constexpr uint16_t kBoth = 3;
        const uint64_t d_act = smem_desc(s_act, 1024, kLayoutSw128);
        const uint64_t d_gx = smem_desc(s_gx, 1024, kLayoutSw128);
        const uint64_t d_ring = smem_desc(s_ring, 512, kLayoutSw64);
        auto a_desc = [&](int l, int s, int c) -> uint64_t {
            if (l == 0) return d_gx + (uint64_t)(s * (kGxBytes >> 4) + c * 4);
            if (l == 5 && c >= Fm::kActChunks)
                return d_gx + (uint64_t)(s * (kGxBytes >> 4) + (c - Fm::kActChunks) * 4);
            return d_act + (uint64_t)(s * (kActBytes >> 4) + (c >> 1) * 1024 + (c & 1) * 4);
        };
        auto issue = [&](int l, int s, int c, uint32_t st, uint32_t idesc) {
            const uint64_t ad = a_desc(l, s, c);
            const uint64_t bd = d_ring + (uint64_t)(st * (Pf::kHalf >> 4));
            const uint32_t d = tmem + s * 256;
            if constexpr (F8) {
                mma2_f8(d, ad, bd, idesc, c ? 1u : 0u);
                mma2_f8(d, ad + 2, bd + 2, idesc, 1u);
            } else {
                mma2_bf16(d, ad, bd, idesc, c ? 1u : 0u);
                mma2_bf16(d, ad + 2, bd + 2, idesc, 1u);
            }
        };
        auto gate = [&]() -> bool { return !named_bar_or(1, 64, false); };
        for (long long u = u0; u < n_units && ok; u += du) {
            for (int l = 0; l < kLayers && ok; ++l) {
                const int nch = layer_chunks(F8, l);
                const uint32_t idesc = (l == 8) ? id144 : id256;
                if constexpr (STAG) {
                    // Staggered tiles over parts of at most kStages half-blocks
                    // (the ring holds a whole part: a whole layer but the
                    // skip layer's, which runs as 2 + 8 blocks in BF16), each
                    // part run by tile 0 and then by tile 1 on the same
                    // resident blocks, so each tile's epilogue overlaps the
                    // other tile's whole layer.  Tile 0 takes the part's
                    // blocks in runs of landed blocks (the count the gate
                    // releases), tile 1 the whole part at once.
                    for (int c0 = 0; c0 < nch && ok;) {
                        const int np = (c0 == 0 && nch % kStages) ? nch % kStages : kStages;
                        for (int c = c0; c < c0 + np;) {
                            const int k = (int)named_bar_popc(1, 64, false);
                            if (k < 1 || k > c0 + np - c) { ok = false; break; }
                            if (lane == 0) {
                                tc_fence_after();
                                for (int j = 0; j < k; ++j) {
                                    issue(l, 0, c + j, (g + c + j) % kStages, idesc);
                                    if (c + j == nch - 1) mma_commit2_mc(smem_u32(&bars.acc_full[0]), kBoth);
                                }
                            }
                            __syncwarp();
                            c += k;
                        }
                        if (!ok) break;
                        if (!gate()) { ok = false; break; }
                        if (lane == 0) {
                            tc_fence_after();
                            for (int c = c0; c < c0 + np; ++c) {
                                const uint32_t st = (g + c) % kStages;
                                issue(l, 1, c, st, idesc);
                                mma_commit2_mc(smem_u32(&bars.empty[st]), kBoth);
                            }
                            if (c0 + np == nch) mma_commit2_mc(smem_u32(&bars.acc_full[1]), kBoth);
                        }
                        __syncwarp();
                        c0 += np;
                    }
                    g += nch;
                } else {
                    for (int c = 0; c < nch; ++c, ++g) {
                        const uint32_t st = g % kStages;
                        if (!gate()) { ok = false; break; }
                        if (lane == 0) {
                            tc_fence_after();
                            issue(l, 0, c, st, idesc);
                            if (c == nch - 1) mma_commit2_mc(smem_u32(&bars.acc_full[0]), kBoth);
                            if (c > 0) {
                                issue(l, 1, c, st, idesc);
                                if (c == nch - 1) mma_commit2_mc(smem_u32(&bars.acc_full[1]), kBoth);
                                mma_commit2_mc(smem_u32(&bars.empty[st]), kBoth);
                            }
                        }
                        __syncwarp();
                        if (c == 0) {
                            if (!gate()) { ok = false; break; }
                            if (lane == 0) {
                                tc_fence_after();
                                issue(l, 1, 0, st, idesc);
                                if (nch == 1) mma_commit2_mc(smem_u32(&bars.acc_full[1]), kBoth);
                                mma_commit2_mc(smem_u32(&bars.empty[st]), kBoth);
                            }
                            __syncwarp();
                        }
                    }
                }
            }
        }
        if (lane == 0) {
            if (!ok) record_abort(p);
            // all issued MMAs (they write both CTAs' TMEM and read both CTAs'
            // shared memory) complete before either CTA releases TMEM or exits
            mma_commit2_mc(smem_u32(&bars.drain), 1);
            mbar_wait(smem_u32(&bars.drain), 0, nullptr);
        }
        __syncwarp();
    } else if (warp == 2) {
        // ------------------------------------------------ gate (even CTA)
        if (rank == 0) {
            uint32_t g = 0;
            uint32_t rdy_ph = 0;   // bit s: phase parity of a_ready[s]
            bool ok = true;
            auto wait_ready = [&](int s) -> bool {
                const bool r = mbar_wait_cluster<false>(smem_u32(&bars.a_ready[s]), (rdy_ph >> s) & 1u, abort_flag);
                rdy_ph ^= 1u << s;
                return r;
            };
            // block gi present in both CTAs
            auto wait_block = [&](uint32_t gi) -> bool {
                const uint32_t st = gi % kStages, ph = (gi / kStages) & 1u;
                const bool r = mbar_wait(smem_u32(&bars.full[st]), ph, abort_flag);
                const bool r2 = r && mbar_wait_cluster<false>(smem_u32(&bars.pfull[st]), ph, abort_flag);
                return r2;
            };
            auto release = [&](bool good) -> bool {
                __syncwarp();
                return !named_bar_or(1, 64, !good);
            };
            for (long long u = u0; u < n_units && ok; u += du) {
                for (int l = 0; l < kLayers && ok; ++l) {
                    const int nch = layer_chunks(F8, l);
                    if constexpr (STAG) {
                        for (int c0 = 0; c0 < nch && ok;) {
                            const int np = (c0 == 0 && nch % kStages) ? nch % kStages : kStages;
                            for (int c = c0; c < c0 + np;) {
                                // block c (and, for the layer's first, tile 0's
                                // activations) in both CTAs; lane j > 0 probes
                                // block c + j of the part without waiting; the
                                // release counts the run of landed blocks (0 on
                                // failure, which stops the MMA warp)
                                bool good = true;
                                if (c == 0) good = wait_ready(0);
                                good = good && wait_block(g + c);
                                const int rem = c0 + np - c;
                                bool landed = lane == 0;
                                if (lane > 0 && lane < rem) {
                                    const uint32_t gi = g + c + lane;
                                    const uint32_t st = gi % kStages, ph = (gi / kStages) & 1u;
                                    landed = mbar_try_wait(smem_u32(&bars.full[st]), ph) &&
                                             mbar_try_wait_cluster(smem_u32(&bars.pfull[st]), ph);
                                }
                                const uint32_t m = __ballot_sync(0xffffffffu, landed);
                                const int k = good ? __ffs(~m) - 1 : 0;
                                __syncwarp();
                                named_bar_popc(1, 64, lane < k);
                                if (!good) { ok = false; break; }
                                c += k;
                            }
                            if (!ok) break;
                            if (!release(c0 == 0 ? wait_ready(1) : true)) { ok = false; break; }
                            c0 += np;
                        }
                        g += nch;
                    } else {
                        for (int c = 0; c < nch; ++c, ++g) {
                            bool good = wait_block(g);
                            if (c == 0) good = good && wait_ready(0);
                            if (!release(good)) { ok = false; break; }
                            if (c == 0 && !release(wait_ready(1))) { ok = false; break; }
                        }
                    }
                }
            }
            if (!ok && lane == 0) record_abort(p);
        }
    } else {
        const uint32_t rdy0 = mapa_shared(smem_u32(&bars.a_ready[0]), 0);
        const uint32_t rdy1 = mapa_shared(smem_u32(&bars.a_ready[1]), 0);
        epilogue_warps<F8, 4, true>(p, warp, 3, lane, tmem, s_act, s_gx, rdy0, rdy1,
                                    smem_u32(&bars.acc_full[0]), smem_u32(&bars.acc_full[1]), M, u0, du,
                                    n_units, 512, (long long)rank * 256, smem);
    }
    __syncwarp();
    tc_fence_before();
    cluster_sync_all();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc2(tmem, 512);
    }
}

// ---------------------------------------------------------------------------
// BF16, split schedule: every layer runs as two 128-column halves (N = 128)
// over weight blocks [128 output rows x 64 k] (128-byte swizzle), tiles in
// lockstep.  Half 0's accumulators are committed once every MMA that reads
// activation columns 0..127 has completed (after half 1's first two K
// chunks), so the epilogue of columns 0..127 runs while half 1 finishes, and
// the next layer's first two K chunks start as soon as it is done; the
// epilogue of columns 128..255 then overlaps those.  The last layer's half 1
// is the density head (one row, N = 16).  Same arithmetic as the lockstep
// kernel.
struct __align__(8) SplitBars {
    uint64_t full[4];
    uint64_t empty[4];
    uint64_t acc_lo[2], acc_hi[2];
    uint64_t rdy_lo[2], rdy_hi[2];
    uint64_t drain;
    uint32_t tmem_base;
};
constexpr int kSplitStages = 4;
constexpr int kSplitThreads = 64 + 2 * 128;
constexpr uint32_t kSplitSmem = Form<false>::kSmemBytes;

// K chunks (64 k each) of layer l: trunk1 gamma(x) (64), skip layer 320, else 256
__device__ __forceinline__ int split_chunks(int l) { return l == 0 ? 1 : (l == 5 ? 5 : 4); }

__global__ void __launch_bounds__(kSplitThreads, 1) k_mlp_tc_split(const __grid_constant__ Params p) {
    constexpr uint32_t kActBytes = Form<false>::kActBytes;
    extern __shared__ uint8_t smem_raw[];
    __shared__ SplitBars bars;
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const uint32_t s_act = smem_u32(smem);
    const uint32_t s_gx = s_act + 2 * kActBytes;
    const uint32_t s_ring = s_gx + 2 * kGxBytes;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    volatile int* abort_flag = p.abort_flag;
    const long long M = p.M_dev ? min(p.M, (long long)*p.M_dev) : p.M;
    const long long n_pairs = (M + 255) / 256;
    if (tid == 0) {
        for (int i = 0; i < kSplitStages; ++i) {
            mbar_init(smem_u32(&bars.full[i]), 1);
            mbar_init(smem_u32(&bars.empty[i]), 1);
        }
        for (int s = 0; s < 2; ++s) {
            mbar_init(smem_u32(&bars.acc_lo[s]), 1);
            mbar_init(smem_u32(&bars.acc_hi[s]), 1);
            mbar_init(smem_u32(&bars.rdy_lo[s]), 128);
            mbar_init(smem_u32(&bars.rdy_hi[s]), 128);
        }
        mbar_init(smem_u32(&bars.drain), 1);
        fence_mbar_init();
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
        if (lane == 0) {
            uint32_t g = 0;
            bool ok = true;
            for (long long pr = blockIdx.x; pr < n_pairs && ok; pr += gridDim.x) {
                for (int b = 0; b < Form<false>::kBlocks; ++b, ++g) {
                    const uint32_t st = g % kSplitStages, ph = (g / kSplitStages) & 1u;
                    if (!mbar_wait(smem_u32(&bars.empty[st]), ph ^ 1u, abort_flag)) {
                        ok = false;
                        break;
                    }
                    mbar_arrive_expect_tx(smem_u32(&bars.full[st]), kStageBytes);
                    bulk_load(s_ring + st * kStageBytes, p.wblocks + (size_t)b * kStageBytes,
                              kStageBytes, smem_u32(&bars.full[st]));
                }
            }
            if (!ok) record_abort(p);
            for (uint32_t k = 0; k < (uint32_t)kSplitStages && k < g; ++k) {
                const uint32_t gl = g - 1 - k;
                mbar_wait(smem_u32(&bars.full[gl % kSplitStages]), (gl / kSplitStages) & 1u, nullptr);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            uint32_t g = 0;
            uint32_t ph_lo[2] = {0, 0}, ph_hi[2] = {0, 0};
            bool ok = true;
            const uint32_t id128 = idesc_bf16(128, 128), id16 = idesc_bf16(128, 16);
            auto wait_rdy = [&](uint64_t* bar, uint32_t& ph) -> bool {
                if (!mbar_wait(smem_u32(bar), ph, abort_flag)) return false;
                ph ^= 1u;
                tc_fence_after();
                return true;
            };
            for (long long pr = blockIdx.x; pr < n_pairs && ok; pr += gridDim.x) {
                for (int l = 0; l < kLayers && ok; ++l) {
                    const int nch = split_chunks(l);
                    for (int h = 0; h < 2 && ok; ++h) {
                        const uint32_t idesc = (l == 8 && h == 1) ? id16 : id128;
                        for (int c = 0; c < nch && ok; ++c) {
                            const uint32_t st = g % kSplitStages, ph = (g / kSplitStages) & 1u;
                            if (!mbar_wait(smem_u32(&bars.full[st]), ph, abort_flag)) {
                                ok = false;
                                break;
                            }
                            for (int s = 0; s < 2 && ok; ++s) {
                                // accumulator half h of tile s is free and its
                                // A chunk written: columns 0..127 of the previous
                                // output before K chunk 0, 128..255 before chunk 2
                                if (h == 0 && c == 0) ok = wait_rdy(&bars.rdy_lo[s], ph_lo[s]);
                                if (ok && ((l > 0 && h == 0 && c == 2) || (l == 0 && h == 1 && c == 0)))
                                    ok = wait_rdy(&bars.rdy_hi[s], ph_hi[s]);
                                if (!ok) break;
                                uint32_t a0;
                                if (l == 0) a0 = s_gx + s * kGxBytes;
                                else if (l == 5 && c == 4) a0 = s_gx + s * kGxBytes;
                                else a0 = s_act + s * kActBytes + c * 16384;
#pragma unroll
                                for (int kk = 0; kk < 4; ++kk) {
                                    const uint64_t ad = smem_desc(a0 + kk * 32, 1024, kLayoutSw128);
                                    const uint64_t bd =
                                        smem_desc(s_ring + st * kStageBytes + kk * 32, 1024, kLayoutSw128);
                                    mma_bf16(tmem + s * 256 + h * 128, ad, bd, idesc, (c | kk) ? 1u : 0u);
                                }
                                // columns 0..127 are final once no pending MMA reads
                                // activation columns 0..127: after half 0 (layer 0:
                                // reads gamma(x) only) or after half 1's chunk 1
                                if ((l == 0 && h == 0 && c == nch - 1) || (l > 0 && h == 1 && c == 1))
                                    mma_commit(smem_u32(&bars.acc_lo[s]));
                                if (h == 1 && c == nch - 1) mma_commit(smem_u32(&bars.acc_hi[s]));
                            }
                            if (!ok) break;
                            mma_commit(smem_u32(&bars.empty[st]));
                            ++g;
                        }
                    }
                }
            }
            if (!ok) record_abort(p);
            mma_commit(smem_u32(&bars.drain));
            mbar_wait(smem_u32(&bars.drain), 0, nullptr);
        }
    } else {
        const int slot = (warp - 2) >> 2;
        const int quad = warp & 3;
        const uint32_t r = quad * 32 + lane;
        const uint32_t t_row = tmem + ((uint32_t)(quad * 32) << 16) + slot * 256;
        const uint32_t a_base = s_act + slot * kActBytes;
        const uint32_t g_base = s_gx + slot * kGxBytes;
        const uint32_t b_lo = smem_u32(&bars.acc_lo[slot]), b_hi = smem_u32(&bars.acc_hi[slot]);
        const uint32_t r_lo = smem_u32(&bars.rdy_lo[slot]), r_hi = smem_u32(&bars.rdy_hi[slot]);
        uint32_t ph_lo = 0, ph_hi = 0;
        bool ok = true;
        for (long long pr = blockIdx.x; pr < n_pairs && ok; pr += gridDim.x) {
            const long long grow = pr * 256 + slot * 128 + r;
            const bool valid = grow < M;
            const long long ray = valid ? grow / p.S : 0;
            {
                float x[3] = {0.f, 0.f, 0.f};
                if (valid) {
                    const Ray R = p.rays[ray];
                    const float zz = p.z[grow];
                    x[0] = fmaf(zz, R.dx, R.ox);
                    x[1] = fmaf(zz, R.dy, R.oy);
                    x[2] = fmaf(zz, R.dz, R.oz);
                }
                for (int half = 0; half < 2; ++half) {
                    float v[32];
                    if (valid) {
                        if (half == 0) pe_half<0>(x, v);
                        else pe_half<1>(x, v);
                    } else {
#pragma unroll
                        for (int i = 0; i < 32; ++i) v[i] = 0.0f;
                    }
#pragma unroll
                    for (int j = 0; j < 4; ++j)
                        st_shared_v4(g_base + sw128_offset(r, 4 * half + j),
                                     pack_bf16x2(v[8 * j], v[8 * j + 1]),
                                     pack_bf16x2(v[8 * j + 2], v[8 * j + 3]),
                                     pack_bf16x2(v[8 * j + 4], v[8 * j + 5]),
                                     pack_bf16x2(v[8 * j + 6], v[8 * j + 7]));
                }
                fence_proxy_async_smem();
                tc_fence_before();
                mbar_arrive(r_lo);
                mbar_arrive(r_hi);
            }
            float o0 = 0.f, o1 = 0.f, o2 = 0.f;
            const float4* rb4 = reinterpret_cast<const float4*>(p.ray_bias + ray * 128);
            const float* wo = &p.ec.w_out[0][0];
            for (int l = 0; l < kLayers && ok; ++l) {
                for (int h = 0; h < 2 && ok; ++h) {
                    if (!mbar_wait(h ? b_hi : b_lo, h ? ph_hi : ph_lo, abort_flag)) {
                        ok = false;
                        break;
                    }
                    if (h) ph_hi ^= 1u;
                    else ph_lo ^= 1u;
                    tc_fence_after();
                    const uint32_t t_acc = t_row + h * 128;
                    if (l < 8) {
                        const uint32_t* bb = p.ec.bias2[l] + h * 64;
                        uint32_t va[32], vb[32];
                        tmem_ld32(t_acc, va);
#pragma unroll 1
                        for (int c32 = 0; c32 < 4; c32 += 2) {
                            tmem_ld_wait();
                            tmem_ld32(t_acc + (c32 + 1) * 32, vb);
                            const uint32_t blk = a_base + (2 * h + (c32 >> 1)) * 16384;
                            epi_chunk_store(va, bb + c32 * 16, blk, r, 0);
                            tmem_ld_wait();
                            if (c32 + 2 < 4) tmem_ld32(t_acc + (c32 + 2) * 32, va);
                            epi_chunk_store(vb, bb + (c32 + 1) * 16, blk, r, 4);
                        }
                        fence_proxy_async_smem();
                        tc_fence_before();
                        mbar_arrive(h ? r_hi : r_lo);
                    } else if (h == 0) {
                        uint32_t va[32], vb[32];
                        tmem_ld32(t_acc, va);
#pragma unroll 1
                        for (int c32 = 0; c32 < 4; c32 += 2) {
                            tmem_ld_wait();
                            tmem_ld32(t_acc + (c32 + 1) * 32, vb);
                            rgb_group<false>(va, rb4, wo, nullptr, c32, o0, o1, o2);
                            tmem_ld_wait();
                            if (c32 + 2 < 4) tmem_ld32(t_acc + (c32 + 2) * 32, va);
                            rgb_group<false>(vb, rb4, wo, nullptr, c32 + 1, o0, o1, o2);
                        }
                    } else {
                        // density head: accumulator column 128 of the last layer
                        uint32_t vs[32];
                        tmem_ld32(t_acc, vs);
                        tmem_ld_wait();
                        tc_fence_before();
                        if (valid) {
                            float4 res;
                            res.x = __uint_as_float(vs[0]) + p.b_sigma;
                            res.y = 1.0f / (1.0f + __expf(-(o0 + p.b_out0)));
                            res.z = 1.0f / (1.0f + __expf(-(o1 + p.b_out1)));
                            res.w = 1.0f / (1.0f + __expf(-(o2 + p.b_out2)));
                            p.out[grow] = res;
                        }
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

// ---------------------------------------------------------------------------
// BF16, pipelined single tile: one 128-row tile per CTA at a time, its
// accumulators double-buffered in TMEM (layer l in columns 256 (l & 1) ..
// +255), and the activation columns handed to the next layer 64 at a time:
// the epilogue of layer l releases K chunks 2q, 2q + 1 of layer l + 1 as
// soon as it has written columns 64q .. 64q + 63, so the MMAs of layer l + 1
// run under the rest of layer l's epilogue.  Nine-stage weight ring (more
// than a layer), same weight blocks and arithmetic as the lockstep kernel.
struct __align__(8) PipeBars {
    uint64_t full[9];
    uint64_t empty[9];
    uint64_t acc_full[2];
    uint64_t q_ready[4];
    uint64_t gx_ready;
    uint64_t drain;
    uint32_t tmem_base;
};
constexpr int kPipeStages = 9;
constexpr int kPipeThreads = 64 + 128;
constexpr uint32_t kPipeSmem = 1024 + Form<false>::kActBytes + kGxBytes + kPipeStages * kStageBytes;
static_assert(kPipeSmem <= 232448, "pipelined kernel shared memory");

__global__ void __launch_bounds__(kPipeThreads, 1) k_mlp_tc_pipe(const __grid_constant__ Params p) {
    extern __shared__ uint8_t smem_raw[];
    __shared__ PipeBars bars;
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const uint32_t s_act = smem_u32(smem);
    const uint32_t s_gx = s_act + Form<false>::kActBytes;
    const uint32_t s_ring = s_gx + kGxBytes;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    volatile int* abort_flag = p.abort_flag;
    const long long M = p.M_dev ? min(p.M, (long long)*p.M_dev) : p.M;
    const long long n_tiles = (M + 127) / 128;
    if (tid == 0) {
        for (int i = 0; i < kPipeStages; ++i) {
            mbar_init(smem_u32(&bars.full[i]), 1);
            mbar_init(smem_u32(&bars.empty[i]), 1);
        }
        for (int b = 0; b < 2; ++b) mbar_init(smem_u32(&bars.acc_full[b]), 1);
        for (int q = 0; q < 4; ++q) mbar_init(smem_u32(&bars.q_ready[q]), 128);
        mbar_init(smem_u32(&bars.gx_ready), 128);
        mbar_init(smem_u32(&bars.drain), 1);
        fence_mbar_init();
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
        if (lane == 0) {
            uint32_t g = 0;
            bool ok = true;
            for (long long t = blockIdx.x; t < n_tiles && ok; t += gridDim.x) {
                for (int b = 0; b < Form<false>::kBlocks; ++b, ++g) {
                    const uint32_t st = g % kPipeStages, ph = (g / kPipeStages) & 1u;
                    if (!mbar_wait(smem_u32(&bars.empty[st]), ph ^ 1u, abort_flag)) {
                        ok = false;
                        break;
                    }
                    mbar_arrive_expect_tx(smem_u32(&bars.full[st]), kStageBytes);
                    bulk_load(s_ring + st * kStageBytes, p.wblocks + (size_t)b * kStageBytes,
                              kStageBytes, smem_u32(&bars.full[st]));
                }
            }
            if (!ok) record_abort(p);
            for (uint32_t k = 0; k < (uint32_t)kPipeStages && k < g; ++k) {
                const uint32_t gl = g - 1 - k;
                mbar_wait(smem_u32(&bars.full[gl % kPipeStages]), (gl / kPipeStages) & 1u, nullptr);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            uint32_t g = 0, ph_bits = 0;   // bit q: parity of q_ready[q]; bit 4: gx_ready
            bool ok = true;
            const uint32_t id256 = idesc_bf16(128, 256), id144 = idesc_bf16(128, 144);
            for (long long t = blockIdx.x; t < n_tiles && ok; t += gridDim.x) {
                for (int l = 0; l < kLayers && ok; ++l) {
                    const int nch = layer_chunks(false, l);
                    const uint32_t idesc = (l == 8) ? id144 : id256;
                    const uint32_t d = tmem + (l & 1) * 256;
                    for (int c = 0; c < nch && ok; ++c) {
                        const uint32_t st = g % kPipeStages, ph = (g / kPipeStages) & 1u;
                        if (!mbar_wait(smem_u32(&bars.full[st]), ph, abort_flag)) {
                            ok = false;
                            break;
                        }
                        // A chunk written: gamma(x) (layer 0) or columns 64q .. +63
                        // of the previous layer's output (chunks 2q, 2q + 1);
                        // phase parities kept as bits of one register
                        int wsel = -1;
                        if (l == 0 && c == 0) wsel = 4;
                        else if (l > 0 && c < 8 && (c & 1) == 0) wsel = c >> 1;
                        if (wsel >= 0) {
                            const uint32_t wb = wsel == 4 ? smem_u32(&bars.gx_ready)
                                                          : smem_u32(&bars.q_ready[wsel]);
                            const uint32_t wp = (ph_bits >> wsel) & 1u;
                            if (!mbar_wait(wb, wp, abort_flag)) {
                                ok = false;
                                break;
                            }
                            ph_bits ^= 1u << wsel;
                            tc_fence_after();
                        }
#pragma unroll
                        for (int kk = 0; kk < 2; ++kk) {
                            uint32_t a_addr;
                            if (l == 0) a_addr = s_gx + (c * 2 + kk) * 32;
                            else if (l == 5 && c >= 8) a_addr = s_gx + ((c - 8) * 2 + kk) * 32;
                            else {
                                const int ks = c * 2 + kk;
                                a_addr = s_act + (ks >> 2) * 16384 + (ks & 3) * 32;
                            }
                            const uint64_t ad = smem_desc(a_addr, 1024, kLayoutSw128);
                            const uint64_t bd = smem_desc(s_ring + st * kStageBytes + kk * 32, 512, kLayoutSw64);
                            mma_bf16(d, ad, bd, idesc, (c | kk) ? 1u : 0u);
                        }
                        mma_commit(smem_u32(&bars.empty[st]));
                        ++g;
                    }
                    if (ok) mma_commit(smem_u32(&bars.acc_full[l & 1]));
                }
            }
            if (!ok) record_abort(p);
            mma_commit(smem_u32(&bars.drain));
            mbar_wait(smem_u32(&bars.drain), 0, nullptr);
        }
    } else {
        const int quad = warp & 3;
        const uint32_t r = quad * 32 + lane;
        const uint32_t t_lane = tmem + ((uint32_t)(quad * 32) << 16);
        uint32_t ph_acc[2] = {0, 0};
        bool ok = true;
        for (long long t = blockIdx.x; t < n_tiles && ok; t += gridDim.x) {
            const long long grow = t * 128 + r;
            const bool valid = grow < M;
            const long long ray = valid ? grow / p.S : 0;
            {
                float x[3] = {0.f, 0.f, 0.f};
                if (valid) {
                    const Ray R = p.rays[ray];
                    const float zz = p.z[grow];
                    x[0] = fmaf(zz, R.dx, R.ox);
                    x[1] = fmaf(zz, R.dy, R.oy);
                    x[2] = fmaf(zz, R.dz, R.oz);
                }
                for (int half = 0; half < 2; ++half) {
                    float v[32];
                    if (valid) {
                        if (half == 0) pe_half<0>(x, v);
                        else pe_half<1>(x, v);
                    } else {
#pragma unroll
                        for (int i = 0; i < 32; ++i) v[i] = 0.0f;
                    }
#pragma unroll
                    for (int j = 0; j < 4; ++j)
                        st_shared_v4(s_gx + sw128_offset(r, 4 * half + j), pack_bf16x2(v[8 * j], v[8 * j + 1]),
                                     pack_bf16x2(v[8 * j + 2], v[8 * j + 3]),
                                     pack_bf16x2(v[8 * j + 4], v[8 * j + 5]),
                                     pack_bf16x2(v[8 * j + 6], v[8 * j + 7]));
                }
                fence_proxy_async_smem();
                tc_fence_before();
                mbar_arrive(smem_u32(&bars.gx_ready));
            }
            for (int l = 0; l < kLayers && ok; ++l) {
                const int b = l & 1;
                if (!mbar_wait(smem_u32(&bars.acc_full[b]), ph_acc[b], abort_flag)) {
                    ok = false;
                    break;
                }
                ph_acc[b] ^= 1u;
                tc_fence_after();
                const uint32_t t_acc = t_lane + b * 256;
                if (l < 8) {
                    // 64 columns at a time (one 128-byte K block of the next
                    // layer), each released to the MMAs as soon as it is stored
                    const uint32_t* bb = p.ec.bias2[l];
                    uint32_t va[32], vb[32];
                    tmem_ld32(t_acc, va);
#pragma unroll 1
                    for (int q = 0; q < 4; ++q) {
                        tmem_ld_wait();
                        tmem_ld32(t_acc + (2 * q + 1) * 32, vb);
                        const uint32_t blk = s_act + q * 16384;
                        epi_chunk_store(va, bb + (2 * q) * 16, blk, r, 0);
                        tmem_ld_wait();
                        if (q + 1 < 4) tmem_ld32(t_acc + (2 * q + 2) * 32, va);
                        epi_chunk_store(vb, bb + (2 * q + 1) * 16, blk, r, 4);
                        fence_proxy_async_smem();
                        tc_fence_before();
                        mbar_arrive(smem_u32(&bars.q_ready[q]));
                    }
                } else {
                    const float4* rb4 = reinterpret_cast<const float4*>(p.ray_bias + ray * 128);
                    const float* wo = &p.ec.w_out[0][0];
                    float o0 = 0.f, o1 = 0.f, o2 = 0.f;
                    uint32_t va[32], vb[32];
                    tmem_ld32(t_acc, va);
#pragma unroll 1
                    for (int c32 = 0; c32 < 4; c32 += 2) {
                        tmem_ld_wait();
                        tmem_ld32(t_acc + (c32 + 1) * 32, vb);
                        rgb_group<false>(va, rb4, wo, nullptr, c32, o0, o1, o2);
                        tmem_ld_wait();
                        if (c32 + 2 < 4) tmem_ld32(t_acc + (c32 + 2) * 32, va);
                        rgb_group<false>(vb, rb4, wo, nullptr, c32 + 1, o0, o1, o2);
                    }
                    uint32_t vs[32];
                    tmem_ld32(t_acc + 128, vs);
                    tmem_ld_wait();
                    tc_fence_before();
                    if (valid) {
                        float4 res;
                        res.x = __uint_as_float(vs[0]) + p.b_sigma;
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
    for (int i = 0; i < kGd; ++i) s = fmaf(Wd[i * 128 + o], g[i], s);   // Wd: [27][128]
    out[t] = s;
}

// The kernel variants (see Variant): precision, epilogue warps, staggered.
struct TcVariant {
    int precision, epi_warps;
    bool staggered;             // FP8: staggered tiles; BF16: split schedule (own weight layout)
    void (*fn)(Params);
    int threads;
    uint32_t smem;
    int cluster;                // 1, or 2: CTA pairs over 512-row units
};
template <bool F8, int W, bool S>
constexpr TcVariant make_variant() {
    return TcVariant{F8 ? MCL_PREC_FP8 : MCL_PREC_BF16, W, S, &k_mlp_tc<F8, W, S>,
                     Variant<F8, W, S>::kThreads, Form<F8>::kSmemBytes, 1};
}
template <bool F8, bool S>
constexpr TcVariant make_pair_variant() {
    return TcVariant{F8 ? MCL_PREC_FP8 : MCL_PREC_BF16, 4, S, &k_mlp_tc2<F8, S>, kPairThreads,
                     PairForm<F8>::kSmemBytes, 2};
}
const TcVariant kVariants[] = {
    make_variant<false, 4, false>(), make_variant<false, 8, false>(),
    make_variant<true, 4, false>(),  make_variant<true, 8, false>(),
    make_variant<true, 4, true>(),   make_variant<true, 8, true>(),
    TcVariant{MCL_PREC_BF16, 4, true, &k_mlp_tc_split, kSplitThreads, kSplitSmem, 1},
    TcVariant{MCL_PREC_BF16, 4, false, &k_mlp_tc_pipe, kPipeThreads, kPipeSmem, 1},
    make_pair_variant<false, false>(), make_pair_variant<true, false>(),
    make_pair_variant<true, true>(),     make_variant<false, 4, true>(),
    make_variant<false, 8, true>(),      make_pair_variant<false, true>(),
};
// Fused passes (Params::fuse 1, 2) run on the single-CTA kernel with 4
// epilogue warps per tile (the fused ray epilogues need one thread per row)
// and staggered tiles.
void (*const kFusedKernels[2][2])(Params) = {
    {&k_mlp_tc<false, 4, true, 1>, &k_mlp_tc<false, 4, true, 2>},
    {&k_mlp_tc<true, 4, true, 1>, &k_mlp_tc<true, 4, true, 2>}};
constexpr int kNumVariants = sizeof(kVariants) / sizeof(kVariants[0]);
static_assert(kNumVariants == MCL_MLP_VARIANTS, "variant table");
// untuned choice per precision: 8 epilogue warps per tile, staggered tiles
// (the autotuner's pick on GB300 at 0.3 M and 2.5 M rows: BF16 about 1.5 %,
// FP8 about 7 % faster than with 4 warps).
constexpr int kDefaultVariant[3] = {-1, 12, 5};
// The variant whose launch shape (threads, shared memory) the fused passes'
// kernels (kFusedKernels: staggered, 4 epilogue warps per tile) share:
// checked when the map's forms are set up.
constexpr int kFusedVariant[3] = {-1, 11, 4};

struct TcForm {
    uint8_t* wblocks = nullptr;  // weight blocks in consumption order, 64-byte swizzled
    bool ready = false;
};

struct TcState {
    TcForm bf16, fp8, bf16_split;
    float* aux = nullptr;      // fp32 biases, scales and small heads
    float* ray_bias = nullptr; // [max_rays][128]
    int* abort_flag = nullptr;
    EpiConsts ec;              // copied into every launch's parameter block
    const float* beta_g = nullptr;
    float alpha[8] = {1, 1, 1, 1, 1, 1, 1, 1};
    const float* Wd = nullptr;
    const float* bprime = nullptr;
    float b_sigma = 0.f, b_out[3] = {0.f, 0.f, 0.f};
    float alpha_sigma = 1.f, s_gx = 1.f;
    int n_sm = 0;
    int max_pairs = 0;         // co-resident CTA pairs of the pair kernels
    int variant[3] = {-1, kDefaultVariant[1], kDefaultVariant[2]};   // by precision
    int hold_launches = 0;                 // failure injection: launches left
    unsigned long long hold_wait_ns = 0;   // their wait limit
    float tuned_ms[kNumVariants] = {};                                // last autotune
    bool tuned[3] = {false, false, false};
};

inline uint16_t f2bf(float f) {
    uint32_t u;
    memcpy(&u, &f, 4);
    if ((u & 0x7fffffffu) > 0x7f800000u) return 0x7fc0;  // NaN
    const uint32_t lsb = (u >> 16) & 1u;
    u += 0x7fffu + lsb;                                   // round to nearest even
    return (uint16_t)(u >> 16);
}

inline uint8_t f2e4m3(double f) {
    return (uint8_t)__nv_cvt_float_to_fp8((float)f, __NV_SATFINITE, __NV_E4M3);
}

// Largest |value| of each layer's input over calibration points of a box
// that holds the cameras and the [near, far] sample range of the workloads
// (positions in [-8, 8]^3, unit directions): [0] gamma(x), [l] the output of
// trunk layer l (l = 1..8).  FP64 host forward of the trunk.
void calibrate(const float* const* Wp, const float* const* bp, const int* fin,
               double (&amax)[kDepth + 1]) {
    for (double& a : amax) a = 0.0;
    uint64_t st = 0x9E3779B97F4A7C15ull;
    auto uni = [&]() {  // SplitMix64 -> [0, 1)
        uint64_t z = (st += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        return (double)(z >> 11) * (1.0 / 9007199254740992.0);
    };
    std::vector<double> gx(kGx), h(kWidth + kGx), t(kWidth);
    for (int n = 0; n < 1024; ++n) {
        const double x[3] = {16.0 * uni() - 8.0, 16.0 * uni() - 8.0, 16.0 * uni() - 8.0};
        for (int c = 0; c < 3; ++c) gx[c] = x[c];
        for (int k = 0; k < kLxyz; ++k)
            for (int c = 0; c < 3; ++c) {
                gx[3 + 6 * k + c] = sin(ldexp(x[c], k));
                gx[6 + 6 * k + c] = cos(ldexp(x[c], k));
            }
        for (int i = 0; i < kGx; ++i) amax[0] = fmax(amax[0], fabs(gx[i]));
        for (int i = 0; i < kGx; ++i) h[i] = gx[i];
        for (int l = 0; l < kDepth; ++l) {
            for (int o = 0; o < kWidth; ++o) {
                double sum = bp[l][o];
                const float* w = Wp[l] + (size_t)o * fin[l];
                for (int i = 0; i < fin[l]; ++i) sum += (double)w[i] * h[i];
                t[o] = sum > 0.0 ? sum : 0.0;
                amax[l + 1] = fmax(amax[l + 1], t[o]);
            }
            for (int o = 0; o < kWidth; ++o) h[o] = t[o];
            if (l + 1 == kSkip)
                for (int i = 0; i < kGx; ++i) h[kWidth + i] = gx[i];
        }
    }
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
    // weight of padded layer l (0..8) at output row n, padded input column k
    // ([h, gamma(x)] order for the skip layer; padding columns are 0); layer
    // 8 is the last MMA: rows 0..127 RGB hidden (folded), row 128 density
    auto weight = [&](int l, int n, int k) -> double {
        if (l == 8) {
            if (n < kRgbW) return Wfold[(size_t)n * kWidth + k];
            return n == kRgbW ? (double)Wp[8][k] : 0.0;
        }
        if (k >= fin[l]) return 0.0;
        return (double)Wp[l][(size_t)n * fin[l] + k];
    };
    auto padded_k = [&](int l) { return l == 0 ? kGxPad : (l == kSkip ? kWidth + kGxPad : kWidth); };
    // ---- BF16 weight blocks [256 rows][32 k] in consumption order
    const int nb16 = Form<false>::kBlocks;
    std::vector<uint16_t> blk((size_t)nb16 * 256 * 32, 0);
    int b = 0;
    for (int l = 0; l < kLayers; ++l) {
        const int nrows = (l == 8) ? kRgbW + 1 : kWidth;
        for (int k0 = 0; k0 < padded_k(l); k0 += 32, ++b)
            for (int n = 0; n < nrows; ++n)
                for (int k = 0; k < 32; ++k)
                    blk[((size_t)b * 256 + n) * 32 + k] = f2bf((float)weight(l, n, k0 + k));
    }
    if (b != nb16) return fail(MCL_ERR_UNSUPPORTED, "internal: weight block count %d", b);
    // ---- FP8 form: activation scales from calibration (largest value -> 224,
    //      half the E4M3 range), per-row weight scales (largest |w| -> 448)
    double amax[kDepth + 1];
    calibrate(Wp, bp, fin, amax);
    double sa[kDepth + 1];
    for (int l = 0; l <= kDepth; ++l) sa[l] = 224.0 / (amax[l] > 1e-30 ? amax[l] : 1.0);
    // scale of input column k of layer l
    auto in_scale = [&](int l, int k) -> double {
        if (l == 0) return sa[0];
        if (l == kSkip && k >= kWidth) return sa[0];
        return sa[l];
    };
    const int nb8 = Form<true>::kBlocks;
    std::vector<uint8_t> blk8((size_t)nb8 * 256 * 64, 0);
    std::vector<float> beta((size_t)kDepth * kWidth);
    std::vector<float> alpha_last(kRgbW);
    double alpha_sigma = 1.0;
    b = 0;
    for (int l = 0; l < kLayers; ++l) {
        const int nrows = (l == 8) ? kRgbW + 1 : kWidth;
        const int K = padded_k(l);
        // operand scale of layer l's accumulator: the layer's main input
        const double s_acc = (l == 0) ? sa[0] : sa[l];
        // weight scales: one per trunk layer (the epilogue multiplies by a
        // single alpha), one per row of the last layer (applied in FP32)
        std::vector<double> sw(nrows, 1.0);
        double lmax = 0.0;
        for (int n = 0; n < nrows; ++n) {
            double mx = 0.0;
            for (int k = 0; k < K; ++k) mx = fmax(mx, fabs(weight(l, n, k) * s_acc / in_scale(l, k)));
            sw[n] = mx > 0.0 ? 448.0 / mx : 1.0;
            lmax = fmax(lmax, mx);
        }
        if (l < kDepth)
            for (int n = 0; n < nrows; ++n) sw[n] = lmax > 0.0 ? 448.0 / lmax : 1.0;
        for (int k0 = 0; k0 < K; k0 += 64, ++b)
            for (int n = 0; n < nrows; ++n)
                for (int k = 0; k < 64; ++k) {
                    const int kk = k0 + k;
                    blk8[((size_t)b * 256 + n) * 64 + k] =
                        f2e4m3(weight(l, n, kk) * sw[n] * s_acc / in_scale(l, kk));
                }
        if (l < kDepth) {
            // next input scale sa[l + 1]; accumulator = s_acc sw (W . x)
            st->alpha[l] = (float)(sa[l + 1] / (s_acc * sw[0]));
            for (int n = 0; n < kWidth; ++n) beta[(size_t)l * kWidth + n] = (float)(bp[l][n] * sa[l + 1]);
        } else {
            for (int n = 0; n < kRgbW; ++n) alpha_last[n] = (float)(1.0 / (s_acc * sw[n]));
            alpha_sigma = 1.0 / (s_acc * sw[kRgbW]);
        }
    }
    if (b != nb8) return fail(MCL_ERR_UNSUPPORTED, "internal: FP8 weight block count %d", b);
    // ---- per-column epilogue constants (parameter block): BF16 trunk
    //      biases as pairs [8][128], FP8 beta [8][256], FP8 alpha of the RGB
    //      hidden layer [128], w_out [3][128]
    for (int l = 0; l < kDepth; ++l)
        for (int j = 0; j < kWidth / 2; ++j)
            st->ec.bias2[l][j] = (uint32_t)f2bf(bp[l][2 * j]) | ((uint32_t)f2bf(bp[l][2 * j + 1]) << 16);
    for (int l = 0; l < kDepth; ++l)
        for (int n = 0; n < kWidth; ++n) st->ec.beta[l][n] = beta[(size_t)l * kWidth + n];
    for (int n = 0; n < kRgbW; ++n) st->ec.alpha_last[n] = alpha_last[n];
    for (int c = 0; c < 3; ++c)
        for (int n = 0; n < kRgbW; ++n) st->ec.w_out[c][n] = Wp[11][(size_t)c * kRgbW + n];
    // ---- aux (device): FP8 beta [8][256], W_d transposed [27][128], b' [128]
    //      of the per-ray colour bias
    std::vector<float> aux;
    const size_t o_beta = aux.size();
    aux.insert(aux.end(), beta.begin(), beta.end());
    const size_t o_wd = aux.size();
    for (int i = 0; i < kGd; ++i)
        for (int o = 0; o < kRgbW; ++o) aux.push_back(Wp[10][(size_t)o * fin[10] + kWidth + i]);
    const size_t o_bp = aux.size();
    for (int o = 0; o < kRgbW; ++o) aux.push_back((float)bfold[o]);
    st->b_sigma = bp[8][0];
    for (int c = 0; c < 3; ++c) st->b_out[c] = bp[11][c];
    st->alpha_sigma = (float)alpha_sigma;
    st->s_gx = (float)sa[0];

    // blocks of 256 rows x 64 bytes are stored as the 64-byte swizzle lays
    // them out in shared memory, so one contiguous bulk copy fills a stage
    auto swizzle = [](const uint8_t* src, size_t n_blocks) {
        std::vector<uint8_t> out(n_blocks * kStageBytes);
        for (size_t b = 0; b < n_blocks; ++b)
            for (uint32_t r = 0; r < 256; ++r)
                for (uint32_t c = 0; c < 64; ++c)
                    out[b * kStageBytes + sw64_offset(r, c)] = src[b * kStageBytes + r * 64 + c];
        return out;
    };
    const std::vector<uint8_t> sw16 = swizzle(reinterpret_cast<const uint8_t*>(blk.data()), nb16);
    // split-schedule BF16 blocks: [128 output rows x 64 k] per (layer, half,
    // K chunk), 128-byte rows in the 128-byte swizzle; the last layer's half
    // 1 holds the density head in its row 0
    std::vector<uint8_t> spl((size_t)nb16 * kStageBytes, 0);
    {
        size_t bi = 0;
        for (int l = 0; l < kLayers; ++l)
            for (int h = 0; h < 2; ++h)
                for (int k0 = 0; k0 < padded_k(l); k0 += 64, ++bi)
                    for (int n = 0; n < 128; ++n) {
                        const int row = h * 128 + n;
                        if (l == 8 && h == 1 && n > 0) continue;
                        for (int k = 0; k < 64; ++k) {
                            const uint16_t w = f2bf((float)weight(l, row, k0 + k));
                            const uint32_t byte = (uint32_t)n * 128u + (uint32_t)k * 2u;
                            const uint32_t off = byte ^ (((byte >> 7) & 7u) << 4);
                            spl[bi * kStageBytes + off] = (uint8_t)(w & 0xFF);
                            spl[bi * kStageBytes + off + 1] = (uint8_t)(w >> 8);
                        }
                    }
        if (bi != (size_t)nb16) return fail(MCL_ERR_UNSUPPORTED, "internal: split block count %zu", bi);
    }
    const std::vector<uint8_t> sw8 = swizzle(blk8.data(), nb8);
    int rc;
    if ((rc = cuda_check(cudaMalloc(&st->bf16_split.wblocks, spl.size()), "cudaMalloc(split weights)")) ||
        (rc = cuda_check(cudaMemcpy(st->bf16_split.wblocks, spl.data(), spl.size(),
                                    cudaMemcpyHostToDevice),
                         "upload split weights")) ||
        (rc = cuda_check(cudaMalloc(&st->bf16.wblocks, sw16.size()), "cudaMalloc(tc weights)")) ||
        (rc = cuda_check(cudaMemcpy(st->bf16.wblocks, sw16.data(), sw16.size(), cudaMemcpyHostToDevice),
                         "upload tc weights")) ||
        (rc = cuda_check(cudaMalloc(&st->fp8.wblocks, sw8.size()), "cudaMalloc(fp8 weights)")) ||
        (rc = cuda_check(cudaMemcpy(st->fp8.wblocks, sw8.data(), sw8.size(), cudaMemcpyHostToDevice),
                         "upload fp8 weights")) ||
        (rc = cuda_check(cudaMalloc(&st->aux, aux.size() * 4), "cudaMalloc(tc aux)")) ||
        (rc = cuda_check(cudaMemcpy(st->aux, aux.data(), aux.size() * 4, cudaMemcpyHostToDevice),
                         "upload tc aux")) ||
        (rc = cuda_check(cudaMalloc(&st->ray_bias, (size_t)m->cfg.max_rays * 128 * 4), "ray bias")) ||
        (rc = cuda_check(cudaMalloc(&st->abort_flag, sizeof(int)), "abort flag")))
        return rc;
    st->beta_g = st->aux + o_beta;
    st->Wd = st->aux + o_wd;
    st->bprime = st->aux + o_bp;

    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&st->n_sm, cudaDevAttrMultiProcessorCount, dev);
    int major = 0, minor = 0;
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
    cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
    if (major != 10 || minor != 3) return MCL_OK;  // kernels are built for sm_103a only
    for (const TcVariant& v : kVariants)
        if ((rc = cuda_check(cudaFuncSetAttribute(v.fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                  (int)v.smem),
                             "smem attribute")))
            return rc;
    // the fused kernels launch with their shape variant's threads and smem
    if (kVariants[kFusedVariant[MCL_PREC_BF16]].fn != &k_mlp_tc<false, 4, true> ||
        kVariants[kFusedVariant[MCL_PREC_FP8]].fn != &k_mlp_tc<true, 4, true>)
        return fail(MCL_ERR_UNSUPPORTED, "fused-pass launch shape: variant table mismatch");
    for (int f8 = 0; f8 < 2; ++f8)
        for (int mode = 0; mode < 2; ++mode)
            if ((rc = cuda_check(cudaFuncSetAttribute(kFusedKernels[f8][mode],
                                                      cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                      (int)kVariants[kFusedVariant[f8 + 1]].smem),
                                 "smem attribute (fused)")))
                return rc;
    {
        // persistent grid of the pair kernels: every pair resident at once
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)(st->n_sm & ~1));
        cfg.blockDim = dim3(kPairThreads);
        cfg.dynamicSmemBytes = PairForm<false>::kSmemBytes;
        if ((rc = cuda_check(cudaOccupancyMaxActiveClusters(&st->max_pairs, &k_mlp_tc2<false, false>, &cfg),
                             "pair occupancy")))
            return rc;
        st->max_pairs = std::min(st->max_pairs, st->n_sm / 2);
        if (st->max_pairs < 1) return fail(MCL_ERR_UNSUPPORTED, "no CTA pair fits on an SM pair");
    }
    st->bf16.ready = st->fp8.ready = st->bf16_split.ready = true;
    return MCL_OK;
}

void mlp_tc_free(mcl_map* m) {
    TcState* st = (TcState*)m->tc_aux;
    if (!st) return;
    if (st->bf16.wblocks) cudaFree(st->bf16.wblocks);
    if (st->fp8.wblocks) cudaFree(st->fp8.wblocks);
    if (st->bf16_split.wblocks) cudaFree(st->bf16_split.wblocks);
    if (st->aux) cudaFree(st->aux);
    if (st->ray_bias) cudaFree(st->ray_bias);
    if (st->abort_flag) cudaFree(st->abort_flag);
    delete st;
    m->tc_aux = nullptr;
}

bool mlp_tc_available(const mcl_map* m, int precision) {
    const TcState* st = (const TcState*)m->tc_aux;
    if (!st) return false;
    if (precision == MCL_PREC_BF16) return st->bf16.ready;
    if (precision == MCL_PREC_FP8) return st->fp8.ready;
    return false;
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

static cudaError_t mlp_tc_variant(mcl_map* m, int precision, int variant, const Ray* rays,
                                  const float* z, int S, int n_rays, const int* rows_dev,
                                  float4* out, cudaStream_t s, const FuseArgs* fuse = nullptr);

// The fused ray epilogues work on whole rays inside a 128-row tile (S divides
// 128) and stage a tile's samples in its activation buffer (see warp_part);
// the first-pass samples of a tile's rays are prefetched two per row thread.
bool mlp_tc_can_fuse(int mode, int S, int S1) {
    // whole rays per tile, at most four (one compositing warp each), each
    // ray's staged samples within its warp's 4 KB part of the buffer
    if (S < 32 || S > 128 || 128 % S != 0) return false;
    const int R = 128 / S;
    if (mode == 1) return 3 * S + 1 <= 1024;
    if (mode == 2) return S1 >= 0 && S1 <= kMaxCoarse && R * S1 <= 256 && 5 * (S + S1) <= 1024;
    return false;
}

cudaError_t mlp_tc(mcl_map* m, int precision, const Ray* rays, const float* gd, const float* z,
                   int S, int n_rays, const int* rows_dev, float4* out, cudaStream_t s,
                   const FuseArgs* fuse) {
    (void)gd;
    return mlp_tc_variant(m, precision, -1, rays, z, S, n_rays, rows_dev, out, s, fuse);
}

static cudaError_t mlp_tc_variant(mcl_map* m, int precision, int variant, const Ray* rays,
                                  const float* z, int S, int n_rays, const int* rows_dev,
                                  float4* out, cudaStream_t s, const FuseArgs* fuse) {
    TcState* st = (TcState*)m->tc_aux;
    if (!mlp_tc_available(m, precision)) return cudaErrorNotSupported;
    Params p;
    memset(&p, 0, sizeof(p));
    int vi = variant >= 0 ? variant : st->variant[precision];
    // fused passes run on their own instantiations of the staggered
    // single-CTA kernel with 4 epilogue warps per tile (kFusedKernels)
    if (fuse) vi = kFusedVariant[precision];
    p.wblocks = precision == MCL_PREC_FP8 ? st->fp8.wblocks
                : kVariants[vi].fn == &k_mlp_tc_split ? st->bf16_split.wblocks
                                                      : st->bf16.wblocks;
    p.rays = rays;
    p.z = z;
    p.S = S;
    p.M = (long long)n_rays * S;
    p.n_pairs = (p.M + 255) / 256;
    p.M_dev = rows_dev;
    for (int l = 0; l < 8; ++l) p.alpha[l] = st->alpha[l];
    p.ec = st->ec;
    p.beta_g = st->beta_g;
    p.alpha_sigma = st->alpha_sigma;
    p.s_gx = st->s_gx;
    p.b_sigma = st->b_sigma;
    p.ray_bias = st->ray_bias;
    p.b_out0 = st->b_out[0];
    p.b_out1 = st->b_out[1];
    p.b_out2 = st->b_out[2];
    p.out = out;
    if (fuse) {
        // the first pass's tail writes at most 4 samples per lane (the
        // importance samples are the last pass's S <= 128 samples)
        if (fuse->mode == 1 && (fuse->nf_out < 1 || fuse->nf_out > 128)) return cudaErrorInvalidValue;
        p.fuse = fuse->mode;
        p.nf_out = fuse->nf_out;
        p.z_out = fuse->z_out;
        p.z_first = fuse->z_first;
        p.out_first = fuse->out_first;
        p.S1 = fuse->S1;
        p.eq5_alpha = fuse->alpha;
        p.tau = fuse->tau;
        p.use_rej = fuse->use_rej;
        p.obs = fuse->obs;
        p.e_ray = fuse->e_ray;
        p.rgb_out = fuse->rgb_out;
        p.E_out = fuse->E_out;
        p.F_out = fuse->F_out;
        p.zt_out = fuse->zt_out;
        p.zo_out = fuse->zo_out;
    }
    p.abort_flag = st->abort_flag;
    p.status_code = &m->status->code;
    p.wait_ns = kWaitNs;
    p.hold_weights = 0;
    int vsel = vi;
    if (st->hold_launches > 0) {
        // failure injection: the untuned single-CTA kernel with its weight
        // stream held and a short wait limit
        --st->hold_launches;
        p.hold_weights = 1;
        p.wait_ns = st->hold_wait_ns;
        vsel = fuse ? kFusedVariant[precision] : kDefaultVariant[precision];
        p.wblocks = precision == MCL_PREC_FP8 ? st->fp8.wblocks : st->bf16.wblocks;
    }
    cudaError_t e = cudaMemsetAsync(st->abort_flag, 0, sizeof(int), s);
    if (e) return e;
    // persistent grid: one CTA per SM at most, one per work unit (a pair of
    // tiles, a single tile for the pipelined kernel, 512 rows for a CTA pair)
    const TcVariant& v = kVariants[vsel];
    void (*fn)(Params) = fuse ? kFusedKernels[precision == MCL_PREC_FP8][fuse->mode - 1] : v.fn;
    long long grid;
    if (v.cluster == 2) {
        const long long units = (p.M + 511) / 512;
        grid = 2 * (units < st->max_pairs ? units : st->max_pairs);
    } else {
        const long long units = v.fn == &k_mlp_tc_pipe ? (p.M + 127) / 128 : p.n_pairs;
        grid = units < st->n_sm ? units : st->n_sm;
    }
    note_launch();
    fn<<<(unsigned)grid, v.threads, v.smem, s>>>(p);
    return cudaGetLastError();
}

// Synthetic inputs for timing the kernel variants: rays from points in
// [-1, 1]^3 in unit directions, z uniform in [2, 6], gamma(d) zero.
__global__ void k_tune_inputs(Ray* __restrict__ rays, float* __restrict__ z,
                              float* __restrict__ gd, int n_rays, int S) {
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < (long)n_rays * S) {
        uint32_t h = (uint32_t)t * 2654435761u + 12345u;
        h ^= h >> 15; h *= 0x2c1b3c6du; h ^= h >> 12;
        z[t] = 2.0f + 4.0f * (float)(h >> 8) * (1.0f / 16777216.0f);
    }
    if (t < n_rays) {
        uint32_t h = (uint32_t)t * 0x9E3779B9u + 777u;
        float v[6];
        for (int i = 0; i < 6; ++i) {
            h ^= h >> 15; h *= 0x2c1b3c6du; h ^= h >> 12;
            v[i] = 2.0f * (float)(h >> 8) * (1.0f / 16777216.0f) - 1.0f;
        }
        const float n = rsqrtf(v[3] * v[3] + v[4] * v[4] + v[5] * v[5] + 1e-6f);
        Ray r{};
        r.ox = v[0]; r.oy = v[1]; r.oz = v[2];
        r.dx = v[3] * n; r.dy = v[4] * n; r.dz = v[5] * n;
        r.dnorm = 1.0f;
        rays[t] = r;
        for (int i = 0; i < kGdPad; ++i) gd[(long)t * kGdPad + i] = 0.0f;
    }
}

int mlp_tc_set_variant(mcl_map* m, int precision, int variant) {
    TcState* st = (TcState*)m->tc_aux;
    if (!mlp_tc_available(m, precision)) return fail(MCL_ERR_UNSUPPORTED, "precision %d unavailable", precision);
    if (variant < 0 || variant >= kNumVariants || kVariants[variant].precision != precision)
        return fail(MCL_ERR_ARG, "variant %d is not a variant of precision %d", variant, precision);
    st->variant[precision] = variant;
    return MCL_OK;
}

int mlp_tc_autotune(mcl_map* m, int precision, long long rows, int* chosen, float* ms_out,
                    cudaStream_t s) {
    TcState* st = (TcState*)m->tc_aux;
    if (!mlp_tc_available(m, precision)) return fail(MCL_ERR_UNSUPPORTED, "precision %d unavailable", precision);
    const int S = std::min(64, m->cfg.max_samples);
    const long long cap = (long long)m->cfg.max_rays * S;
    if (rows < 256 || rows > cap) return fail(MCL_ERR_ARG, "autotune rows %lld not in [256, %lld]", rows, cap);
    const int n_rays = (int)((rows + S - 1) / S);
    int rc;
    note_launch();
    k_tune_inputs<<<(unsigned)(((long)n_rays * S + 255) / 256), 256, 0, s>>>(m->rays, m->zc, m->gd,
                                                                             n_rays, S);
    if ((rc = cuda_check(cudaGetLastError(), "tune inputs")) ||
        (rc = cuda_check(mlp_tc_ray_bias(m, m->gd, n_rays, nullptr, s), "tune ray bias")))
        return rc;
    cudaEvent_t a = nullptr, b = nullptr;
    if ((rc = cuda_check(cudaEventCreate(&a), "event")) || (rc = cuda_check(cudaEventCreate(&b), "event")))
        return rc;
    int best = -1;
    float best_ms = 0.f;
    for (int v = 0; v < kNumVariants && !rc; ++v) {
        if (ms_out) ms_out[v] = -1.f;
        if (kVariants[v].precision != precision) continue;
        float tot = 0.f;
        for (int rep = 0; rep < 4 && !rc; ++rep) {
            rc = cuda_check(cudaEventRecord(a, s), "event");
            if (!rc) rc = cuda_check(mlp_tc_variant(m, precision, v, m->rays, m->zc, S, n_rays, nullptr,
                                                    m->out_c, s), "tune launch");
            if (!rc) rc = cuda_check(cudaEventRecord(b, s), "event");
            if (!rc) rc = cuda_check(cudaEventSynchronize(b), "event sync");
            float ms = 0.f;
            if (!rc) rc = cuda_check(cudaEventElapsedTime(&ms, a, b), "elapsed");
            if (rep > 0) tot += ms;       // the first launch warms caches
        }
        if (rc) break;
        const float mean = tot / 3.f;
        st->tuned_ms[v] = mean;
        if (ms_out) ms_out[v] = mean;
        if (best < 0 || mean < best_ms) {
            best = v;
            best_ms = mean;
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (rc) return rc;
    if (m->status) {
        // a timed-out wait inside a trial launch is an error, not a timing
        int code = 0;
        if ((rc = cuda_check(cudaMemcpy(&code, &m->status->code, sizeof(int), cudaMemcpyDeviceToHost),
                             "read status")))
            return rc;
        if (code) return fail(code, "autotune: a trial launch reported error %d", code);
    }
    st->variant[precision] = best;
    st->tuned[precision] = true;
    if (chosen) *chosen = best;
    return MCL_OK;
}

int mlp_tc_hold_weights(mcl_map* m, int n_launches, unsigned long long wait_ns) {
    TcState* st = (TcState*)m->tc_aux;
    if (!st) return fail(MCL_ERR_UNSUPPORTED, "no tensor-core MLP on this map");
    st->hold_launches = n_launches;
    st->hold_wait_ns = wait_ns;
    return MCL_OK;
}

bool mlp_tc_tuned(const mcl_map* m, int precision) {
    const TcState* st = (const TcState*)m->tc_aux;
    return st && precision >= 0 && precision < 3 && st->tuned[precision];
}

}  // namespace mcl
