// mlp_fp32.cu -- the plain FP32 form of the NeRF MLP: positional encoding,
// one SIMT FP32 GEMM launch per layer with bias and ReLU, and two row-wise
// head kernels.  Activations live in HBM (chunks of rows), so this form is
// also the unfused comparison point for the tensor-core path.
#include <math.h>

#include "internal.cuh"

namespace mcl {

// gamma(x) of x = o + z d for rows [r0, r0 + n) of a pass with S samples per
// ray: [x, sin(2^k x), cos(2^k x)]_{k<10}, padded with a zero to 64.  x and
// the arguments 2^k x are formed in FP64 and reduced modulo 2 pi there, so the
// sines carry FP32 error rather than FP32 error of x amplified by 2^9.
// rows_dev (optional): rows of the pass in device memory; rows at or beyond
// it are skipped (every kernel of this file).
__device__ __forceinline__ int rows_in_chunk(int n, long r0, const int* rows_dev) {
    if (!rows_dev) return n;
    const long left = (long)*rows_dev - r0;
    return left < 0 ? 0 : (left < n ? (int)left : n);
}

__global__ void k_pe_xyz(const Ray* __restrict__ rays, const float* __restrict__ z, int S, long r0,
                         int n, const int* __restrict__ rows_dev, float* __restrict__ gx) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= rows_in_chunk(n, r0, rows_dev)) return;
    const long row = r0 + t;
    const Ray ray = rays[row / S];
    const double zz = (double)z[row];
    const double p[3] = {(double)ray.ox + zz * ((double)ray.dx + (double)ray.lx),
                         (double)ray.oy + zz * ((double)ray.dy + (double)ray.ly),
                         (double)ray.oz + zz * ((double)ray.dz + (double)ray.lz)};
    const double two_pi = 6.283185307179586476925286766559;
    const double inv_two_pi = 0.15915494309189533576888376337251;
    float v[kGxPad];
    v[0] = (float)p[0]; v[1] = (float)p[1]; v[2] = (float)p[2];
#pragma unroll
    for (int k = 0; k < kLxyz; ++k) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            // n = rint(a / 2 pi) from a product with 1 / (2 pi) (an n off by
            // one leaves rr one period further, still within 2 pi of 0);
            // a - 2 pi n is formed with a single rounding in FP64
            const double a = ldexp(p[c], k);
            const double rr = fma(-two_pi, rint(a * inv_two_pi), a);
            float sn, cs;
            sincosf((float)rr, &sn, &cs);
            v[3 + 6 * k + c] = sn;
            v[6 + 6 * k + c] = cs;
        }
    }
    v[kGx] = 0.f;
    // the row as 16-byte stores (rows are 256 bytes, 16-byte aligned)
    float4* g = reinterpret_cast<float4*>(gx + (size_t)t * kGxPad);
#pragma unroll
    for (int q = 0; q < kGxPad / 4; ++q) g[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
}

// C[M, N] = act([A1 | A2] W^T + b).  A1: [M, K1] (lda1); A2 row for output
// row r is (r + a2_off) / a2_div (lda2, K2 columns); W: [N, K1 + K2]
// row-major.  K1, K2 multiples of 16, N a multiple of 128.  128x128 tile,
// 256 threads, 8x8 outputs per thread.  Shared memory holds two k-tiles of
// 16: while the threads multiply one, the next is loaded from global memory
// into registers and stored into the other buffer, so each k-tile costs one
// barrier.  Every output accumulates its products in ascending k with one
// FMA each.
template <bool RELU>
__global__ __launch_bounds__(256, 2) void k_sgemm(const float* __restrict__ A1, int lda1, int K1,
                                               const float* __restrict__ A2, int lda2, int K2,
                                               long a2_off, int a2_div,
                                               const float* __restrict__ W,
                                               const float* __restrict__ bias,
                                               float* __restrict__ C, int ldc, int M,
                                               const int* __restrict__ rows_dev, long r0) {
    constexpr int BM = 128, BN = 128, BK = 16, PAD = 4;
    __shared__ __align__(16) float As[2][BK][BM + PAD];
    __shared__ __align__(16) float Bs[2][BK][BN + PAD];
    const int tid = threadIdx.x;
    const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
    M = rows_in_chunk(M, r0, rows_dev);
    if (m0 >= M) return;
    const int K = K1 + K2;
    const int lr = tid >> 2, lk = (tid & 3) << 2;
    const int tx = tid & 15, ty = tid >> 4;
    // acc[p][j]: rows 2p, 2p + 1 of the thread's 8 x 8 outputs, column j;
    // each pair is updated by one packed FP32 FMA (two independent FMAs with
    // round-to-nearest, the arithmetic of two fmaf calls), which halves the
    // instructions of this issue-bound loop
    float2 acc[4][8];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = make_float2(0.f, 0.f);
    float4 ra[2], rb[2];
    auto load = [&](int k0) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int row = m0 + lr + h * 64;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (row < M) {
                if (k0 < K1) {
                    v = *reinterpret_cast<const float4*>(A1 + (size_t)row * lda1 + k0 + lk);
                } else {
                    const long r2 = ((long)row + a2_off) / a2_div;
                    v = *reinterpret_cast<const float4*>(A2 + (size_t)r2 * lda2 + (k0 - K1) + lk);
                }
            }
            ra[h] = v;
            const int nr = n0 + lr + h * 64;
            rb[h] = *reinterpret_cast<const float4*>(W + (size_t)nr * K + k0 + lk);
        }
    };
    auto store = [&](int buf) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int c = lr + h * 64;
            As[buf][lk + 0][c] = ra[h].x; As[buf][lk + 1][c] = ra[h].y;
            As[buf][lk + 2][c] = ra[h].z; As[buf][lk + 3][c] = ra[h].w;
            Bs[buf][lk + 0][c] = rb[h].x; Bs[buf][lk + 1][c] = rb[h].y;
            Bs[buf][lk + 2][c] = rb[h].z; Bs[buf][lk + 3][c] = rb[h].w;
        }
    };
    load(0);
    store(0);
    __syncthreads();
    int cur = 0;
    for (int k0 = 0; k0 < K; k0 += BK) {
        const bool more = k0 + BK < K;
        if (more) load(k0 + BK);
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            const float4 a0 = *reinterpret_cast<const float4*>(&As[cur][kk][ty * 4]);
            const float4 a1 = *reinterpret_cast<const float4*>(&As[cur][kk][64 + ty * 4]);
            const float4 b0 = *reinterpret_cast<const float4*>(&Bs[cur][kk][tx * 4]);
            const float4 b1 = *reinterpret_cast<const float4*>(&Bs[cur][kk][64 + tx * 4]);
            const float2 a[4] = {make_float2(a0.x, a0.y), make_float2(a0.z, a0.w),
                                 make_float2(a1.x, a1.y), make_float2(a1.z, a1.w)};
            const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const float2 bj = make_float2(b[j], b[j]);
#pragma unroll
                for (int i = 0; i < 4; ++i) acc[i][j] = __ffma2_rn(a[i], bj, acc[i][j]);
            }
        }
        if (more) {
            // the other buffer was last read before the previous barrier
            store(cur ^ 1);
            __syncthreads();
            cur ^= 1;
        }
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int row = m0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + (i - 4));
        if (row >= M) continue;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int col = n0 + h * 64 + tx * 4;
            float4 v;
            const float2* ar = acc[i >> 1];
            v.x = ((i & 1) ? ar[h * 4 + 0].y : ar[h * 4 + 0].x) + bias[col + 0];
            v.y = ((i & 1) ? ar[h * 4 + 1].y : ar[h * 4 + 1].x) + bias[col + 1];
            v.z = ((i & 1) ? ar[h * 4 + 2].y : ar[h * 4 + 2].x) + bias[col + 2];
            v.w = ((i & 1) ? ar[h * 4 + 3].y : ar[h * 4 + 3].x) + bias[col + 3];
            if (RELU) {
                v.x = fmaxf(v.x, 0.f); v.y = fmaxf(v.y, 0.f);
                v.z = fmaxf(v.z, 0.f); v.w = fmaxf(v.w, 0.f);
            }
            *reinterpret_cast<float4*>(C + (size_t)row * ldc + col) = v;
        }
    }
}

// sigma_raw = w_sigma . h + b_sigma, one half-warp per row: lane l of the
// half takes the 16-byte groups l, l + 16, l + 32, l + 48 of the row (each
// load instruction of the warp reads two rows' 256 contiguous bytes), then a
// butterfly over the 16 lanes.
__global__ void k_sigma_head(const float* __restrict__ h, int ldh, const float* __restrict__ w,
                             const float* __restrict__ b, int n, const int* __restrict__ rows_dev,
                             long r0, float4* __restrict__ out) {
    const int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 4;
    const int l = threadIdx.x & 15;
    const bool live = row < rows_in_chunk(n, r0, rows_dev);
    float s = 0.f;
    if (live) {
        const float4* x = reinterpret_cast<const float4*>(h + (size_t)row * ldh);
        const float4* w4 = reinterpret_cast<const float4*>(w);
#pragma unroll
        for (int q = 0; q < kWidth / 64; ++q) {
            const float4 xv = x[l + 16 * q], wv = __ldg(w4 + l + 16 * q);
            s = fmaf(wv.x, xv.x, s);
            s = fmaf(wv.y, xv.y, s);
            s = fmaf(wv.z, xv.z, s);
            s = fmaf(wv.w, xv.w, s);
        }
    }
    for (int o = 8; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (live && l == 0) reinterpret_cast<float*>(out)[4 * (size_t)row] = s + b[0];
}

// rgb = sigmoid(W_out h + b_out), one half-warp per row (the 128 hidden
// values as 16-byte groups l and l + 16 of lane l).
__global__ void k_rgb_head(const float* __restrict__ h, int ldh, const float* __restrict__ W,
                           const float* __restrict__ b, int n, const int* __restrict__ rows_dev,
                           long r0, float4* __restrict__ out) {
    const int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 4;
    const int l = threadIdx.x & 15;
    const bool live = row < rows_in_chunk(n, r0, rows_dev);
    float s[3] = {0.f, 0.f, 0.f};
    if (live) {
        const float4* x = reinterpret_cast<const float4*>(h + (size_t)row * ldh);
        const float4* W4 = reinterpret_cast<const float4*>(W);
#pragma unroll
        for (int q = 0; q < kRgbW / 64; ++q) {
            const float4 xv = x[l + 16 * q];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const float4 wv = __ldg(W4 + c * (kRgbW / 4) + l + 16 * q);
                s[c] = fmaf(wv.x, xv.x, s[c]);
                s[c] = fmaf(wv.y, xv.y, s[c]);
                s[c] = fmaf(wv.z, xv.z, s[c]);
                s[c] = fmaf(wv.w, xv.w, s[c]);
            }
        }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c)
        for (int o = 8; o > 0; o >>= 1) s[c] += __shfl_xor_sync(0xffffffffu, s[c], o);
    if (live && l == 0) {
        float* dst = reinterpret_cast<float*>(out) + 4 * (size_t)row;
#pragma unroll
        for (int c = 0; c < 3; ++c) dst[1 + c] = 1.0f / (1.0f + expf(-(s[c] + b[c])));
    }
}

static cudaError_t gemm(const float* A1, int lda1, int K1, const float* A2, int lda2, int K2,
                        long a2_off, int a2_div, const LayerF32& L, float* C, int ldc, int M,
                        bool relu, const int* rows_dev, long r0, cudaStream_t s);

cudaError_t fp32_gemm(const float* A1, int lda1, int K1, const float* A2, int lda2, int K2,
                      long a2_off, int a2_div, const float* W, const float* bias, int n_out,
                      float* C, int ldc, int M, bool relu, cudaStream_t s) {
    LayerF32 L{W, bias, n_out, K1 + K2};
    return gemm(A1, lda1, K1, A2, lda2, K2, a2_off, a2_div, L, C, ldc, M, relu, nullptr, 0, s);
}

cudaError_t fp32_pe(const Ray* rays, const float* z, int n, float* gx, cudaStream_t s) {
    note_launch();
    k_pe_xyz<<<(n + 127) / 128, 128, 0, s>>>(rays, z, 1, 0, n, nullptr, gx);
    return cudaGetLastError();
}

cudaError_t fp32_heads(const float* h, const LayerF32& sigma, const float* hid, const LayerF32& rgb,
                       int n, float4* out, cudaStream_t s) {
    note_launch(2);
    k_sigma_head<<<(n * 16 + 255) / 256, 256, 0, s>>>(h, kWidth, sigma.W, sigma.b, n, nullptr, 0, out);
    k_rgb_head<<<(n * 16 + 255) / 256, 256, 0, s>>>(hid, kWidth, rgb.W, rgb.b, n, nullptr, 0, out);
    return cudaGetLastError();
}

static cudaError_t gemm(const float* A1, int lda1, int K1, const float* A2, int lda2, int K2,
                        long a2_off, int a2_div, const LayerF32& L, float* C, int ldc, int M,
                        bool relu, const int* rows_dev, long r0, cudaStream_t s) {
    dim3 grid((M + 127) / 128, L.n / 128);
    note_launch();
    if (relu)
        k_sgemm<true><<<grid, 256, 0, s>>>(A1, lda1, K1, A2, lda2, K2, a2_off, a2_div, L.W, L.b, C,
                                           ldc, M, rows_dev, r0);
    else
        k_sgemm<false><<<grid, 256, 0, s>>>(A1, lda1, K1, A2, lda2, K2, a2_off, a2_div, L.W, L.b, C,
                                            ldc, M, rows_dev, r0);
    return cudaGetLastError();
}

cudaError_t mlp_fp32(mcl_map* m, const Ray* rays, const float* gd, const float* z, int S,
                     int n_rays, float4* out, cudaStream_t s, const int* rows_dev) {
    const long rows = (long)n_rays * S;
    cudaError_t e = cudaSuccess;
    for (long r0 = 0; r0 < rows; r0 += m->chunk_rows) {
        const int n = (int)((rows - r0) < m->chunk_rows ? (rows - r0) : m->chunk_rows);
        note_launch();
        k_pe_xyz<<<(n + 127) / 128, 128, 0, s>>>(rays, z, S, r0, n, rows_dev, m->gxbuf);
        float* a = m->act0;
        float* b = m->act1;
        // trunk layer 1 reads gamma(x)
        if ((e = gemm(m->gxbuf, kGxPad, kGxPad, nullptr, 0, 0, 0, 1, m->L[0], a, kWidth, n, true,
                      rows_dev, r0, s)))
            return e;
        for (int l = 1; l < kDepth; ++l) {
            if (l == kSkip) {
                // layer skip+1 reads [h_skip, gamma(x)]
                e = gemm(a, kWidth, kWidth, m->gxbuf, kGxPad, kGxPad, 0, 1, m->L[l], b, kWidth, n,
                         true, rows_dev, r0, s);
            } else {
                e = gemm(a, kWidth, kWidth, nullptr, 0, 0, 0, 1, m->L[l], b, kWidth, n, true,
                         rows_dev, r0, s);
            }
            if (e) return e;
            float* t = a; a = b; b = t;
        }
        // a = trunk output
        note_launch();
        k_sigma_head<<<(n * 16 + 255) / 256, 256, 0, s>>>(a, kWidth, m->L[8].W, m->L[8].b, n,
                                                          rows_dev, r0, out + r0);
        if ((e = gemm(a, kWidth, kWidth, nullptr, 0, 0, 0, 1, m->L[9], b, kWidth, n, false,
                      rows_dev, r0, s)))
            return e;
        // rgb hidden reads [feature, gamma(d)], gamma(d) row = ray = (r0 + r) / S
        if ((e = gemm(b, kWidth, kWidth, gd, kGdPad, kGdPad, r0, S, m->L[10], a, kWidth, n, true,
                      rows_dev, r0, s)))
            return e;
        note_launch();
        k_rgb_head<<<(n * 16 + 255) / 256, 256, 0, s>>>(a, kWidth, m->L[11].W, m->L[11].b, n,
                                                        rows_dev, r0, out + r0);
        if ((e = cudaGetLastError())) return e;
    }
    return cudaSuccess;
}

}  // namespace mcl
