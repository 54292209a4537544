// resample.cu -- systematic resampling on an exact integer CDF, the motion
// (prediction) step, the box downscale of the observed image, and the
// position spread used by the refinement test.
#include <math.h>

#include "internal.cuh"
#include "rng.cuh"

namespace mcl {

typedef unsigned long long u64;
typedef unsigned __int128 u128;

constexpr int kResThreads = 1024;

// Inclusive scan of one u64 per thread across the block; returns the
// inclusive prefix and writes the block total to *total.
__device__ u64 block_scan_u64(u64 v, u64* sh, u64* total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const u64 t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    __syncthreads();
    if (lane == 31) sh[wid] = v;
    __syncthreads();
    if (wid == 0) {
        u64 s = lane < nw ? sh[lane] : 0ull;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const u64 t = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += t;
        }
        if (lane < nw) sh[lane] = s;  // inclusive warp-total prefix
    }
    __syncthreads();
    const u64 before = wid > 0 ? sh[wid - 1] : 0ull;
    *total = sh[nw - 1];
    return v + before;
}

// d_idx[k] = smallest i with C_i N_out 2^53 > (k 2^53 + U) T, where
// q_i = floor(w_i 2^s), s = 50 - e - ceil(log2 N_in), e = exponent of max w,
// C = inclusive prefix of q, T = C_{N_in-1}, U = floor(u0 2^53).
__global__ __launch_bounds__(kResThreads) void k_resample(const double* __restrict__ w, int n_in,
                                                          int n_out, double u0,
                                                          int32_t* __restrict__ idx,
                                                          u64* __restrict__ cdf, Status* status) {
    __shared__ u64 shu[32];
    __shared__ double shd[32];
    __shared__ int bad;
    if (threadIdx.x == 0) bad = 0;
    __syncthreads();
    double mx = 0.0;
    for (int i = threadIdx.x; i < n_in; i += blockDim.x) {
        const double wi = w[i];
        if (!(wi >= 0.0) || isinf(wi)) bad = 1;
        else mx = fmax(mx, wi);
    }
    // block max
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) shd[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = threadIdx.x < (blockDim.x >> 5) ? shd[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
        if (threadIdx.x == 0) shd[0] = v;
    }
    __syncthreads();
    mx = shd[0];
    if (bad || !(mx > 0.0)) {
        for (int k = threadIdx.x; k < n_out; k += blockDim.x) idx[k] = -1;
        if (threadIdx.x == 0) atomicCAS(&status->code, 0, MCL_ERR_DEGENERATE);
        return;
    }
    int e;
    frexp(mx, &e);
    int lg = 0;
    while ((1ll << lg) < (long long)n_in) ++lg;
    const int sh = 50 - e - lg;
    u64 carry = 0;
    for (int base = 0; base < n_in; base += blockDim.x) {
        const int i = base + threadIdx.x;
        const u64 q = i < n_in ? (u64)floor(ldexp(w[i], sh)) : 0ull;
        u64 tot;
        const u64 incl = block_scan_u64(q, shu, &tot);
        if (i < n_in) cdf[i] = carry + incl;
        carry += tot;
        __syncthreads();
    }
    const u64 T = carry;
    const u64 U = (u64)floor(ldexp(u0, 53));
    __syncthreads();
    if (T == 0ull) {
        for (int k = threadIdx.x; k < n_out; k += blockDim.x) idx[k] = -1;
        if (threadIdx.x == 0) atomicCAS(&status->code, 0, MCL_ERR_DEGENERATE);
        return;
    }
    for (int k = threadIdx.x; k < n_out; k += blockDim.x) {
        const u128 rhs = (((u128)(u64)k * T) << 53) + (u128)U * T;
        int lo = 0, hi = n_in - 1;  // answer in [lo, hi]; C_{n_in-1} always satisfies
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            const u128 lhs = ((u128)cdf[mid] * (u64)n_out) << 53;
            if (lhs > rhs) hi = mid;
            else lo = mid + 1;
        }
        idx[k] = lo;
    }
}

cudaError_t launch_resample(const double* w, int n_in, int n_out, double u0, int32_t* idx,
                            unsigned long long* cdf, Status* status, cudaStream_t s) {
    note_launch();
    k_resample<<<1, kResThreads, 0, s>>>(w, n_in, n_out, u0, idx, cdf, status);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Prediction: out_k = in_{idx_k} * Exp(rho, (0, yaw, 0)), FP64 arithmetic.
// SE(3) exponential: R = I + a K + b K^2, t = (I + b K + c K^2) rho with
// K = [omega]x, th = |omega|, a = sin th / th, b = (1 - cos th)/th^2,
// c = (th - sin th)/th^3 (series values below th = 1e-8).
// ---------------------------------------------------------------------------
__global__ void k_predict(const float* __restrict__ in, int n_in, const int32_t* __restrict__ idx, int n,
                          float sigma_t, float sigma_yaw, uint64_t seed, uint64_t ctr,
                          float* __restrict__ out) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int src = idx ? idx[k] : k;
    float* O = out + 12 * (size_t)k;
    if (src < 0 || src >= n_in) {
        for (int c = 0; c < 12; ++c) O[c] = __int_as_float(0x7fc00000);
        return;
    }
    double q[4];
#pragma unroll
    for (int c = 0; c < 4; ++c)
        q[c] = (c < 3 ? (double)sigma_t : (double)sigma_yaw) * cb_normal(seed, ctr, 4ull * k + c);
    const double om[3] = {0.0, q[3], 0.0};
    const double th2 = om[0] * om[0] + om[1] * om[1] + om[2] * om[2];
    const double th = sqrt(th2);
    const double K[9] = {0.0, -om[2], om[1], om[2], 0.0, -om[0], -om[1], om[0], 0.0};
    double K2[9];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c)
            K2[3 * r + c] = K[3 * r] * K[c] + K[3 * r + 1] * K[3 + c] + K[3 * r + 2] * K[6 + c];
    double a, b, cc;
    if (th < 1e-8) {
        a = 1.0; b = 0.5; cc = 1.0 / 6.0;
    } else {
        a = sin(th) / th;
        b = (1.0 - cos(th)) / th2;
        cc = (th - sin(th)) / (th2 * th);
    }
    double E[12];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        double t = 0.0;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const double I = (r == c) ? 1.0 : 0.0;
            E[4 * r + c] = I + a * K[3 * r + c] + b * K2[3 * r + c];
            t += (I + b * K[3 * r + c] + cc * K2[3 * r + c]) * q[c];
        }
        E[4 * r + 3] = t;
    }
    const float* P = in + 12 * (size_t)src;
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            double s = (c == 3) ? (double)P[4 * r + 3] : 0.0;
#pragma unroll
            for (int m = 0; m < 3; ++m) s += (double)P[4 * r + m] * E[4 * m + c];
            O[4 * r + c] = (float)s;
        }
}

cudaError_t launch_predict(const float* in, int n_in, const int32_t* idx, int n_out, float sigma_t,
                           float sigma_yaw, uint64_t seed, uint64_t counter, float* out,
                           cudaStream_t s) {
    note_launch();
    k_predict<<<(n_out + 127) / 128, 128, 0, s>>>(in, n_in, idx, n_out, sigma_t, sigma_yaw, seed, counter,
                                                   out);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Box downscale: one thread per output pixel, f x f block summed in row order.
// ---------------------------------------------------------------------------
__global__ void k_downscale(const float* __restrict__ img, int W, int H, int f,
                            float* __restrict__ out) {
    const int Wl = W / f, Hl = H / f;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= Wl * Hl) return;
    const int u = p % Wl, v = p / Wl;
    float s0 = 0.f, s1 = 0.f, s2 = 0.f;
    for (int dy = 0; dy < f; ++dy) {
        const float* row = img + ((size_t)(v * f + dy) * W + (size_t)u * f) * 3;
        for (int dx = 0; dx < f; ++dx) {
            s0 += row[3 * dx]; s1 += row[3 * dx + 1]; s2 += row[3 * dx + 2];
        }
    }
    const float inv = 1.0f / (float)(f * f);
    out[3 * (size_t)p] = s0 * inv;
    out[3 * (size_t)p + 1] = s1 * inv;
    out[3 * (size_t)p + 2] = s2 * inv;
}

cudaError_t launch_downscale(const float* img, int W, int H, int f, float* out, cudaStream_t s) {
    const int n = (W / f) * (H / f);
    note_launch();
    k_downscale<<<(n + 255) / 256, 256, 0, s>>>(img, W, H, f, out);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Mean position and trace of the population covariance (FP64), one block.
// ---------------------------------------------------------------------------
__global__ __launch_bounds__(1024) void k_spread(const float* __restrict__ P, int N,
                                                 double* __restrict__ out) {
    __shared__ double sh[3][32];
    double m[3] = {0.0, 0.0, 0.0};
    for (int i = threadIdx.x; i < N; i += blockDim.x)
        for (int c = 0; c < 3; ++c) m[c] += (double)P[12 * (size_t)i + 4 * c + 3];
    for (int c = 0; c < 3; ++c) {
        double v = m[c];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0) sh[c][threadIdx.x >> 5] = v;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        for (int c = 0; c < 3; ++c) {
            double v = threadIdx.x < (blockDim.x >> 5) ? sh[c][threadIdx.x] : 0.0;
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (threadIdx.x == 0) sh[c][0] = v / N;
        }
    }
    __syncthreads();
    const double mu[3] = {sh[0][0], sh[1][0], sh[2][0]};
    __syncthreads();
    double t = 0.0;
    for (int i = threadIdx.x; i < N; i += blockDim.x)
        for (int c = 0; c < 3; ++c) {
            const double d = (double)P[12 * (size_t)i + 4 * c + 3] - mu[c];
            t += d * d;
        }
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if ((threadIdx.x & 31) == 0) sh[0][threadIdx.x >> 5] = t;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = threadIdx.x < (blockDim.x >> 5) ? sh[0][threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (threadIdx.x == 0) {
            out[0] = mu[0]; out[1] = mu[1]; out[2] = mu[2];
            out[3] = v / N;
        }
    }
}

cudaError_t launch_position_spread(const float* poses, int N, double* out, cudaStream_t s) {
    note_launch();
    k_spread<<<1, 1024, 0, s>>>(poses, N, out);
    return cudaGetLastError();
}

}  // namespace mcl
