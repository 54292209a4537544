// resample.cu -- systematic resampling on an exact integer CDF, the motion
// (prediction) step, the box downscale of the observed image, and the
// position spread used by the refinement test.
#include <math.h>

#include "stages.cuh"

namespace mcl {

constexpr int kResThreads = 1024;

__global__ __launch_bounds__(kResThreads) void k_resample(const double* __restrict__ w, int n_in,
                                                          int n_out, double u0,
                                                          int32_t* __restrict__ idx,
                                                          u64* __restrict__ cdf, Status* status) {
    if (!resample_block(w, n_in, n_out, u0, idx, cdf) && threadIdx.x == 0 && status)
        atomicCAS(&status->code, 0, MCL_ERR_DEGENERATE);
}

cudaError_t launch_resample(const double* w, int n_in, int n_out, double u0, int32_t* idx,
                            unsigned long long* cdf, Status* status, cudaStream_t s) {
    note_launch();
    k_resample<<<1, kResThreads, 0, s>>>(w, n_in, n_out, u0, idx, cdf, status);
    return cudaGetLastError();
}

// Prediction: out_k = in_{idx_k} * Exp(rho, (0, yaw, 0)) (stages.cuh).
__global__ void k_predict(const float* __restrict__ in, int n_in, const int32_t* __restrict__ idx,
                          int n, const float* __restrict__ odom, float sigma_t, float sigma_yaw,
                          uint64_t seed, uint64_t ctr, float* __restrict__ out) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int src = idx ? idx[k] : k;
    float* O = out + 12 * (size_t)k;
    if (src < 0 || src >= n_in) {
        for (int c = 0; c < 12; ++c) O[c] = __int_as_float(0x7fc00000);
        return;
    }
    double q[4];
    motion_noise(seed, ctr, k, sigma_t, sigma_yaw, q);
    predict_pose(in + 12 * (size_t)src, q, O, odom);
}

cudaError_t launch_predict(const float* in, int n_in, const int32_t* idx, int n_out,
                           const float* odom, float sigma_t, float sigma_yaw, uint64_t seed,
                           uint64_t counter, float* out, cudaStream_t s) {
    note_launch();
    k_predict<<<(n_out + 127) / 128, 128, 0, s>>>(in, n_in, idx, n_out, odom, sigma_t, sigma_yaw, seed,
                                                   counter, out);
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

// Mean position and trace of the population covariance (FP64), one block.
__global__ __launch_bounds__(1024) void k_spread(const float* __restrict__ P, int N,
                                                 double* __restrict__ out) {
    spread_block(P, N, out);
}

cudaError_t launch_position_spread(const float* poses, int N, double* out, cudaStream_t s) {
    note_launch();
    k_spread<<<1, 1024, 0, s>>>(poses, N, out);
    return cudaGetLastError();
}

}  // namespace mcl
