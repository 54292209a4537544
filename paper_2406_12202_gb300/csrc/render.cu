// render.cu -- the SIMT stages of one weight update around the NeRF MLP:
// ray generation and stratified samples, coarse compositing with importance
// sampling, the final composite with Eq. 5 / F and the photometric match, and
// the Eq. 6 weights with FP64 log-sum-exp normalisation (bodies in
// stages.cuh).
#include <math.h>

#include "stages.cuh"

namespace mcl {

// One thread per ray r = i*B + j: pixel-centre ray of particle i through
// pixel j with the level intrinsics, gamma(d), stratified coarse samples.
__global__ void k_raygen(const float* __restrict__ P, int N, const int32_t* __restrict__ px,
                         int B, float fx, float fy, float cx, float cy, int nc, float near_z,
                         float far_z, int jitter, uint64_t seed, uint64_t ctr,
                         Ray* __restrict__ rays, float* __restrict__ gd, float* __restrict__ zc,
                         const float* __restrict__ img, int W, int H, int factor,
                         float4* __restrict__ obs) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= N * B) return;
    const int i = r / B, j = r - (r / B) * B;
    Ray ray;
    make_ray(P + 12 * (size_t)i, px[2 * j], px[2 * j + 1], fx, fy, cx, cy, ray,
             gd + (size_t)r * kGdPad);
    rays[r] = ray;
    coarse_samples(r, nc, near_z, far_z, jitter, seed, ctr, zc + (size_t)r * nc);
    if (obs) obs[r] = observed_colour(img, W, H, factor, px[2 * j], px[2 * j + 1]);
}

// Point queries: one "ray" per point with o = x, d = 0 and one sample at
// z = 0, so x = o + z d = x; gamma(d) of the normalised view direction.
__global__ void k_query_setup(const float* __restrict__ X, const float* __restrict__ D, int n,
                              Ray* __restrict__ rays, float* __restrict__ gd, float* __restrict__ z) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    Ray ray;
    ray.ox = X[3 * i]; ray.oy = X[3 * i + 1]; ray.oz = X[3 * i + 2]; ray.dnorm = 1.f;
    ray.dx = ray.dy = ray.dz = 0.f; ray.pad = 0.f;
    ray.lx = ray.ly = ray.lz = 0.f; ray.pad2 = 0.f;
    rays[i] = ray;
    z[i] = 0.f;
    const double d0 = D[3 * i], d1 = D[3 * i + 1], d2 = D[3 * i + 2];
    const double dn = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
    const float h[3] = {(float)(d0 / dn), (float)(d1 / dn), (float)(d2 / dn)};
    float* g = gd + (size_t)i * kGdPad;
    g[0] = h[0]; g[1] = h[1]; g[2] = h[2];
#pragma unroll
    for (int k = 0; k < kLdir; ++k) {
        const float f = (float)(1 << k);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            float sn, cs;
            sincosf(f * h[c], &sn, &cs);
            g[3 + 6 * k + c] = sn;
            g[6 + 6 * k + c] = cs;
        }
    }
#pragma unroll
    for (int c = kGd; c < kGdPad; ++c) g[c] = 0.f;
}

cudaError_t launch_query_setup(const float* X, const float* D, int n, Ray* rays, float* gd,
                               float* z, cudaStream_t s) {
    note_launch();
    k_query_setup<<<(n + 127) / 128, 128, 0, s>>>(X, D, n, rays, gd, z);
    return cudaGetLastError();
}

cudaError_t launch_raygen(const float* particles, int N, const int32_t* pixels, int B, float fx,
                          float fy, float cx, float cy, const mcl_opts& o, Ray* rays, float* gd,
                          float* zc, cudaStream_t s, const float* image, int W, int H, int factor,
                          float4* obs) {
    const int n = N * B, tb = 128;
    note_launch();
    k_raygen<<<(n + tb - 1) / tb, tb, 0, s>>>(particles, N, pixels, B, fx, fy, cx, cy, o.n_coarse,
                                               o.near_z, o.far_z, o.jitter, o.seed, o.counter,
                                               rays, gd, zc, image, W, H, factor,
                                               image ? obs : nullptr);
    return cudaGetLastError();
}

// Coarse composite and importance samples, one thread per ray.  n_rays_dev
// (optional) bounds the rays from device memory.
__global__ void k_coarse_to_fine(const Ray* __restrict__ rays, int n_rays,
                                 const int* __restrict__ n_rays_dev, const float* __restrict__ zc,
                                 int nc, const float4* __restrict__ out_c, int nf,
                                 float* __restrict__ zf) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = n_rays_dev ? min(n_rays, *n_rays_dev) : n_rays;
    if (r >= n) return;
    importance_samples(zc + (size_t)r * nc, out_c + (size_t)r * nc, nc, rays[r].dnorm, nf,
                       zf + (size_t)r * nf);
}

cudaError_t launch_coarse_to_fine(const Ray* rays, int n_rays, const int* n_rays_dev,
                                  const float* zc, int nc, const float4* out_c, int nf, float* zf,
                                  cudaStream_t s) {
    const int tb = 128;
    note_launch();
    k_coarse_to_fine<<<(n_rays + tb - 1) / tb, tb, 0, s>>>(rays, n_rays, n_rays_dev, zc, nc, out_c,
                                                            nf, zf);
    return cudaGetLastError();
}

// Final composite, Eq. 5 / F and E against the level image, one thread per
// ray.  image == NULL: render only (rgb_out / F_out).
__global__ void k_final(const Ray* __restrict__ rays, int n_rays, const float* __restrict__ zc,
                        const float4* __restrict__ oc, int nc, const float* __restrict__ zf,
                        const float4* __restrict__ of, int nf, const float* __restrict__ img,
                        int W, int H, int factor, const int32_t* __restrict__ px, int B, float alpha,
                        float tau, int use_rej, float* __restrict__ e_ray, float* __restrict__ d_rgb,
                        float* __restrict__ d_E, float* __restrict__ d_F, float* __restrict__ d_zt,
                        float* __restrict__ d_zo) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n_rays) return;
    const float dn = rays[r].dnorm;
    const RayResult c = composite_ray(dn, zc + (size_t)r * nc, oc + (size_t)r * nc, nc,
                                      zf + (size_t)r * nf, of + (size_t)r * nf, nf, alpha, tau,
                                      use_rej);
    if (d_rgb) { d_rgb[3 * (size_t)r] = c.r; d_rgb[3 * (size_t)r + 1] = c.g; d_rgb[3 * (size_t)r + 2] = c.b; }
    if (d_F) d_F[r] = c.F;
    if (d_zt) d_zt[r] = c.z_trans;
    if (d_zo) d_zo[r] = c.z_opaque;
    if (img) {
        const int j = r % B;
        const int u = px[2 * j], v = px[2 * j + 1];
        if (u < 0 || v < 0 || u >= W / factor || v >= H / factor) {
            // pixel outside the level image: no observation, loss is NaN
            if (d_E) d_E[r] = __int_as_float(0x7fc00000);
            e_ray[r] = __int_as_float(0x7fc00000);
            return;
        }
        const float E = photometric_E(img, W, factor, u, v, c, dn);
        if (d_E) d_E[r] = E;
        e_ray[r] = E * c.F;
    }
}

cudaError_t launch_final_composite(const Ray* rays, int n_rays, const float* zc, const float4* out_c,
                                   int nc, const float* zf, const float4* out_f, int nf,
                                   const float* image, int W, int H, int factor,
                                   const int32_t* pixels, int B, const mcl_opts& o, float* e_ray,
                                   const mcl_debug* dbg, float* rgb_out, float* F_out,
                                   cudaStream_t s) {
    const int tb = 128;
    float* d_rgb = rgb_out ? rgb_out : (dbg ? dbg->rgb : nullptr);
    float* d_F = F_out ? F_out : (dbg ? dbg->F : nullptr);
    note_launch();
    k_final<<<(n_rays + tb - 1) / tb, tb, 0, s>>>(
        rays, n_rays, zc, out_c, nc, zf, out_f, nf, image, W, H, factor, pixels, B, o.alpha, o.tau,
        o.use_rejection, e_ray, d_rgb, dbg ? dbg->E : nullptr, d_F, dbg ? dbg->z_trans : nullptr,
        dbg ? dbg->z_opaque : nullptr);
    return cudaGetLastError();
}

constexpr int kNormThreads = 1024;

__global__ __launch_bounds__(kNormThreads) void k_weights(
    const float* __restrict__ e_ray, int N, int B, double s_min, double rho,
    float* __restrict__ logw, double* __restrict__ l64, double* __restrict__ w,
    uint8_t* __restrict__ mask, float* __restrict__ S_dbg, Status* status) {
    const int nbad = weights_block(e_ray, N, B, s_min, rho, logw, l64, w, mask, S_dbg);
    if (threadIdx.x == 0 && nbad > 0) {
        atomicAdd(&status->n_nonfinite, nbad);
        atomicCAS(&status->code, 0, MCL_ERR_NONFINITE);
    }
}

cudaError_t launch_weights(const float* e_ray, int N, int B, const mcl_opts& o, float* logw,
                           double* logw64, double* w, uint8_t* mask, float* S_dbg, Status* status,
                           cudaStream_t s) {
    note_launch();
    k_weights<<<1, kNormThreads, 0, s>>>(e_ray, N, B, o.s_min, o.rho_reject, logw, logw64, w, mask,
                                         S_dbg, status);
    return cudaGetLastError();
}

}  // namespace mcl
