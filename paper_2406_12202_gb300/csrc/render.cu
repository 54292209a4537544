// render.cu -- the SIMT stages of the weight update around the NeRF MLP:
// ray generation and stratified samples, coarse compositing with importance
// sampling, the final composite with Eq. 5 / F and the photometric match, and
// the Eq. 6 weights with FP64 log-sum-exp normalisation.
#include <math.h>

#include "internal.cuh"
#include "rng.cuh"

namespace mcl {

// ---------------------------------------------------------------------------
// Ray generation (pixel-centre rays of R K, camera looking along -z, +y up)
// and stratified coarse samples z_k = near + (far - near)(k + u_k)/n_c with
// u_k = 1/2, or SplitMix64 stream (seed, counter) value ray*n_c + k.  Also
// gamma(d) of the unit direction (positional encoding with 4 frequencies),
// which is constant along the ray.  One thread per ray r = i*B + j.
// ---------------------------------------------------------------------------
__global__ void k_raygen(const float* __restrict__ P, int N, const int32_t* __restrict__ px,
                         int B, float fx, float fy, float cx, float cy, int nc, float near_z,
                         float far_z, int jitter, uint64_t seed, uint64_t ctr,
                         Ray* __restrict__ rays, float* __restrict__ gd, float* __restrict__ zc) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= N * B) return;
    const int i = r / B, j = r - (r / B) * B;
    const float* p = P + 12 * (size_t)i;
    // direction in FP64 (pose and pixel are exact FP32 inputs), kept as a
    // rounded FP32 value plus its rounding error
    const double u = (double)px[2 * j], v = (double)px[2 * j + 1];
    const double ax = (u + 0.5 - (double)cx) / (double)fx;
    const double ay = -(v + 0.5 - (double)cy) / (double)fy;
    const double az = -1.0;
    double d[3];
#pragma unroll
    for (int c = 0; c < 3; ++c)
        d[c] = (double)p[4 * c] * ax + (double)p[4 * c + 1] * ay + (double)p[4 * c + 2] * az;
    const double dn64 = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    const float dx = (float)d[0], dy = (float)d[1], dz = (float)d[2];
    // a pose with a non-finite entry marks its rays invalid (|d| = NaN); the
    // composite turns that into a NaN loss, so the particle gets no weight
    bool finite_pose = true;
#pragma unroll
    for (int c = 0; c < 12; ++c) finite_pose = finite_pose && isfinite(p[c]);
    const float dn = finite_pose ? (float)dn64 : __int_as_float(0x7fc00000);
    Ray ray;
    ray.ox = p[3]; ray.oy = p[7]; ray.oz = p[11]; ray.dnorm = dn;
    ray.dx = dx; ray.dy = dy; ray.dz = dz; ray.pad = 0.f;
    ray.lx = (float)(d[0] - (double)dx);
    ray.ly = (float)(d[1] - (double)dy);
    ray.lz = (float)(d[2] - (double)dz);
    ray.pad2 = 0.f;
    rays[r] = ray;
    const float h[3] = {(float)(d[0] / dn64), (float)(d[1] / dn64), (float)(d[2] / dn64)};
    float* g = gd + (size_t)r * kGdPad;
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
    float* z = zc + (size_t)r * nc;
    const float span = far_z - near_z;
    for (int k = 0; k < nc; ++k) {
        const float uk = jitter ? (float)cb_uniform(seed, ctr, (uint64_t)r * nc + k) : 0.5f;
        z[k] = near_z + span * ((float)k + uk) / (float)nc;
    }
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
                          float* zc, cudaStream_t s) {
    const int n = N * B, tb = 128;
    note_launch();
    k_raygen<<<(n + tb - 1) / tb, tb, 0, s>>>(particles, N, pixels, B, fx, fy, cx, cy, o.n_coarse,
                                               o.near_z, o.far_z, o.jitter, o.seed, o.counter,
                                               rays, gd, zc);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Coarse composite (Eq. 1 quadrature) and inverse-CDF importance samples.
// Edges = midpoints of consecutive coarse z; pdf over the interior bins
// proportional to w_1..w_{n_c-2} + 1e-5; u_j = j/(n_f - 1); the bin is the
// first CDF entry strictly greater than u_j (u sorted, so one sweep).  One
// thread per ray.
// ---------------------------------------------------------------------------
__global__ void k_coarse_to_fine(const Ray* __restrict__ rays, int n_rays,
                                 const float* __restrict__ zc, int nc,
                                 const float4* __restrict__ out_c, int nf, float* __restrict__ zf) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n_rays) return;
    const float* z = zc + (size_t)r * nc;
    const float4* o = out_c + (size_t)r * nc;
    const float dn = rays[r].dnorm;
    float cdf[kMaxCoarse];
    // weights of the interior samples go straight into pdf slots cdf[1..nc-2]
    float T = 1.0f;
    float tot = 0.0f;
    for (int k = 0; k < nc; ++k) {
        const float sg = fmaxf(o[k].x, 0.0f);
        const float delta = (k < nc - 1) ? (z[k + 1] - z[k]) * dn : 1e10f;
        const float a = 1.0f - expf(-sg * delta);
        const float w = T * a;
        T *= (1.0f - a);
        if (k >= 1 && k <= nc - 2) {
            cdf[k] = w + 1e-5f;
            tot += w + 1e-5f;
        }
    }
    const int ne = nc - 1;
    cdf[0] = 0.0f;
    float run = 0.0f;
    for (int i = 1; i < ne; ++i) {
        run += cdf[i] / tot;
        cdf[i] = run;
    }
    float* out = zf + (size_t)r * nf;
    int idx = 0;
    for (int j = 0; j < nf; ++j) {
        const float u = nf > 1 ? (float)j / (float)(nf - 1) : 0.0f;
        while (idx < ne && cdf[idx] <= u) ++idx;
        const int below = idx - 1 < 0 ? 0 : idx - 1;
        const int above = idx > ne - 1 ? ne - 1 : idx;
        float denom = cdf[above] - cdf[below];
        if (denom < 1e-5f) denom = 1.0f;
        const float t = (u - cdf[below]) / denom;
        const float eb = 0.5f * (z[below] + z[below + 1]);
        const float ea = 0.5f * (z[above] + z[above + 1]);
        out[j] = eb + t * (ea - eb);
    }
}

cudaError_t launch_coarse_to_fine(const Ray* rays, int n_rays, const float* zc, int nc,
                                  const float4* out_c, int nf, float* zf, cudaStream_t s) {
    const int tb = 128;
    note_launch();
    k_coarse_to_fine<<<(n_rays + tb - 1) / tb, tb, 0, s>>>(rays, n_rays, zc, nc, out_c, nf, zf);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Final composite over the merged coarse + fine samples (both sorted; equal z
// take the coarse sample first), Eq. 5 on the running weight sum, F of
// Eq. 6, and E = squared RGB distance to the box-filtered observed pixel.
// image == NULL: render only (rgb_out / F_out).  One thread per ray.
// ---------------------------------------------------------------------------
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
    const float* za = zc + (size_t)r * nc;
    const float4* oa = oc + (size_t)r * nc;
    const float* zb = zf + (size_t)r * nf;
    const float4* ob = of + (size_t)r * nf;
    int ia = 0, ib = 0;
    auto take = [&](float& z, float4& v) {
        if (ib >= nf || (ia < nc && za[ia] <= zb[ib])) {
            z = za[ia]; v = oa[ia]; ++ia;
        } else {
            z = zb[ib]; v = ob[ib]; ++ib;
        }
    };
    const int n = nc + nf;
    float zcur, znext = 0.f;
    float4 vcur, vnext = make_float4(0.f, 0.f, 0.f, 0.f);
    take(zcur, vcur);
    const float z0 = zcur;
    float T = 1.0f, cr = 0.f, cg = 0.f, cb = 0.f, Wc = 0.f;
    float zt = z0, zo = z0;
    bool have_t = false;
    for (int k = 0; k < n; ++k) {
        if (k < n - 1) take(znext, vnext);
        const float delta = (k < n - 1) ? (znext - zcur) * dn : 1e10f;
        const float sg = fmaxf(vcur.x, 0.0f);
        const float a = 1.0f - expf(-sg * delta);
        const float w = T * a;
        cr += w * vcur.y; cg += w * vcur.z; cb += w * vcur.w;
        T *= (1.0f - a);
        Wc += w;
        if (!have_t && Wc >= alpha) { zt = zcur; have_t = true; }
        if (Wc <= 1.0f - alpha) zo = zcur;
        zcur = znext; vcur = vnext;
    }
    const float F = use_rej ? fmaxf(zo - zt, tau) : 1.0f;
    if (d_rgb) { d_rgb[3 * (size_t)r] = cr; d_rgb[3 * (size_t)r + 1] = cg; d_rgb[3 * (size_t)r + 2] = cb; }
    if (d_F) d_F[r] = F;
    if (d_zt) d_zt[r] = zt;
    if (d_zo) d_zo[r] = zo;
    if (img) {
        const int j = r % B;
        const int u = px[2 * j], v = px[2 * j + 1];
        if (u < 0 || v < 0 || u >= W / factor || v >= H / factor) {
            // pixel outside the level image: no observation, loss is NaN
            if (d_E) d_E[r] = __int_as_float(0x7fc00000);
            e_ray[r] = __int_as_float(0x7fc00000);
            return;
        }
        float s0 = 0.f, s1 = 0.f, s2 = 0.f;
        for (int dy = 0; dy < factor; ++dy) {
            const float* row = img + ((size_t)(v * factor + dy) * W + (size_t)u * factor) * 3;
            for (int dx = 0; dx < factor; ++dx) {
                s0 += row[3 * dx]; s1 += row[3 * dx + 1]; s2 += row[3 * dx + 2];
            }
        }
        const float inv = 1.0f / (float)(factor * factor);
        const float e0 = s0 * inv - cr, e1 = s1 * inv - cg, e2 = s2 * inv - cb;
        const float E = isfinite(dn) ? e0 * e0 + e1 * e1 + e2 * e2 : __int_as_float(0x7fc00000);
        if (d_E) d_E[r] = E;
        e_ray[r] = E * F;
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

// ---------------------------------------------------------------------------
// Eq. 6 weights: S_i = sum_j E_ij F_ij (FP32, in j order), log w_i =
// 4 (log B - log max(S_i, s_min)) and the normalisation
// w_i = exp(log w_i - logsumexp) in FP64; mask_i = (w_i >= rho / N).  One
// block; non-finite S_i -> log w = -inf, counted in the status word.
// ---------------------------------------------------------------------------
constexpr int kNormThreads = 1024;

__device__ double block_reduce_max(double v, double* sh) {
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) sh[w] = v;
    __syncthreads();
    if (w == 0) {
        v = l < (int)(blockDim.x >> 5) ? sh[l] : -INFINITY;
        for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
        if (l == 0) sh[0] = v;
    }
    __syncthreads();
    return sh[0];
}

__device__ double block_reduce_sum(double v, double* sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) sh[w] = v;
    __syncthreads();
    if (w == 0) {
        v = l < (int)(blockDim.x >> 5) ? sh[l] : 0.0;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (l == 0) sh[0] = v;
    }
    __syncthreads();
    return sh[0];
}

__global__ __launch_bounds__(kNormThreads) void k_weights(
    const float* __restrict__ e_ray, int N, int B, double s_min, double rho,
    float* __restrict__ logw, double* __restrict__ l64, double* __restrict__ w,
    uint8_t* __restrict__ mask, float* __restrict__ S_dbg, Status* status) {
    __shared__ double sh[32];
    __shared__ int nbad;
    if (threadIdx.x == 0) nbad = 0;
    __syncthreads();
    const double logB = log((double)B);
    double mx = -INFINITY;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        const float* e = e_ray + (size_t)i * B;
        float S = 0.0f;
        for (int j = 0; j < B; ++j) S += e[j];
        if (S_dbg) S_dbg[i] = S;
        double l;
        if (isfinite(S)) {
            const double sc = fmax((double)S, s_min);
            l = 4.0 * (logB - log(sc));
        } else {
            l = -INFINITY;
            atomicAdd(&nbad, 1);
        }
        l64[i] = l;
        logw[i] = (float)l;
        mx = fmax(mx, l);
    }
    mx = block_reduce_max(mx, sh);
    double acc = 0.0;
    if (mx > -INFINITY)
        for (int i = threadIdx.x; i < N; i += blockDim.x) acc += exp(l64[i] - mx);
    acc = block_reduce_sum(acc, sh);
    const double lse = mx + log(acc);
    const double thr = rho / (double)N;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        const double wi = (mx > -INFINITY) ? exp(l64[i] - lse) : 0.0;
        w[i] = wi;
        mask[i] = (uint8_t)(wi >= thr && wi > 0.0);
    }
    __syncthreads();
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
