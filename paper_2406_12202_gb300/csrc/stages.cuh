// stages.cuh -- per-ray, per-particle and per-block bodies of the SIMT stages
// of one weight update, shared by the single-update kernels (render.cu,
// resample.cu) and the device-driven loop kernels (loop.cu), so both run the
// same arithmetic.
#pragma once
#include <math.h>

#include "internal.cuh"
#include "rng.cuh"

namespace mcl {

typedef unsigned long long u64;
typedef unsigned __int128 u128;

// ---------------------------------------------------------------------------
// Pixel-centre ray of pose p (row-major 3x4 [R|t], camera looking along -z,
// +y up) through level-image pixel (u, v) with level intrinsics; the
// direction is formed in FP64 and kept as FP32 value + FP32 rounding error.
// A pose with a non-finite entry yields |d| = NaN (the particle's loss
// becomes NaN and it gets no weight).  gd receives gamma(d) of the unit
// direction (4 frequencies, 27 values, zero-padded to 32).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void make_ray(const float* __restrict__ p, int u, int v, float fx,
                                         float fy, float cx, float cy, Ray& ray,
                                         float* __restrict__ g) {
    const double ax = ((double)u + 0.5 - (double)cx) / (double)fx;
    const double ay = -((double)v + 0.5 - (double)cy) / (double)fy;
    const double az = -1.0;
    double d[3];
#pragma unroll
    for (int c = 0; c < 3; ++c)
        d[c] = (double)p[4 * c] * ax + (double)p[4 * c + 1] * ay + (double)p[4 * c + 2] * az;
    const double dn64 = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    bool finite_pose = true;
#pragma unroll
    for (int c = 0; c < 12; ++c) finite_pose = finite_pose && isfinite(p[c]);
    const float dx = (float)d[0], dy = (float)d[1], dz = (float)d[2];
    ray.ox = p[3]; ray.oy = p[7]; ray.oz = p[11];
    ray.dnorm = finite_pose ? (float)dn64 : __int_as_float(0x7fc00000);
    ray.dx = dx; ray.dy = dy; ray.dz = dz; ray.pad = 0.f;
    ray.lx = (float)(d[0] - (double)dx);
    ray.ly = (float)(d[1] - (double)dy);
    ray.lz = (float)(d[2] - (double)dz);
    ray.pad2 = 0.f;
    const float h[3] = {(float)(d[0] / dn64), (float)(d[1] / dn64), (float)(d[2] / dn64)};
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

// Query pixel set: B distinct pixels of a W x H level image, uniformly without
// replacement, by Floyd's sampling algorithm (Bentley & Floyd, CACM 1987):
// for j = n-B .. n-1 draw t uniform in [0, j] and take t unless already
// taken, else j.  t = floor(r (j + 1) / 2^64), r = value j-(n-B) of
// SplitMix64 stream (seed, ctr).  out[2i], out[2i+1] = (q % W, q / W).
// One thread; O(B^2) membership tests.
__device__ __forceinline__ void draw_pixel_set(int W, int H, int B, uint64_t seed, uint64_t ctr,
                                               int32_t* __restrict__ out) {
    const long n = (long)W * H;
    for (long j = n - B, m = 0; j < n; ++j, ++m) {
        const uint64_t r = cb_rand(seed, ctr, (uint64_t)(j - (n - B)));
        const long t = (long)(((u128)r * (u128)(uint64_t)(j + 1)) >> 64);
        bool dup = false;
        for (long i = 0; i < m; ++i)
            if ((long)out[2 * i + 1] * W + out[2 * i] == t) { dup = true; break; }
        const long c = dup ? j : t;
        out[2 * m] = (int32_t)(c % W);
        out[2 * m + 1] = (int32_t)(c / W);
    }
}

// Stratified coarse samples of ray r: z_k = near + (far - near)(k + u_k)/n_c,
// u_k = 1/2 or value r*n_c + k of SplitMix64 stream (seed, ctr).
__device__ __forceinline__ void coarse_samples(long r, int nc, float near_z, float far_z,
                                               int jitter, uint64_t seed, uint64_t ctr,
                                               float* __restrict__ z) {
    const float span = far_z - near_z;
    for (int k = 0; k < nc; ++k) {
        const float uk = jitter ? (float)cb_uniform(seed, ctr, (uint64_t)r * nc + k) : 0.5f;
        z[k] = near_z + span * ((float)k + uk) / (float)nc;
    }
}

// Coarse composite (Eq. 1 quadrature) and inverse-CDF importance samples of
// one ray: edges = midpoints of consecutive coarse z; pdf over the interior
// bins proportional to w_1..w_{n_c-2} + 1e-5; u_j = j/(n_f - 1); the bin is
// the first CDF entry strictly greater than u_j (u sorted: one sweep).
__device__ __forceinline__ void importance_samples(const float* __restrict__ z,
                                                   const float4* __restrict__ o, int nc, float dn,
                                                   int nf, float* __restrict__ out) {
    float cdf[kMaxCoarse];
    float T = 1.0f;
    float tot = 0.0f;
    for (int k = 0; k < nc; ++k) {
        const float sg = fmaxf(o[k].x, 0.0f);
        const float delta = (k < nc - 1) ? (z[k + 1] - z[k]) * dn : 1e10f;
        const float a = 1.0f - expf(-sg * delta);
        const float w = T * a;
        T *= (1.0f - a);
        if (k >= 1 && k <= nc - 2) {
            cdf[k] = w + 1e-5f;   // pdf of bin k-1, normalised below
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

struct RayResult {
    float r, g, b;
    float z_trans, z_opaque, F;
};

// Final composite over the merged coarse + fine samples (both sorted; equal
// z take the coarse sample first), Eq. 5 on the running weight sum and F of
// Eq. 6 (F = 1 without rejection).
__device__ __forceinline__ RayResult composite_ray(float dn, const float* __restrict__ za,
                                                   const float4* __restrict__ oa, int nc,
                                                   const float* __restrict__ zb,
                                                   const float4* __restrict__ ob, int nf,
                                                   float alpha, float tau, int use_rej) {
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
    RayResult res;
    res.r = cr; res.g = cg; res.b = cb;
    res.z_trans = zt; res.z_opaque = zo;
    res.F = use_rej ? fmaxf(zo - zt, tau) : 1.0f;
    return res;
}

// Box-filtered colour of level-image pixel (u, v) (factor x factor block of
// the full-resolution image, W pixels per row); NaN outside the level image.
__device__ __forceinline__ float4 observed_colour(const float* __restrict__ img, int W, int H,
                                                  int factor, int u, int v) {
    if (u < 0 || v < 0 || u >= W / factor || v >= H / factor) {
        const float nan = __int_as_float(0x7fc00000);
        return make_float4(nan, nan, nan, nan);
    }
    float s0 = 0.f, s1 = 0.f, s2 = 0.f;
    for (int dy = 0; dy < factor; ++dy) {
        const float* row = img + ((size_t)(v * factor + dy) * W + (size_t)u * factor) * 3;
        for (int dx = 0; dx < factor; ++dx) {
            s0 += row[3 * dx]; s1 += row[3 * dx + 1]; s2 += row[3 * dx + 2];
        }
    }
    const float inv = 1.0f / (float)(factor * factor);
    return make_float4(s0 * inv, s1 * inv, s2 * inv, 0.f);
}

// E = squared RGB distance between the rendered colour and the box-filtered
// observed pixel (u, v) of the level image (factor x factor block of the
// full-resolution image, W pixels per row).  NaN when the ray is invalid.
__device__ __forceinline__ float photometric_E(const float* __restrict__ img, int W, int factor,
                                               int u, int v, const RayResult& c, float dn) {
    float s0 = 0.f, s1 = 0.f, s2 = 0.f;
    for (int dy = 0; dy < factor; ++dy) {
        const float* row = img + ((size_t)(v * factor + dy) * W + (size_t)u * factor) * 3;
        for (int dx = 0; dx < factor; ++dx) {
            s0 += row[3 * dx]; s1 += row[3 * dx + 1]; s2 += row[3 * dx + 2];
        }
    }
    const float inv = 1.0f / (float)(factor * factor);
    const float e0 = s0 * inv - c.r, e1 = s1 * inv - c.g, e2 = s2 * inv - c.b;
    return isfinite(dn) ? e0 * e0 + e1 * e1 + e2 * e2 : __int_as_float(0x7fc00000);
}

// ---------------------------------------------------------------------------
// Block reductions (blockDim.x a multiple of 32, at most 1024).
// ---------------------------------------------------------------------------
__device__ __forceinline__ double block_max_d(double v, double* sh) {
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

__device__ __forceinline__ double block_sum_d(double v, double* sh) {
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

// Inclusive scan of one u64 per thread across the block; returns the
// inclusive prefix and writes the block total to *total.
__device__ __forceinline__ u64 block_scan_u64(u64 v, u64* sh, u64* total) {
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
        if (lane < nw) sh[lane] = s;
    }
    __syncthreads();
    const u64 before = wid > 0 ? sh[wid - 1] : 0ull;
    *total = sh[nw - 1];
    return v + before;
}

// ---------------------------------------------------------------------------
// Eq. 6 weights of one particle set, by one block: S_i = sum_j E_ij F_ij
// (FP32, j order), log w_i = 4 (log B - log max(S_i, s_min)), normalisation
// w_i = exp(log w_i - logsumexp) in FP64, mask_i = (w_i >= rho / N).
// Non-finite S_i -> log w = -inf (returned count of such particles).
// ---------------------------------------------------------------------------
__device__ __forceinline__ int weights_block(const float* __restrict__ e_ray, int N, int B,
                                             double s_min, double rho, float* __restrict__ logw,
                                             double* __restrict__ l64, double* __restrict__ w,
                                             uint8_t* __restrict__ mask, float* __restrict__ S_dbg) {
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
        if (logw) logw[i] = (float)l;
        mx = fmax(mx, l);
    }
    mx = block_max_d(mx, sh);
    double acc = 0.0;
    if (mx > -INFINITY)
        for (int i = threadIdx.x; i < N; i += blockDim.x) acc += exp(l64[i] - mx);
    acc = block_sum_d(acc, sh);
    const double lse = mx + log(acc);
    const double thr = rho / (double)N;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        const double wi = (mx > -INFINITY) ? exp(l64[i] - lse) : 0.0;
        w[i] = wi;
        mask[i] = (uint8_t)(wi >= thr && wi > 0.0);
    }
    __syncthreads();
    return nbad;
}

// ---------------------------------------------------------------------------
// Systematic resampling on an exact integer CDF, by one block:
// d_idx[k] = smallest i with C_i N_out 2^53 > (k 2^53 + U) T, where
// q_i = floor(w_i 2^s), s = 50 - e - ceil(log2 N_in), e = exponent of max w,
// C = inclusive prefix of q, T = C_{N_in-1}, U = floor(u0 2^53).  Returns
// false (every idx = -1) for negative, non-finite or all-zero weights.
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool resample_block(const double* __restrict__ w, int n_in, int n_out,
                                               double u0, int32_t* __restrict__ idx,
                                               u64* __restrict__ cdf) {
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
    mx = block_max_d(mx, shd);
    if (bad || !(mx > 0.0)) {
        for (int k = threadIdx.x; k < n_out; k += blockDim.x) idx[k] = -1;
        return false;
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
        return false;
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
    return true;
}

// ---------------------------------------------------------------------------
// Prediction of one particle: O = P * Exp(q[0..2], (0, q[3], 0)) in FP64.
// SE(3) exponential: R = I + a K + b K^2, t = (I + b K + c K^2) rho with
// K = [omega]x, th = |omega|, a = sin th / th, b = (1 - cos th)/th^2,
// c = (th - sin th)/th^3 (series values below th = 1e-8).
// ---------------------------------------------------------------------------
// x Exp(delta) for the pose P (optionally x O_t Exp(delta): odom is the 3x4
// relative motion O_t, NULL for the identity), FP64 arithmetic.
__device__ __forceinline__ void predict_pose(const float* __restrict__ P0, const double q[4],
                                             float* __restrict__ O,
                                             const float* __restrict__ odom = nullptr) {
    double P[12];
    if (odom) {
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                double s = (c == 3) ? (double)P0[4 * r + 3] : 0.0;
#pragma unroll
                for (int m = 0; m < 3; ++m) s += (double)P0[4 * r + m] * (double)odom[4 * m + c];
                P[4 * r + c] = s;
            }
    } else {
#pragma unroll
        for (int k = 0; k < 12; ++k) P[k] = (double)P0[k];
    }
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
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            double s = (c == 3) ? P[4 * r + 3] : 0.0;
#pragma unroll
            for (int m = 0; m < 3; ++m) s += P[4 * r + m] * E[4 * m + c];
            O[4 * r + c] = (float)s;
        }
}

// Motion noise of particle k: normals 4k .. 4k+3 of stream (seed, ctr)
// scaled by (sigma_t, sigma_t, sigma_t, sigma_yaw).
__device__ __forceinline__ void motion_noise(uint64_t seed, uint64_t ctr, long k, float sigma_t,
                                             float sigma_yaw, double q[4]) {
#pragma unroll
    for (int c = 0; c < 4; ++c)
        q[c] = (c < 3 ? (double)sigma_t : (double)sigma_yaw) * cb_normal(seed, ctr, 4ull * k + c);
}

// Mean position and trace of the population covariance (FP64), one block.
__device__ __forceinline__ void spread_block(const float* __restrict__ P, int N,
                                             double* __restrict__ out) {
    __shared__ double sh[32];
    double m[3];
    for (int c = 0; c < 3; ++c) {
        double v = 0.0;
        for (int i = threadIdx.x; i < N; i += blockDim.x) v += (double)P[12 * (size_t)i + 4 * c + 3];
        m[c] = block_sum_d(v, sh) / N;
    }
    double t = 0.0;
    for (int i = threadIdx.x; i < N; i += blockDim.x)
        for (int c = 0; c < 3; ++c) {
            const double d = (double)P[12 * (size_t)i + 4 * c + 3] - m[c];
            t += d * d;
        }
    t = block_sum_d(t, sh);
    if (threadIdx.x == 0) {
        out[0] = m[0]; out[1] = m[1]; out[2] = m[2];
        out[3] = t / N;
    }
}

}  // namespace mcl
