// proposal.cu -- the learned proposal sampler (a project extension; the paper
// has none): a small MLP from gamma(x) (6 frequencies) through four ReLU
// layers of 64 units to a density, composited over stratified samples as
// Eq. 1, whose weights drive the inverse-CDF sampler in place of the coarse
// pass of the NeRF MLP.  It is distilled from the full hierarchical sampler:
// targets are the sampler's final weights re-binned onto the proposal's
// intervals, the loss is the cross-entropy of the normalised proposal
// weights, and training runs here in FP32 with Adam.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <random>
#include <vector>

#include "stages.cuh"

namespace mcl {

constexpr int kPL = 6;                  // frequencies of gamma(x)
constexpr int kPIn = 3 + 6 * kPL;       // 39
constexpr int kPInPad = 40;
constexpr int kPW = 64;                 // width
constexpr int kPDepth = 4;
// blob offsets: P1 W[64][39] b[64], P2..P4 W[64][64] b[64], head w[64] b[1]
constexpr int kPOff1 = 0;
// offset of layer l (0-based); layers 1..3 are 64x64
__host__ __device__ constexpr int prop_off(int l) {
    return l == 0 ? 0 : kPW * kPIn + kPW + (l - 1) * (kPW * kPW + kPW);
}
constexpr int kPOffHead = kPW * kPIn + kPW + 3 * (kPW * kPW + kPW);
constexpr int kPN = kPOffHead + kPW + 1;  // 15105
static_assert(kPN == 15105, "proposal blob size");

// gamma(x) with 6 frequencies (identity, then sin / cos of 2^k x per axis).
__device__ __forceinline__ void prop_pe(const float x[3], float* g) {
    g[0] = x[0]; g[1] = x[1]; g[2] = x[2];
#pragma unroll
    for (int k = 0; k < kPL; ++k) {
        const float f = (float)(1 << k);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            float sn, cs;
            sincosf(f * x[c], &sn, &cs);
            g[3 + 6 * k + c] = sn;
            g[6 + 6 * k + c] = cs;
        }
    }
}

// Forward of one point with weights in shared memory; h (optional) receives
// the post-ReLU activations [4][64], g the encoding.
__device__ __forceinline__ float prop_point(const float* __restrict__ Wsh, const float x[3],
                                            float* __restrict__ g, float* __restrict__ hsave) {
    float in[kPW], out[kPW];
    prop_pe(x, g);
    // outer loops over output units are not unrolled (the inner dot products
    // are): the same arithmetic per unit, a fraction of the code size
#pragma unroll 1
    for (int o = 0; o < kPW; ++o) {
        const float* w = Wsh + kPOff1 + o * kPIn;
        float s = Wsh[kPOff1 + kPW * kPIn + o];
#pragma unroll
        for (int i = 0; i < kPIn; ++i) s = fmaf(w[i], g[i], s);
        in[o] = fmaxf(s, 0.0f);
    }
    if (hsave)
#pragma unroll
        for (int o = 0; o < kPW; ++o) hsave[o] = in[o];
#pragma unroll
    for (int l = 1; l < kPDepth; ++l) {
        const float* W = Wsh + prop_off(l);
        const float* b = W + kPW * kPW;
#pragma unroll 1
        for (int o = 0; o < kPW; ++o) {
            float s = b[o];
#pragma unroll
            for (int i = 0; i < kPW; ++i) s = fmaf(W[o * kPW + i], in[i], s);
            out[o] = fmaxf(s, 0.0f);
        }
#pragma unroll
        for (int o = 0; o < kPW; ++o) in[o] = out[o];
        if (hsave)
#pragma unroll
            for (int o = 0; o < kPW; ++o) hsave[l * kPW + o] = in[o];
    }
    float s = Wsh[kPOffHead + kPW];
#pragma unroll
    for (int i = 0; i < kPW; ++i) s = fmaf(Wsh[kPOffHead + i], in[i], s);
    return s;
}

__device__ __forceinline__ void load_weights_smem(const float* __restrict__ W, float* sh) {
    for (int i = threadIdx.x; i < kPN; i += blockDim.x) sh[i] = W[i];
    __syncthreads();
}

// Inference: raw proposal density of sample k of ray r (stratified midpoints
// z = near + (far - near)(k + 1/2)/n_p, written by raygen into z) into
// out[r * n_p + k].x.
__global__ void k_prop_infer(const float* __restrict__ W, const Ray* __restrict__ rays,
                             const float* __restrict__ z, int n_p, long n_rows,
                             const int* __restrict__ n_rays_dev, float4* __restrict__ out) {
    extern __shared__ float wsh[];
    load_weights_smem(W, wsh);
    const long rows = n_rays_dev ? min(n_rows, (long)*n_rays_dev * n_p) : n_rows;
    for (long row = (long)blockIdx.x * blockDim.x + threadIdx.x; row < rows;
         row += (long)gridDim.x * blockDim.x) {
        const Ray R = rays[row / n_p];
        const float zz = z[row];
        const float x[3] = {fmaf(zz, R.dx, R.ox), fmaf(zz, R.dy, R.oy), fmaf(zz, R.dz, R.oz)};
        float g[kPInPad];
        out[row] = make_float4(prop_point(wsh, x, g, nullptr), 0.f, 0.f, 0.f);
    }
}

// ---------------------------------------------------------------- training
// Forward with saved encodings [rows][40] and activations [rows][4][64].
__global__ void k_prop_fwd_train(const float* __restrict__ W, const float* __restrict__ O,
                                 const float* __restrict__ D, int n_rays, int nb, float near_z,
                                 float far_z, float* __restrict__ gsave, float* __restrict__ hsave,
                                 float* __restrict__ s_out) {
    extern __shared__ float wsh[];
    load_weights_smem(W, wsh);
    const long rows = (long)n_rays * nb;
    for (long row = (long)blockIdx.x * blockDim.x + threadIdx.x; row < rows;
         row += (long)gridDim.x * blockDim.x) {
        const long r = row / nb;
        const int k = (int)(row - r * nb);
        const float zz = near_z + (far_z - near_z) * ((float)k + 0.5f) / (float)nb;
        const float x[3] = {fmaf(zz, D[3 * r], O[3 * r]), fmaf(zz, D[3 * r + 1], O[3 * r + 1]),
                            fmaf(zz, D[3 * r + 2], O[3 * r + 2])};
        float* g = gsave + row * kPInPad;
        s_out[row] = prop_point(wsh, x, g, hsave + row * (kPDepth * kPW));
        g[kPIn] = 0.0f;
    }
}

// Per ray: composite of the raw densities, cross-entropy against hist and
// dL/ds per sample (masked by s > 0):
//   g_j = -h_j / (p_j W) + sum_b h_b w_b / (p_b W^2),  p_b = w_b / W + 1e-8,
//   dL/dsigma_j = delta_j (g_j T_j (1 - alpha_j) - sum_{k>j} g_k w_k).
// A ray with no density (W = 0) contributes -log(1e-8) and no gradient.
__global__ void k_prop_loss_bwd(const float* __restrict__ s, const float* __restrict__ D,
                                int n_rays, int nb, float near_z, float far_z,
                                const float* __restrict__ hist, float scale, double lscale,
                                float* __restrict__ ds, double* __restrict__ loss_acc) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n_rays) return;
    const float dn = sqrtf(D[3 * r] * D[3 * r] + D[3 * r + 1] * D[3 * r + 1] + D[3 * r + 2] * D[3 * r + 2]);
    const float dz = (far_z - near_z) / (float)nb;
    const float* sr = s + (long)r * nb;
    const float* h = hist + (long)r * nb;
    float* dsr = ds + (long)r * nb;
    float w[kMaxCoarse], T[kMaxCoarse], al[kMaxCoarse];
    float trans = 1.0f, Wt = 0.0f;
    for (int k = 0; k < nb; ++k) {
        const float delta = (k < nb - 1) ? dz * dn : 1e10f;
        const float sg = fmaxf(sr[k], 0.0f);
        al[k] = 1.0f - expf(-sg * delta);
        T[k] = trans;
        w[k] = trans * al[k];
        trans *= (1.0f - al[k]);
        Wt += w[k];
    }
    double L = 0.0;
    if (!(Wt > 0.0f)) {
        for (int b = 0; b < nb; ++b) {
            L -= (double)h[b] * log(1e-8);
            dsr[b] = 0.0f;
        }
    } else {
        float c = 0.0f;
        for (int b = 0; b < nb; ++b) {
            const float p = w[b] / Wt + 1e-8f;
            L -= (double)h[b] * log((double)p);
            c += h[b] * w[b] / (p * Wt * Wt);
        }
        float tail = 0.0f;
        for (int j = nb - 1; j >= 0; --j) {
            const float p = w[j] / Wt + 1e-8f;
            const float gj = -h[j] / (p * Wt) + c;
            const float delta = (j < nb - 1) ? dz * dn : 1e10f;
            const float dsig = delta * (gj * T[j] * (1.0f - al[j]) - tail);
            dsr[j] = sr[j] > 0.0f ? dsig * scale : 0.0f;
            tail += gj * w[j];
        }
    }
    atomicAdd(loss_acc, L * lscale);
}

// Backward data pass per sample: da_l = (W_{l+1}^T da_{l+1}) masked by
// h_l > 0, starting from da_4 = ds * head; saved as [rows][4][64].
__global__ void k_prop_bwd_data(const float* __restrict__ W, const float* __restrict__ hsave,
                                const float* __restrict__ ds, long rows,
                                float* __restrict__ dasave) {
    extern __shared__ float wsh[];
    load_weights_smem(W, wsh);
    for (long row = (long)blockIdx.x * blockDim.x + threadIdx.x; row < rows;
         row += (long)gridDim.x * blockDim.x) {
        const float* h = hsave + row * (kPDepth * kPW);
        float* da = dasave + row * (kPDepth * kPW);
        const float d = ds[row];
        float cur[kPW];
#pragma unroll
        for (int i = 0; i < kPW; ++i) {
            const float v = h[(kPDepth - 1) * kPW + i] > 0.0f ? d * wsh[kPOffHead + i] : 0.0f;
            cur[i] = v;
            da[(kPDepth - 1) * kPW + i] = v;
        }
#pragma unroll
        for (int l = kPDepth - 1; l >= 1; --l) {
            const float* Wl = wsh + prop_off(l);
            float nxt[kPW];
#pragma unroll 1
            for (int i = 0; i < kPW; ++i) {
                float s = 0.0f;
#pragma unroll
                for (int o = 0; o < kPW; ++o) s = fmaf(Wl[o * kPW + i], cur[o], s);
                nxt[i] = h[(l - 1) * kPW + i] > 0.0f ? s : 0.0f;
            }
#pragma unroll
            for (int i = 0; i < kPW; ++i) {
                cur[i] = nxt[i];
                da[(l - 1) * kPW + i] = nxt[i];
            }
        }
    }
}

// Weight gradients summed over rows: layer l (0..3): dW[o][i] += da_l[o]
// in_l[i], db[o] += da_l[o], with in_0 = gamma(x) (40 padded), in_l = h_{l-1};
// head: dw[i] += ds h_3[i], db += ds.  One block per chunk of rows, 256
// threads, each owning a 4 x 4 patch of the 64 x 64 product; every block
// writes its partial sums of all weights to its own row of `part`
// (k_grad_reduce adds the rows in block order, so the result is the same on
// every run).
constexpr int kWgThreads = 256;

__global__ __launch_bounds__(kWgThreads) void k_prop_wgrad(
    const float* __restrict__ gsave, const float* __restrict__ hsave,
    const float* __restrict__ dasave, const float* __restrict__ ds, long rows, int chunk,
    float* __restrict__ part) {
    float* __restrict__ grad = part + (size_t)blockIdx.x * kPN;
    const long r0 = (long)blockIdx.x * chunk;
    const long r1 = min(rows, r0 + chunk);
    if (r0 >= rows) return;
    const int t = threadIdx.x, ty = t >> 4, tx = t & 15;
    for (int l = 0; l < kPDepth; ++l) {
        const int fin = (l == 0) ? kPIn : kPW;
        float acc[4][4] = {};
        float accb[4] = {0.f, 0.f, 0.f, 0.f};
        for (long row = r0; row < r1; ++row) {
            const float4 a4 = *reinterpret_cast<const float4*>(dasave + row * (kPDepth * kPW) + l * kPW + ty * 4);
            float4 x4;
            if (l == 0) {
                x4 = tx * 4 < kPInPad ? *reinterpret_cast<const float4*>(gsave + row * kPInPad + tx * 4)
                                      : make_float4(0.f, 0.f, 0.f, 0.f);
            } else {
                x4 = *reinterpret_cast<const float4*>(hsave + row * (kPDepth * kPW) + (l - 1) * kPW + tx * 4);
            }
            const float a[4] = {a4.x, a4.y, a4.z, a4.w};
            const float x[4] = {x4.x, x4.y, x4.z, x4.w};
#pragma unroll
            for (int i = 0; i < 4; ++i) {
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], x[j], acc[i][j]);
                accb[i] += a[i];
            }
        }
        float* gW = grad + prop_off(l);
        float* gb = gW + kPW * fin;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int o = ty * 4 + i;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int in = tx * 4 + j;
                if (in < fin) gW[o * fin + in] = acc[i][j];
            }
            if (tx == 0) gb[o] = accb[i];
        }
    }
    // density head
    if (t < kPW + 1) {
        float acc = 0.f;
        for (long row = r0; row < r1; ++row)
            acc += ds[row] * (t < kPW ? hsave[row * (kPDepth * kPW) + (kPDepth - 1) * kPW + t] : 1.0f);
        grad[kPOffHead + t] = acc;
    }
}

// grad[i] = scale * sum over blocks b (in order) of part[b][i].
__global__ void k_grad_reduce(const float* __restrict__ part, int nblk, float scale,
                              float* __restrict__ grad) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kPN) return;
    float s = 0.0f;
    for (int b = 0; b < nblk; ++b) s += part[(size_t)b * kPN + i];
    grad[i] = s * scale;
}

__global__ void k_adam(float* __restrict__ W, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, int n, float lr, float b1, float b2, float eps,
                       float c1, float c2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    W[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

cudaError_t launch_adam(float* W, const float* g, float* m, float* v, int n, float lr, float b1,
                        float b2, float eps, float c1, float c2, cudaStream_t s) {
    note_launch();
    k_adam<<<(n + 255) / 256, 256, 0, s>>>(W, g, m, v, n, lr, b1, b2, eps, c1, c2);
    return cudaGetLastError();
}

// Targets: final weights of the full sampler re-binned onto nb equal
// intervals of [near, far] (interval floor((z - near)/(far - near) nb),
// clamped), normalised (uniform for a ray without weight).
__global__ void k_histogram(const Ray* __restrict__ rays, int n_rays, const float* __restrict__ za,
                            const float4* __restrict__ oa, int nc, const float* __restrict__ zb,
                            const float4* __restrict__ ob, int nf, int nb, float near_z,
                            float far_z, float* __restrict__ hist) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n_rays) return;
    const float dn = rays[r].dnorm;
    const float* a = za + (size_t)r * nc;
    const float4* av = oa + (size_t)r * nc;
    const float* b = zb + (size_t)r * nf;
    const float4* bv = ob + (size_t)r * nf;
    float* h = hist + (size_t)r * nb;
    for (int i = 0; i < nb; ++i) h[i] = 0.0f;
    int ia = 0, ib = 0;
    auto take = [&](float& z, float4& v) {
        if (ib >= nf || (ia < nc && a[ia] <= b[ib])) { z = a[ia]; v = av[ia]; ++ia; }
        else { z = b[ib]; v = bv[ib]; ++ib; }
    };
    const int n = nc + nf;
    float zcur, znext = 0.f;
    float4 vcur, vnext = make_float4(0.f, 0.f, 0.f, 0.f);
    take(zcur, vcur);
    float T = 1.0f, tot = 0.0f;
    for (int k = 0; k < n; ++k) {
        if (k < n - 1) take(znext, vnext);
        const float delta = (k < n - 1) ? (znext - zcur) * dn : 1e10f;
        const float a_k = 1.0f - expf(-fmaxf(vcur.x, 0.0f) * delta);
        const float w = T * a_k;
        T *= (1.0f - a_k);
        int bin = (int)floorf((zcur - near_z) / (far_z - near_z) * (float)nb);
        bin = bin < 0 ? 0 : (bin > nb - 1 ? nb - 1 : bin);
        h[bin] += w;
        tot += w;
        zcur = znext; vcur = vnext;
    }
    for (int i = 0; i < nb; ++i) h[i] = tot > 0.0f ? h[i] / tot : 1.0f / (float)nb;
}

// Unpack rays into (o, d) arrays for training.
__global__ void k_rays_to_od(const Ray* __restrict__ rays, int n, float* __restrict__ O,
                             float* __restrict__ D) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    const Ray R = rays[r];
    O[3 * r] = R.ox; O[3 * r + 1] = R.oy; O[3 * r + 2] = R.oz;
    D[3 * r] = R.dx; D[3 * r + 1] = R.dy; D[3 * r + 2] = R.dz;
}

__global__ void k_gather_rows(const float* __restrict__ src, const int* __restrict__ perm, int n,
                              int width, float* __restrict__ dst) {
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long)n * width) return;
    const long r = t / width;
    const int c = (int)(t - r * width);
    dst[t] = src[(long)perm[r] * width + c];
}

static int grid_for(long rows, int tb) {
    long g = (rows + tb - 1) / tb;
    return (int)(g < 4096 ? (g < 1 ? 1 : g) : 4096);
}

// ----------------------------------------------------------------- host API
int proposal_alloc(mcl_map* m) {
    int rc;
    if ((rc = cuda_check(cudaMalloc(&m->prop_w, sizeof(float) * kPN * 4), "proposal weights"))) return rc;
    m->prop_m = m->prop_w + kPN;
    m->prop_v = m->prop_w + 2 * kPN;
    m->prop_g = m->prop_w + 3 * kPN;
    if ((rc = cuda_check(cudaMemset(m->prop_w, 0, sizeof(float) * kPN * 4), "proposal clear"))) return rc;
    if ((rc = cuda_check(cudaMalloc(&m->prop_packed, 4 * 64 * 64 * sizeof(uint16_t)), "proposal bf16")) ||
        (rc = cuda_check(cudaMemset(m->prop_packed, 0, 4 * 64 * 64 * sizeof(uint16_t)), "proposal bf16")) ||
        (rc = cuda_check(cudaMalloc(&m->prop_abort, sizeof(int)), "proposal abort flag")))
        return rc;
    int dev = 0, major = 0, minor = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&m->n_sm, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
    cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
    if (major == 10 && minor == 3 && (rc = cuda_check(prop_tc_prepare(), "proposal tc smem"))) return rc;
    if ((rc = cuda_check(cudaFuncSetAttribute(k_prop_infer, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              kPN * (int)sizeof(float)),
                         "proposal smem")))
        return rc;
    if ((rc = cuda_check(cudaFuncSetAttribute(k_prop_fwd_train,
                                              cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              kPN * (int)sizeof(float)),
                         "proposal smem")))
        return rc;
    return cuda_check(cudaFuncSetAttribute(k_prop_bwd_data, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           kPN * (int)sizeof(float)),
                      "proposal smem");
}

// Proposal densities at the stratified samples: the tensor-core kernel for
// the BF16 / FP8 forms, the FP32 kernel for the FP32 form.
cudaError_t launch_prop_infer(mcl_map* m, int precision, const Ray* rays, const float* z, int n_p,
                              int n_rays, const int* n_rays_dev, float4* out, cudaStream_t s) {
    if (precision != MCL_PREC_FP32 && mlp_tc_available(m, MCL_PREC_BF16))
        return launch_prop_infer_tc(m, rays, z, n_p, n_rays, n_rays_dev, out, m->n_sm, s);
    const long rows = (long)n_rays * n_p;
    note_launch();
    k_prop_infer<<<grid_for(rows, 128), 128, kPN * sizeof(float), s>>>(m->prop_w, rays, z, n_p, rows,
                                                                        n_rays_dev, out);
    return cudaGetLastError();
}

cudaError_t launch_histogram(const Ray* rays, int n_rays, const float* zc, const float4* oc, int nc,
                             const float* zf, const float4* of, int nf, int nb, float near_z,
                             float far_z, float* hist, cudaStream_t s) {
    note_launch();
    k_histogram<<<(n_rays + 127) / 128, 128, 0, s>>>(rays, n_rays, zc, oc, nc, zf, of, nf, nb,
                                                      near_z, far_z, hist);
    return cudaGetLastError();
}

// Scratch of one training batch (caller-owned buffers).
struct PropBatch {
    float* part; // [blocks of k_prop_wgrad][kPN]
    float* g;    // [rows][40]
    float* h;    // [rows][4][64]
    float* da;   // [rows][4][64]
    float* s;    // [rows]
    float* ds;   // [rows]
};

constexpr int kWgChunk = 512;   // rows per block of k_prop_wgrad

// Loss (summed into *loss_acc, scaled by `lscale`) and gradient (written to
// m->prop_g, scaled by `scale`) of n rays (O, D [n,3]) against hist [n, nb].
static cudaError_t prop_loss_grad_batch(mcl_map* m, const float* O, const float* D, int n, int nb,
                                        float near_z, float far_z, const float* hist, float scale,
                                        double lscale, const PropBatch& sb, double* loss_acc,
                                        cudaStream_t s) {
    const long rows = (long)n * nb;
    note_launch(5);
    k_prop_fwd_train<<<grid_for(rows, 128), 128, kPN * sizeof(float), s>>>(
        m->prop_w, O, D, n, nb, near_z, far_z, sb.g, sb.h, sb.s);
    k_prop_loss_bwd<<<(n + 127) / 128, 128, 0, s>>>(sb.s, D, n, nb, near_z, far_z, hist, scale, lscale,
                                                    sb.ds, loss_acc);
    k_prop_bwd_data<<<grid_for(rows, 128), 128, kPN * sizeof(float), s>>>(m->prop_w, sb.h, sb.ds,
                                                                         rows, sb.da);
    const int nblk = (int)((rows + kWgChunk - 1) / kWgChunk);
    k_prop_wgrad<<<nblk, kWgThreads, 0, s>>>(sb.g, sb.h, sb.da, sb.ds, rows, kWgChunk, sb.part);
    k_grad_reduce<<<(kPN + 255) / 256, 256, 0, s>>>(sb.part, nblk, 1.0f, m->prop_g);
    return cudaGetLastError();
}

static int alloc_batch(PropBatch& b, long rows) {
    int rc;
    const long nblk = (rows + kWgChunk - 1) / kWgChunk;
    if ((rc = cuda_check(cudaMalloc(&b.part, sizeof(float) * nblk * kPN), "batch partials"))) return rc;
    if ((rc = cuda_check(cudaMalloc(&b.g, sizeof(float) * rows * kPInPad), "batch g"))) return rc;
    if ((rc = cuda_check(cudaMalloc(&b.h, sizeof(float) * rows * kPDepth * kPW), "batch h"))) return rc;
    if ((rc = cuda_check(cudaMalloc(&b.da, sizeof(float) * rows * kPDepth * kPW), "batch da"))) return rc;
    if ((rc = cuda_check(cudaMalloc(&b.s, sizeof(float) * rows), "batch s"))) return rc;
    return cuda_check(cudaMalloc(&b.ds, sizeof(float) * rows), "batch ds");
}

static void free_batch(PropBatch& b) {
    if (b.part) cudaFree(b.part);
    if (b.g) cudaFree(b.g);
    if (b.h) cudaFree(b.h);
    if (b.da) cudaFree(b.da);
    if (b.s) cudaFree(b.s);
    if (b.ds) cudaFree(b.ds);
    b = PropBatch{};
}

int proposal_loss_grad(mcl_map* m, const float* O, const float* D, int n, int nb, float near_z,
                       float far_z, const float* hist, double* d_loss, float* d_grad,
                       cudaStream_t s) {
    PropBatch b{};
    int rc = alloc_batch(b, (long)n * nb);
    if (!rc) rc = cuda_check(cudaMemsetAsync(d_loss, 0, sizeof(double), s), "clear loss");
    if (!rc)
        rc = cuda_check(prop_loss_grad_batch(m, O, D, n, nb, near_z, far_z, hist, 1.0f / n, 1.0 / n, b, d_loss, s),
                        "proposal loss/grad");
    if (!rc)
        rc = cuda_check(cudaMemcpyAsync(d_grad, m->prop_g, sizeof(float) * kPN, cudaMemcpyDeviceToDevice, s),
                        "copy grad");
    if (!rc) rc = cuda_check(cudaStreamSynchronize(s), "proposal sync");
    free_batch(b);
    return rc;
}

int proposal_train(mcl_map* m, const float* d_poses, int n_poses, const int32_t* d_pixels, int B,
                   const mcl_intrinsics& K, int level, const mcl_opts& o, const mcl_train_cfg& cfg,
                   float* d_loss_log, cudaStream_t s,
                   int (*render_chunk)(mcl_map*, const float*, int, const mcl_intrinsics*, int,
                                       const int32_t*, int, const mcl_opts*, cudaStream_t)) {
    const int nb = cfg.n_bins;
    const long n_rays = (long)n_poses * B;
    int rc = 0;
    float *O = nullptr, *D = nullptr, *hist = nullptr, *Ob = nullptr, *Db = nullptr, *Hb = nullptr;
    int* perm_d = nullptr;
    double* loss_acc = nullptr;
    PropBatch b{};
    const int batch = cfg.batch_rays;
    auto cleanup = [&]() {
        if (O) cudaFree(O);
        if (D) cudaFree(D);
        if (hist) cudaFree(hist);
        if (Ob) cudaFree(Ob);
        if (Db) cudaFree(Db);
        if (Hb) cudaFree(Hb);
        if (perm_d) cudaFree(perm_d);
        if (loss_acc) cudaFree(loss_acc);
        free_batch(b);
    };
    if ((rc = cuda_check(cudaMalloc(&O, sizeof(float) * 3 * n_rays), "train O")) ||
        (rc = cuda_check(cudaMalloc(&D, sizeof(float) * 3 * n_rays), "train D")) ||
        (rc = cuda_check(cudaMalloc(&hist, sizeof(float) * nb * n_rays), "train hist")) ||
        (rc = cuda_check(cudaMalloc(&Ob, sizeof(float) * 3 * batch), "batch O")) ||
        (rc = cuda_check(cudaMalloc(&Db, sizeof(float) * 3 * batch), "batch D")) ||
        (rc = cuda_check(cudaMalloc(&Hb, sizeof(float) * nb * batch), "batch hist")) ||
        (rc = cuda_check(cudaMalloc(&perm_d, sizeof(int) * n_rays), "perm")) ||
        (rc = cuda_check(cudaMalloc(&loss_acc, sizeof(double)), "loss")) ||
        (rc = alloc_batch(b, (long)batch * nb))) {
        cleanup();
        return rc;
    }
    // 1) targets from the full sampler, in chunks of poses that fit the workspace
    const int chunk_poses = std::max(1, std::min(n_poses, m->cfg.max_rays / B));
    for (int p0 = 0; p0 < n_poses && !rc; p0 += chunk_poses) {
        const int np = std::min(chunk_poses, n_poses - p0);
        const int nr = np * B;
        rc = render_chunk(m, d_poses + 12 * (size_t)p0, np, &K, level, d_pixels, B, &o, s);
        if (rc) break;
        rc = cuda_check(launch_histogram(m->rays, nr, m->zc, m->out_c, o.n_coarse, m->zf, m->out_f,
                                         o.n_fine, nb, o.near_z, o.far_z,
                                         hist + (size_t)p0 * B * nb, s),
                        "histogram");
        if (rc) break;
        note_launch();
        k_rays_to_od<<<(nr + 127) / 128, 128, 0, s>>>(m->rays, nr, O + 3 * (size_t)p0 * B,
                                                       D + 3 * (size_t)p0 * B);
        rc = cuda_check(cudaGetLastError(), "rays to o, d");
    }
    // 2) epochs of Adam over shuffled mini-batches
    std::mt19937_64 rng(cfg.seed);
    std::vector<int> perm(n_rays);
    for (long i = 0; i < n_rays; ++i) perm[i] = (int)i;
    int step = m->prop_step;
    const long steps_per_epoch = (n_rays + batch - 1) / batch;
    const double total_steps = (double)cfg.epochs * steps_per_epoch;
    long local_step = 0;
    const double decay = cfg.lr_end > 0.f ? log((double)cfg.lr_end / cfg.lr) : 0.0;
    for (int ep = 0; ep < cfg.epochs && !rc; ++ep) {
        std::shuffle(perm.begin(), perm.end(), rng);
        if ((rc = cuda_check(cudaMemcpyAsync(perm_d, perm.data(), sizeof(int) * n_rays,
                                             cudaMemcpyHostToDevice, s),
                             "upload permutation")))
            break;
        if ((rc = cuda_check(cudaMemsetAsync(loss_acc, 0, sizeof(double), s), "clear loss"))) break;
        for (long b0 = 0; b0 < n_rays && !rc; b0 += batch) {
            const int nbat = (int)std::min<long>(batch, n_rays - b0);
            note_launch(3);
            k_gather_rows<<<(nbat * 3 + 255) / 256, 256, 0, s>>>(O, perm_d + b0, nbat, 3, Ob);
            k_gather_rows<<<(nbat * 3 + 255) / 256, 256, 0, s>>>(D, perm_d + b0, nbat, 3, Db);
            k_gather_rows<<<(nbat * nb + 255) / 256, 256, 0, s>>>(hist, perm_d + b0, nbat, nb, Hb);
            rc = cuda_check(prop_loss_grad_batch(m, Ob, Db, nbat, nb, o.near_z, o.far_z, Hb,
                                                 1.0f / nbat, 1.0, b, loss_acc, s),
                            "proposal batch");
            if (rc) break;
            ++step;
            const double frac = total_steps > 1 ? (double)local_step / (total_steps - 1) : 0.0;
            const float lr = (float)(cfg.lr * exp(decay * frac));
            ++local_step;
            const float c1 = 1.0f - powf(cfg.beta1, (float)step);
            const float c2 = 1.0f - powf(cfg.beta2, (float)step);
            note_launch();
            k_adam<<<(kPN + 255) / 256, 256, 0, s>>>(m->prop_w, m->prop_g, m->prop_m, m->prop_v, kPN,
                                                     lr, cfg.beta1, cfg.beta2, cfg.eps, c1, c2);
            rc = cuda_check(cudaGetLastError(), "adam");
        }
        if (!rc && d_loss_log) {
            double L = 0.0;
            rc = cuda_check(cudaMemcpyAsync(&L, loss_acc, sizeof(double), cudaMemcpyDeviceToHost, s),
                            "read loss");
            if (!rc) rc = cuda_check(cudaStreamSynchronize(s), "sync");
            const float mean = (float)(L / (double)n_rays);
            if (!rc)
                rc = cuda_check(cudaMemcpyAsync(d_loss_log + ep, &mean, sizeof(float),
                                                cudaMemcpyHostToDevice, s),
                                "write loss");
            if (!rc) rc = cuda_check(cudaStreamSynchronize(s), "sync");
        }
    }
    m->prop_step = step;
    if (!rc) rc = cuda_check(prop_tc_pack(m, s), "pack proposal");
    if (!rc) rc = cuda_check(cudaStreamSynchronize(s), "train sync");
    cleanup();
    if (!rc) m->has_proposal = true;
    return rc;
}

}  // namespace mcl
