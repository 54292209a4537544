// fit.cu -- fitting the NeRF map's FP32 weights to samples of a field: points
// x with view directions and targets (density, r, g, b), loss
//   L = mean over points of  w_sigma (sigma_raw(x) - sigma_t)^2 + |rgb(x, d) - rgb_t|^2,
// minimised by Adam with the library's own kernels: the plain FP32 form's
// forward (gamma(x), SGEMM layers, heads) with every layer's output kept, a
// backward pass of SGEMMs on transposed weights with ReLU masks, and weight
// gradients summed over the batch in a fixed order (the same inputs give the
// same weights).  The map's tensor-core forms are rebuilt from the fitted
// weights.  This stands in for training a map on images (Eq. 2, out of
// scope): it gives maps of analytic scenes whose weights the library itself
// produced.
#include <string.h>

#include <algorithm>
#include <random>
#include <vector>

#include "internal.cuh"

namespace mcl {

namespace {

constexpr int kWgRows = 1024;   // rows per partial sum of a weight gradient
constexpr int kWgTile = 64;     // 64 x 64 outputs per block of k_wgrad

struct FitBuf {
    long B = 0;                 // points per batch
    float *x = nullptr, *dir = nullptr, *tgt = nullptr;   // batch inputs
    Ray* rays = nullptr;
    float *gd = nullptr, *z = nullptr, *gx = nullptr;     // gamma(d) [B,32], z = 0, gamma(x) [B,64]
    float* h = nullptr;         // trunk outputs [8][B][256]
    float* feat = nullptr;      // [B][256]
    float* hid = nullptr;       // [B][256] (128 used)
    float4* out = nullptr;      // [B] (sigma_raw, rgb)
    float *dA = nullptr, *dB = nullptr, *dhid = nullptr;  // [B][256]
    float* dlog = nullptr;      // [B][4]: d rgb logits, d sigma
    float* part = nullptr;      // partial weight gradients
    float* partb = nullptr;     // partial bias gradients
    float* wt = nullptr;        // transposed weights [256][256]
    float* zeros = nullptr;     // [256]
    double* lpart = nullptr;    // per-block loss partials
    double* loss = nullptr;
    float* grad = nullptr;      // [w32_n] gradient in the padded layout
    float *m1 = nullptr, *m2 = nullptr;   // Adam moments
};

void free_buf(FitBuf& b) {
    void* ptrs[] = {b.x, b.dir, b.tgt, b.rays, b.gd, b.z, b.gx, b.h, b.feat, b.hid, b.out, b.dA,
                    b.dB, b.dhid, b.dlog, b.part, b.partb, b.wt, b.zeros, b.lpart, b.loss, b.grad,
                    b.m1, b.m2};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    b = FitBuf{};
}

int alloc_buf(mcl_map* m, FitBuf& b, long B, bool adam) {
    b.B = B;
    const long nchunk = (B + kWgRows - 1) / kWgRows;
    struct {
        void** p;
        size_t bytes;
    } a[] = {
        {(void**)&b.x, sizeof(float) * 3 * B},        {(void**)&b.dir, sizeof(float) * 3 * B},
        {(void**)&b.tgt, sizeof(float) * 4 * B},      {(void**)&b.rays, sizeof(Ray) * B},
        {(void**)&b.gd, sizeof(float) * kGdPad * B},  {(void**)&b.z, sizeof(float) * B},
        {(void**)&b.gx, sizeof(float) * kGxPad * B},  {(void**)&b.h, sizeof(float) * 8 * kWidth * B},
        {(void**)&b.feat, sizeof(float) * kWidth * B}, {(void**)&b.hid, sizeof(float) * kWidth * B},
        {(void**)&b.out, sizeof(float4) * B},          {(void**)&b.dA, sizeof(float) * kWidth * B},
        {(void**)&b.dB, sizeof(float) * kWidth * B},   {(void**)&b.dhid, sizeof(float) * kWidth * B},
        {(void**)&b.dlog, sizeof(float) * 4 * B},
        {(void**)&b.part, sizeof(float) * nchunk * kWidth * (kWidth + kGxPad)},
        {(void**)&b.partb, sizeof(float) * nchunk * kWidth},
        {(void**)&b.wt, sizeof(float) * kWidth * kWidth}, {(void**)&b.zeros, sizeof(float) * kWidth},
        {(void**)&b.lpart, sizeof(double) * ((B + 255) / 256)}, {(void**)&b.loss, sizeof(double)},
        {(void**)&b.grad, sizeof(float) * m->w32_n},
    };
    int rc;
    for (auto& e : a)
        if ((rc = cuda_check(cudaMalloc(e.p, e.bytes), "fit buffers"))) return rc;
    if (adam) {
        if ((rc = cuda_check(cudaMalloc(&b.m1, sizeof(float) * m->w32_n), "fit moments")) ||
            (rc = cuda_check(cudaMalloc(&b.m2, sizeof(float) * m->w32_n), "fit moments")))
            return rc;
        cudaMemset(b.m1, 0, sizeof(float) * m->w32_n);
        cudaMemset(b.m2, 0, sizeof(float) * m->w32_n);
    }
    cudaMemset(b.zeros, 0, sizeof(float) * kWidth);
    return MCL_OK;
}

// Rows idx[r0 .. r0 + n) of x, dir, tgt into the batch buffers.
__global__ void k_fit_gather(const float* __restrict__ x, const float* __restrict__ dir,
                             const float* __restrict__ tgt, const int* __restrict__ idx, long r0,
                             int n, float* __restrict__ bx, float* __restrict__ bd,
                             float* __restrict__ bt) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const long k = idx ? idx[r0 + i] : r0 + i;
    for (int c = 0; c < 3; ++c) {
        bx[3 * i + c] = x[3 * k + c];
        bd[3 * i + c] = dir[3 * k + c];
    }
    for (int c = 0; c < 4; ++c) bt[4 * i + c] = tgt[4 * k + c];
}

// Loss terms and output gradients of each point; per-block FP64 loss sums.
__global__ __launch_bounds__(256) void k_fit_loss(const float4* __restrict__ out,
                                                  const float* __restrict__ tgt, int n, float wsig,
                                                  float scale, float* __restrict__ dlog,
                                                  double* __restrict__ lpart) {
    __shared__ double sh[256];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double L = 0.0;
    if (i < n) {
        const float4 o = out[i];
        const float* t = tgt + 4 * i;
        const float ds = o.x - t[0];
        const float c[3] = {o.y, o.z, o.w};
        L = (double)wsig * ds * ds;
        for (int k = 0; k < 3; ++k) {
            const float e = c[k] - t[1 + k];
            L += (double)e * e;
            dlog[4 * i + k] = 2.0f * e * c[k] * (1.0f - c[k]) * scale;
        }
        dlog[4 * i + 3] = 2.0f * wsig * ds * scale;
    }
    sh[threadIdx.x] = L;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) lpart[blockIdx.x] = sh[0];
}

__global__ void k_fit_loss_sum(const double* __restrict__ lpart, int nblk, double scale,
                               double* __restrict__ loss, float* __restrict__ log_entry) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double s = 0.0;
    for (int b = 0; b < nblk; ++b) s += lpart[b];
    *loss = s * scale;
    if (log_entry) *log_entry = (float)(s * scale);
}

// RGB output layer backward: dhid[p][k] = sum_c dlog[p][c] W_o[c][k], masked
// by hid[p][k] > 0 (the hidden layer's ReLU).
__global__ void k_fit_drgb(const float* __restrict__ dlog, const float* __restrict__ Wo,
                           const float* __restrict__ hid, long n, float* __restrict__ dhid) {
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * kRgbW) return;
    const long p = t / kRgbW;
    const int k = (int)(t - p * kRgbW);
    float s = 0.f;
    for (int c = 0; c < 3; ++c) s = fmaf(dlog[4 * p + c], Wo[c * kRgbW + k], s);
    dhid[p * kWidth + k] = hid[p * kWidth + k] > 0.f ? s : 0.f;
}

// Top of the trunk: d = (d_feature_path + d_sigma w_sigma) masked by h8 > 0.
__global__ void k_fit_dtop(float* __restrict__ d, const float* __restrict__ dlog,
                           const float* __restrict__ wsig, const float* __restrict__ h8, long n) {
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * kWidth) return;
    const long p = t / kWidth;
    const int k = (int)(t - p * kWidth);
    const float v = fmaf(dlog[4 * p + 3], wsig[k], d[t]);
    d[t] = h8[t] > 0.f ? v : 0.f;
}

__global__ void k_fit_mask(float* __restrict__ d, const float* __restrict__ h, long n) {
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n && !(h[t] > 0.f)) d[t] = 0.f;
}

// Wt[k][o] = W[o][k] for o < n_out, k < n_in (W row stride ldw).
__global__ void k_fit_transpose(const float* __restrict__ W, int ldw, int n_out, int n_in,
                                float* __restrict__ Wt) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_out * n_in) return;
    const int k = t / n_out, o = t - k * n_out;
    Wt[t] = W[o * ldw + k];
}

// Partial weight gradients of one row chunk:
//   part[c][o][k] = sum_{rows p of chunk c} dY[p][o] X[p][k],  X = [X1 | X2],
//   partb[c][o] = sum_p dY[p][o].
// 64 x 64 outputs per block (256 threads, 4 x 4 each), rows staged 16 at a
// time in shared memory; every sum runs over the chunk's rows in order.
__global__ __launch_bounds__(256) void k_wgrad(const float* __restrict__ dY, int ldy, int N,
                                               const float* __restrict__ X1, int ld1, int K1,
                                               const float* __restrict__ X2, int ld2, int K2,
                                               long rows, float* __restrict__ part,
                                               float* __restrict__ partb) {
    __shared__ float As[16][kWgTile + 4];
    __shared__ float Bs[16][kWgTile + 4];
    const int K = K1 + K2;
    const int o0 = blockIdx.x * kWgTile, k0 = blockIdx.y * kWgTile, c = blockIdx.z;
    const long p0 = (long)c * kWgRows, p1 = min(rows, p0 + kWgRows);
    const int t = threadIdx.x, ty = t >> 4, tx = t & 15;
    float acc[4][4] = {};
    float accb[4] = {0.f, 0.f, 0.f, 0.f};
    for (long pb = p0; pb < p1; pb += 16) {
        // stage 16 rows: thread t loads element (row t / 16, 4 columns (t % 16) * 4)
        {
            const int r = t >> 4, cc = (t & 15) * 4;
            const long p = pb + r;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int o = o0 + cc + j, k = k0 + cc + j;
                As[r][cc + j] = (p < p1 && o < N) ? dY[p * ldy + o] : 0.f;
                float xv = 0.f;
                if (p < p1 && k < K) xv = k < K1 ? X1[p * ld1 + k] : X2[p * ld2 + (k - K1)];
                Bs[r][cc + j] = xv;
            }
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < 16; ++r) {
            float a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                a[i] = As[r][ty * 4 + i];
                b[i] = Bs[r][tx * 4 + i];
            }
#pragma unroll
            for (int i = 0; i < 4; ++i) {
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
                accb[i] += a[i];
            }
        }
        __syncthreads();
    }
    float* pc = part + (size_t)c * N * K;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int o = o0 + ty * 4 + i;
        if (o >= N) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int k = k0 + tx * 4 + j;
            if (k < K) pc[(size_t)o * K + k] = acc[i][j];
        }
        if (blockIdx.y == 0 && tx == 0) partb[(size_t)c * N + o] = accb[i];
    }
}

// gW[o][k] (row stride ldg) = sum over chunks in order of part[c][o][k];
// gb[o] likewise from partb.
__global__ void k_wgrad_reduce(const float* __restrict__ part, const float* __restrict__ partb,
                               int nchunk, int N, int K, float* __restrict__ gW, int ldg,
                               float* __restrict__ gb) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < N * K) {
        const int o = t / K, k = t - o * K;
        float s = 0.f;
        for (int c = 0; c < nchunk; ++c) s += part[(size_t)c * N * K + t];
        gW[(size_t)o * ldg + k] = s;
    }
    if (t < N) {
        float s = 0.f;
        for (int c = 0; c < nchunk; ++c) s += partb[(size_t)c * N + t];
        gb[t] = s;
    }
}

cudaError_t wgrad(const FitBuf& b, long n, const float* dY, int ldy, int N, const float* X1,
                  int ld1, int K1, const float* X2, int ld2, int K2, float* gW, int ldg,
                  float* gb, cudaStream_t s) {
    const int K = K1 + K2;
    const int nchunk = (int)((n + kWgRows - 1) / kWgRows);
    dim3 grid((N + kWgTile - 1) / kWgTile, (K + kWgTile - 1) / kWgTile, nchunk);
    note_launch(2);
    k_wgrad<<<grid, 256, 0, s>>>(dY, ldy, N, X1, ld1, K1, X2, ld2, K2, n, b.part, b.partb);
    k_wgrad_reduce<<<(N * K + 255) / 256, 256, 0, s>>>(b.part, b.partb, nchunk, N, K, gW, ldg, gb);
    return cudaGetLastError();
}

// Loss and gradient (padded layout, into b.grad) of the first n points held
// in b.x / b.dir / b.tgt; the loss (mean) into *b.loss and *log_entry.
cudaError_t loss_and_grad(mcl_map* m, const FitBuf& b, long n, float wsig, float* log_entry,
                          cudaStream_t s) {
    const LayerF32* L = m->L;
    cudaError_t e;
    float* h = b.h;
    auto H = [&](int l) { return h + (size_t)l * kWidth * n; };   // output of trunk layer l + 1
    auto off = [&](const float* p) { return b.grad + (p - m->w32); };
    // ---- forward, every layer's output kept
    if ((e = launch_query_setup(b.x, b.dir, (int)n, b.rays, b.gd, b.z, s)) ||
        (e = fp32_pe(b.rays, b.z, (int)n, b.gx, s)) ||
        (e = fp32_gemm(b.gx, kGxPad, kGxPad, nullptr, 0, 0, 0, 1, L[0].W, L[0].b, kWidth, H(0), kWidth,
                       (int)n, true, s)))
        return e;
    for (int l = 1; l < kDepth; ++l) {
        if (l == kSkip)
            e = fp32_gemm(H(l - 1), kWidth, kWidth, b.gx, kGxPad, kGxPad, 0, 1, L[l].W, L[l].b, kWidth,
                          H(l), kWidth, (int)n, true, s);
        else
            e = fp32_gemm(H(l - 1), kWidth, kWidth, nullptr, 0, 0, 0, 1, L[l].W, L[l].b, kWidth, H(l),
                          kWidth, (int)n, true, s);
        if (e) return e;
    }
    if ((e = fp32_gemm(H(7), kWidth, kWidth, nullptr, 0, 0, 0, 1, L[9].W, L[9].b, kWidth, b.feat,
                       kWidth, (int)n, false, s)) ||
        (e = fp32_gemm(b.feat, kWidth, kWidth, b.gd, kGdPad, kGdPad, 0, 1, L[10].W, L[10].b, kRgbW,
                       b.hid, kWidth, (int)n, true, s)) ||
        (e = fp32_heads(H(7), L[8], b.hid, L[11], (int)n, b.out, s)))
        return e;
    // ---- loss and output gradients
    const int nblk = (int)((n + 255) / 256);
    note_launch(2);
    k_fit_loss<<<nblk, 256, 0, s>>>(b.out, b.tgt, (int)n, wsig, 1.0f / (float)n, b.dlog, b.lpart);
    k_fit_loss_sum<<<1, 32, 0, s>>>(b.lpart, nblk, 1.0 / (double)n, b.loss, log_entry);
    // ---- backward
    // RGB output layer (3 x 128): gradient, then d hid (masked)
    if ((e = wgrad(b, n, b.dlog, 4, 3, b.hid, kWidth, kRgbW, nullptr, 0, 0, off(L[11].W), L[11].k_pad,
                   off(L[11].b), s)))
        return e;
    note_launch();
    k_fit_drgb<<<(unsigned)((n * kRgbW + 255) / 256), 256, 0, s>>>(b.dlog, L[11].W, b.hid, n, b.dhid);
    // RGB hidden layer (128 x [feature 256 | gamma(d) 32]), then d feature
    if ((e = wgrad(b, n, b.dhid, kWidth, kRgbW, b.feat, kWidth, kWidth, b.gd, kGdPad, kGdPad,
                   off(L[10].W), L[10].k_pad, off(L[10].b), s)))
        return e;
    note_launch();
    k_fit_transpose<<<(kRgbW * kWidth + 255) / 256, 256, 0, s>>>(L[10].W, L[10].k_pad, kRgbW, kWidth, b.wt);
    if ((e = fp32_gemm(b.dhid, kWidth, kRgbW, nullptr, 0, 0, 0, 1, b.wt, b.zeros, kWidth, b.dA, kWidth,
                       (int)n, false, s)))
        return e;
    // feature layer (linear 256 x 256), then d h8 through it
    if ((e = wgrad(b, n, b.dA, kWidth, kWidth, H(7), kWidth, kWidth, nullptr, 0, 0, off(L[9].W),
                   L[9].k_pad, off(L[9].b), s)))
        return e;
    note_launch();
    k_fit_transpose<<<(kWidth * kWidth + 255) / 256, 256, 0, s>>>(L[9].W, L[9].k_pad, kWidth, kWidth, b.wt);
    if ((e = fp32_gemm(b.dA, kWidth, kWidth, nullptr, 0, 0, 0, 1, b.wt, b.zeros, kWidth, b.dB, kWidth,
                       (int)n, false, s)))
        return e;
    // density head (1 x 256) gradient from d sigma (column 3 of dlog)
    if ((e = wgrad(b, n, b.dlog + 3, 4, 1, H(7), kWidth, kWidth, nullptr, 0, 0, off(L[8].W),
                   L[8].k_pad, off(L[8].b), s)))
        return e;
    note_launch();
    k_fit_dtop<<<(unsigned)((n * kWidth + 255) / 256), 256, 0, s>>>(b.dB, b.dlog, L[8].W, H(7), n);
    // trunk layers 8 .. 1: cur holds d of layer l's pre-activation
    float* cur = b.dB;
    float* nxt = b.dA;
    for (int l = kDepth - 1; l >= 0; --l) {
        if (l == 0)
            e = wgrad(b, n, cur, kWidth, kWidth, b.gx, kGxPad, kGxPad, nullptr, 0, 0, off(L[0].W),
                      L[0].k_pad, off(L[0].b), s);
        else if (l == kSkip)
            e = wgrad(b, n, cur, kWidth, kWidth, H(l - 1), kWidth, kWidth, b.gx, kGxPad, kGxPad,
                      off(L[l].W), L[l].k_pad, off(L[l].b), s);
        else
            e = wgrad(b, n, cur, kWidth, kWidth, H(l - 1), kWidth, kWidth, nullptr, 0, 0, off(L[l].W),
                      L[l].k_pad, off(L[l].b), s);
        if (e) return e;
        if (l == 0) break;
        note_launch(2);
        k_fit_transpose<<<(kWidth * kWidth + 255) / 256, 256, 0, s>>>(L[l].W, L[l].k_pad, kWidth, kWidth,
                                                                     b.wt);
        if ((e = fp32_gemm(cur, kWidth, kWidth, nullptr, 0, 0, 0, 1, b.wt, b.zeros, kWidth, nxt, kWidth,
                           (int)n, false, s)))
            return e;
        k_fit_mask<<<(unsigned)((n * kWidth + 255) / 256), 256, 0, s>>>(nxt, H(l - 1), n * kWidth);
        std::swap(cur, nxt);
    }
    return cudaGetLastError();
}

}  // namespace

// Host copy of the FP32 weights in the blob layout of mcl_init_map.
int map_download(mcl_map* m, float* host_blob) {
    int fin[12], fout[12];
    blob_layer_shapes(fin, fout);
    std::vector<float> w(m->w32_n);
    int rc;
    if ((rc = cuda_check(cudaMemcpy(w.data(), m->w32, sizeof(float) * m->w32_n, cudaMemcpyDeviceToHost),
                         "download weights")))
        return rc;
    float* dst = host_blob;
    for (int l = 0; l < 12; ++l) {
        const size_t oW = m->L[l].W - m->w32, ob = m->L[l].b - m->w32;
        for (int o = 0; o < fout[l]; ++o)
            for (int i = 0; i < fin[l]; ++i) *dst++ = w[oW + (size_t)o * m->L[l].k_pad + i];
        for (int o = 0; o < fout[l]; ++o) *dst++ = w[ob + o];
    }
    return MCL_OK;
}

int map_loss_grad(mcl_map* m, const float* d_x, const float* d_dir, const float* d_target, int n,
                  float sigma_weight, double* d_loss, float* d_grad, cudaStream_t s) {
    FitBuf b;
    int rc = alloc_buf(m, b, n, false);
    if (!rc) {
        note_launch();
        k_fit_gather<<<(n + 255) / 256, 256, 0, s>>>(d_x, d_dir, d_target, nullptr, 0, n, b.x, b.dir, b.tgt);
        rc = cuda_check(cudaMemsetAsync(b.grad, 0, sizeof(float) * m->w32_n, s), "clear grad");
    }
    if (!rc) rc = cuda_check(loss_and_grad(m, b, n, sigma_weight, nullptr, s), "loss and gradient");
    if (!rc) rc = cuda_check(cudaMemcpyAsync(d_loss, b.loss, sizeof(double), cudaMemcpyDeviceToDevice, s),
                             "copy loss");
    if (!rc) rc = cuda_check(cudaStreamSynchronize(s), "loss sync");
    if (!rc) {
        // gradient in the blob layout: the same unpadding as the weights
        int fin[12], fout[12];
        blob_layer_shapes(fin, fout);
        std::vector<float> g(m->w32_n), out;
        rc = cuda_check(cudaMemcpy(g.data(), b.grad, sizeof(float) * m->w32_n, cudaMemcpyDeviceToHost),
                        "download grad");
        for (int l = 0; l < 12 && !rc; ++l) {
            const size_t oW = m->L[l].W - m->w32, ob = m->L[l].b - m->w32;
            for (int o = 0; o < fout[l]; ++o)
                for (int i = 0; i < fin[l]; ++i) out.push_back(g[oW + (size_t)o * m->L[l].k_pad + i]);
            for (int o = 0; o < fout[l]; ++o) out.push_back(g[ob + o]);
        }
        if (!rc)
            rc = cuda_check(cudaMemcpy(d_grad, out.data(), sizeof(float) * out.size(), cudaMemcpyHostToDevice),
                            "upload grad");
    }
    free_buf(b);
    return rc;
}

int fit_map(mcl_map* m, const float* d_x, const float* d_dir, const float* d_target, int n,
            const mcl_fit_cfg& cfg, float* d_loss_log, cudaStream_t s) {
    const long B = std::min(n, cfg.batch);
    FitBuf b;
    int* perm_d = nullptr;
    int rc = alloc_buf(m, b, B, true);
    if (!rc) rc = cuda_check(cudaMalloc(&perm_d, sizeof(int) * n), "fit permutation");
    std::mt19937_64 rng(cfg.seed);
    std::vector<int> perm(n);
    for (int i = 0; i < n; ++i) perm[i] = i;
    long pos = n;   // start of the next batch in the current permutation
    const float b1 = cfg.beta1, b2 = cfg.beta2;
    double c1 = 1.0, c2 = 1.0;
    const double decay = (cfg.lr_end > 0.f && cfg.steps > 1)
                             ? std::pow((double)cfg.lr_end / cfg.lr, 1.0 / (cfg.steps - 1))
                             : 1.0;
    for (int t = 0; t < cfg.steps && !rc; ++t) {
        if (pos + B > n) {
            // a new epoch: reshuffle (Fisher-Yates on the seeded generator)
            for (int i = n - 1; i > 0; --i) std::swap(perm[i], perm[rng() % (uint64_t)(i + 1)]);
            rc = cuda_check(cudaMemcpyAsync(perm_d, perm.data(), sizeof(int) * n, cudaMemcpyHostToDevice, s),
                            "upload permutation");
            if (!rc) rc = cuda_check(cudaStreamSynchronize(s), "permutation sync");
            pos = 0;
            if (rc) break;
        }
        note_launch();
        k_fit_gather<<<(unsigned)((B + 255) / 256), 256, 0, s>>>(d_x, d_dir, d_target, perm_d, pos, (int)B,
                                                              b.x, b.dir, b.tgt);
        pos += B;
        rc = cuda_check(cudaMemsetAsync(b.grad, 0, sizeof(float) * m->w32_n, s), "clear grad");
        if (!rc)
            rc = cuda_check(loss_and_grad(m, b, B, cfg.sigma_weight, d_loss_log ? d_loss_log + t : nullptr, s),
                            "fit step");
        c1 *= b1;
        c2 *= b2;
        const float lr = (float)(cfg.lr * std::pow(decay, (double)t));
        if (!rc)
            rc = cuda_check(launch_adam(m->w32, b.grad, b.m1, b.m2, (int)m->w32_n, lr, b1, b2, cfg.eps,
                                        (float)(1.0 - c1), (float)(1.0 - c2), s),
                            "fit adam");
    }
    if (!rc) rc = cuda_check(cudaStreamSynchronize(s), "fit sync");
    if (perm_d) cudaFree(perm_d);
    free_buf(b);
    return rc;
}

}  // namespace mcl
