// internal.cuh -- private declarations shared by the translation units of the
// MCL weight-update library (not part of the public ABI in include/mcl.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/mcl.h"

namespace mcl {

// Fixed architecture served by this build.
constexpr int kLxyz = 10, kLdir = 4, kDepth = 8, kWidth = 256, kSkip = 5, kRgbW = 128;
constexpr int kGx = 3 + 6 * kLxyz;   // 63
constexpr int kGd = 3 + 6 * kLdir;   // 27
constexpr int kGxPad = 64;           // gamma(x) padded to a multiple of 16
constexpr int kGdPad = 32;           // gamma(d) padded
constexpr int kMaxSamples = 512;     // n_coarse + n_fine
constexpr int kMaxCoarse = 256;
constexpr int kMaxFine = 256;

// Padded FP32 layer (row-major [n][k_pad], bias [n]).
struct LayerF32 {
    const float* W;
    const float* b;
    int n, k_pad;
};

// Device status word (one per map).
struct Status {
    int code;         // first MCL_ERR_* seen on the device, 0 if none
    int n_nonfinite;  // particles masked for a non-finite loss
};

// Ray record: o (xyz) + |d|; d (xyz), rounded to FP32; the FP32 rounding
// error of d (d = d_hi + d_lo to about 48 bits), so that paths that need x to
// better than FP32 can rebuild it.
struct __align__(16) Ray {
    float ox, oy, oz, dnorm;
    float dx, dy, dz, pad;
    float lx, ly, lz, pad2;
};

// Device-driven localisation loop (loop.cu).
constexpr int kLoopMaxQueries = 64;
constexpr int kLoopMaxPixels = 256;

struct LoopPlan {
    int total_rays, rows_c, rows_f, pad;
    unsigned long long t_start;   // global timer at the start of the iteration
    int ray_off[kLoopMaxQueries + 1];
    int N[kLoopMaxQueries], B[kLoopMaxQueries], factor[kLoopMaxQueries], Nnext[kLoopMaxQueries];
};

struct LoopQuery {
    int stage, iter_at_stage, N, n_surv, nonfinite, pad;
    double wspread;
};

struct LoopWork {
    LoopPlan* plan = nullptr;
    LoopQuery* qs = nullptr;
    int* n0 = nullptr;
    const float** imgs = nullptr;
    int32_t* pix = nullptr;
    float* P_next = nullptr;
    double* w = nullptr;
    uint8_t* mask = nullptr;
    int32_t* idx = nullptr;
    int max_rays_run = 0;
    cudaGraphExec_t exec = nullptr;
    unsigned long long key = 0;
    // capture stream (graph mode on the legacy default stream) and the
    // events that order it with the caller's stream
    cudaStream_t stream = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
};

}  // namespace mcl

// The map: weights in the forms each MLP path reads, plus the workspace.
struct mcl_map {
    mcl_map_config cfg;
    // FP32 padded layers: 0..7 trunk, 8 sigma(row vector), 9 feature,
    // 10 rgb_hidden ([feat | gamma(d) | 0]), 11 rgb_out.
    float* w32 = nullptr;
    size_t w32_n = 0;               // floats of w32 (padded layers)
    mcl::LayerF32 L[12];
    // tensor-core path weights (filled by mlp_tc_prepare)
    void* tc_blob = nullptr;
    size_t tc_bytes = 0;
    void* tc_aux = nullptr;
    // workspace
    mcl::Ray* rays = nullptr;     // [max_rays]
    float* gd = nullptr;          // [max_rays, 32] gamma(d)
    float* zc = nullptr;          // [max_rays * max_samples] coarse z
    float* zf = nullptr;          // [max_rays * max_samples] fine z
    float4* out_c = nullptr;      // [max_rays * max_samples] (sigma_raw, rgb)
    float4* out_f = nullptr;
    float4* obs = nullptr;        // [max_rays] observed colour per ray (fused epilogue)
    float* e_ray = nullptr;       // [max_rays] E*F
    double* logw64 = nullptr;     // [max_particles]
    unsigned long long* cdf = nullptr;  // [max_particles] resampling CDF
    mcl::Status* status = nullptr;
    // FP32-form activations (chunked)
    float* act0 = nullptr;
    float* act1 = nullptr;
    float* gxbuf = nullptr;
    int chunk_rows = 0;
    // per-phase timing (host side)
    struct Mark {
        int phase;
        cudaEvent_t a, b;
    };
    bool prof = false;
    std::vector<Mark> marks;
    std::vector<cudaEvent_t> pool;
    double phase_ms[MCL_N_PHASES] = {0};
    mcl::LoopWork loop;
    // learned proposal sampler: weights, Adam moments, gradient
    float* prop_w = nullptr;
    float* prop_m = nullptr;
    float* prop_v = nullptr;
    float* prop_g = nullptr;
    int prop_step = 0;
    bool has_proposal = false;
    uint16_t* prop_packed = nullptr;   // BF16 weights of the tensor-core proposal kernel
    int* prop_abort = nullptr;         // per-launch abort flag of that kernel
    int n_sm = 0;
    bool fuse_epilogue = false;        // tensor-core forms: fused ray epilogues (opt-in)
};

namespace mcl {

// Thread-local error reporting (api.cu).
int fail(int code, const char* fmt, ...);
void clear_error();
int cuda_check(cudaError_t e, const char* what);
// Count of kernels launched by the library (api.cu).
void note_launch(int n = 1);

// render.cu
// obs (optional): per-ray box-filtered colour of the level image at the
// ray's pixel (factor x factor block of the full-resolution W x H image;
// NaN for a pixel outside the level image).
cudaError_t launch_raygen(const float* particles, int N, const int32_t* pixels, int B,
                          float fx, float fy, float cx, float cy, const mcl_opts& o,
                          Ray* rays, float* gd, float* zc, cudaStream_t s,
                          const float* image = nullptr, int W = 0, int H = 0, int factor = 1,
                          float4* obs = nullptr);
cudaError_t launch_query_setup(const float* X, const float* D, int n, Ray* rays, float* gd,
                               float* z, cudaStream_t s);
cudaError_t launch_coarse_to_fine(const Ray* rays, int n_rays, const int* n_rays_dev,
                                  const float* zc, int nc, const float4* out_c, int nf, float* zf,
                                  cudaStream_t s);
cudaError_t launch_final_composite(const Ray* rays, int n_rays, const float* zc, const float4* out_c,
                                   int nc, const float* zf, const float4* out_f, int nf,
                                   const float* image, int W, int H, int factor,
                                   const int32_t* pixels, int B, const mcl_opts& o,
                                   float* e_ray, const mcl_debug* dbg, float* rgb_out,
                                   float* F_out, cudaStream_t s);
cudaError_t launch_weights(const float* e_ray, int N, int B, const mcl_opts& o, float* logw,
                           double* logw64, double* w, uint8_t* mask, float* S_dbg,
                           Status* status, cudaStream_t s);

// mlp_fp32.cu: (sigma_raw, rgb) for rows r = ray*S + k of the pass.
// rows_dev (optional): device-side row count (n_rays * S is the bound).
cudaError_t mlp_fp32(mcl_map* m, const Ray* rays, const float* gd, const float* z, int S,
                     int n_rays, float4* out, cudaStream_t s, const int* rows_dev = nullptr);

// mlp_fp32.cu building blocks reused by the map fitter (fit.cu): the FP32
// GEMM C = act([A1 | A2] W^T + b) (W [n_out][K1 + K2], n_out a multiple of
// 128, K1 and K2 multiples of 16), gamma(x) of points (rays with z = 0), and
// the density / colour heads (h [n,256] -> out.x; hid [n,256-stride] -> out.yzw).
cudaError_t fp32_gemm(const float* A1, int lda1, int K1, const float* A2, int lda2, int K2,
                      long a2_off, int a2_div, const float* W, const float* bias, int n_out,
                      float* C, int ldc, int M, bool relu, cudaStream_t s);
cudaError_t fp32_pe(const Ray* rays, const float* z, int n, float* gx, cudaStream_t s);
cudaError_t fp32_heads(const float* h, const LayerF32& sigma, const float* hid, const LayerF32& rgb,
                       int n, float4* out, cudaStream_t s);

// proposal.cu: one Adam step (bias corrections c1 = 1 - b1^t, c2 = 1 - b2^t).
cudaError_t launch_adam(float* W, const float* g, float* m, float* v, int n, float lr, float b1,
                        float b2, float eps, float c1, float c2, cudaStream_t s);

// api.cu: fan-in and fan-out of the 12 layers in blob order.
void blob_layer_shapes(int* fin, int* fout);

// fit.cu
int fit_map(mcl_map* m, const float* d_x, const float* d_dir, const float* d_target, int n,
            const mcl_fit_cfg& cfg, float* d_loss_log, cudaStream_t s);
int map_loss_grad(mcl_map* m, const float* d_x, const float* d_dir, const float* d_target, int n,
                  float sigma_weight, double* d_loss, float* d_grad, cudaStream_t s);
int map_download(mcl_map* m, float* host_blob);

// mlp_tc.cu
int mlp_tc_prepare(mcl_map* m, const float* host_blob);
void mlp_tc_free(mcl_map* m);
bool mlp_tc_available(const mcl_map* m, int precision);
int mlp_tc_set_variant(mcl_map* m, int precision, int variant);
int mlp_tc_autotune(mcl_map* m, int precision, long long rows, int* chosen, float* ms_out,
                    cudaStream_t s);
bool mlp_tc_tuned(const mcl_map* m, int precision);
int mlp_tc_hold_weights(mcl_map* m, int n_launches, unsigned long long wait_ns);
cudaError_t mlp_tc_ray_bias(mcl_map* m, const float* gd, int n_rays, const int* n_rays_dev,
                            cudaStream_t s);
// Fused ray epilogue of a tensor-core MLP pass (tiles hold whole rays).
//   mode 1 (first pass of the hierarchical sampler): Eq. 1 weights of each
//          ray's S samples -> nf_out inverse-CDF samples into z_out [rays,
//          nf_out]; out is written as usual;
//   mode 2 (last pass): merge with the first pass (z_first, out_first
//          [rays, S1]; S1 = 0: none), Eq. 1 composite, Eq. 5 / F, and with
//          obs (per-ray observed colour) E and e_ray = E F; optional per-ray
//          rgb / E / F / z_trans / z_opaque; out is not written.
struct FuseArgs {
    int mode;
    int nf_out;
    float* z_out;
    const float* z_first;
    const float4* out_first;
    int S1;
    float alpha, tau;
    int use_rej;
    const float4* obs;
    float* e_ray;
    float* rgb_out;
    float* E_out;
    float* F_out;
    float* zt_out;
    float* zo_out;
};
// Whether a pass of S samples per ray (and S1 first-pass samples, mode 2)
// can run with the fused epilogue.
bool mlp_tc_can_fuse(int mode, int S, int S1);
// rows_dev (optional): device-side row count (rows = n_rays * S is the bound).
// fuse (optional): fused ray epilogue of the pass.
cudaError_t mlp_tc(mcl_map* m, int precision, const Ray* rays, const float* gd, const float* z,
                   int S, int n_rays, const int* rows_dev, float4* out, cudaStream_t s,
                   const FuseArgs* fuse = nullptr);

// resample.cu
// status may be NULL (degenerate weights then show only as idx = -1)
cudaError_t launch_resample(const double* w, int n_in, int n_out, double u0, int32_t* idx,
                            unsigned long long* cdf, Status* status, cudaStream_t s);
cudaError_t launch_predict(const float* in, int n_in, const int32_t* idx, int n_out,
                           const float* odom, float sigma_t, float sigma_yaw, uint64_t seed,
                           uint64_t counter, float* out, cudaStream_t s);
cudaError_t launch_downscale(const float* img, int W, int H, int f, float* out, cudaStream_t s);
cudaError_t launch_position_spread(const float* poses, int N, double* out, cudaStream_t s);

// proposal.cu
int proposal_alloc(mcl_map* m);
// proposal_tc.cu
cudaError_t prop_tc_pack(mcl_map* m, cudaStream_t s);
cudaError_t prop_tc_prepare();
cudaError_t launch_prop_infer_tc(mcl_map* m, const Ray* rays, const float* z, int n_p, int n_rays,
                                 const int* n_rays_dev, float4* out, int n_sm, cudaStream_t s);
cudaError_t launch_prop_infer(mcl_map* m, int precision, const Ray* rays, const float* z, int n_p, int n_rays,
                              const int* n_rays_dev, float4* out, cudaStream_t s);
cudaError_t launch_histogram(const Ray* rays, int n_rays, const float* zc, const float4* oc, int nc,
                             const float* zf, const float4* of, int nf, int nb, float near_z,
                             float far_z, float* hist, cudaStream_t s);
int proposal_loss_grad(mcl_map* m, const float* O, const float* D, int n, int nb, float near_z,
                       float far_z, const float* hist, double* d_loss, float* d_grad,
                       cudaStream_t s);
int proposal_train(mcl_map* m, const float* d_poses, int n_poses, const int32_t* d_pixels, int B,
                   const mcl_intrinsics& K, int level, const mcl_opts& o, const mcl_train_cfg& cfg,
                   float* d_loss_log, cudaStream_t s,
                   int (*render_chunk)(mcl_map*, const float*, int, const mcl_intrinsics*, int,
                                       const int32_t*, int, const mcl_opts*, cudaStream_t));

// loop.cu
cudaError_t launch_draw_pixels(int W, int H, int B, uint64_t seed, uint64_t ctr, int32_t* out,
                               cudaStream_t s);
int enqueue_localize(mcl_map* m, int nq, float* P_user, int stride, const mcl_intrinsics& K,
                     const mcl_schedule& sch, const mcl_opts& o, mcl_iter_record* d_log,
                     int* d_final_n, cudaStream_t s);

}  // namespace mcl
