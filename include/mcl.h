/*
 * mcl.h -- C ABI of the GB300 (sm_103a) library for the particle-weight update
 * of Fast Loc-NeRF Monte Carlo localisation (Kong, Lee, Lee, Kim, "Fast Global
 * Localization on Neural Radiance Field", arXiv 2406.12202).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Pointers named d_* are DEVICE memory owned by the caller (for example
 *   torch CUDA tensors); the library never frees them.  Host pointers are read
 *   before the call returns and may be reused immediately.
 * - Calls are asynchronous on the CUDA stream passed as `stream` (a
 *   cudaStream_t; NULL = the legacy default stream).  Results are valid once
 *   that stream has reached the point of the call.
 * - Return value: MCL_OK (0) or a negative MCL_ERR_* code; mcl_last_error()
 *   returns a message for the calling thread.  No C++ exception crosses the
 *   boundary.  Argument checks happen on the host before anything is
 *   launched; problems only the device can see (non-finite inputs, degenerate
 *   weights) are recorded in a per-map status word (mcl_read_status).
 * - The library allocates device memory only in mcl_init_map (weights and a
 *   workspace sized by mcl_map_config) and frees it in mcl_destroy_map; the
 *   two proposal-training entry points also allocate (and free before they
 *   return) their own training scratch.
 * - Every floating-point array is row-major and tightly packed.
 * - A map may be used by one stream at a time (the workspace is shared).
 */
#ifndef MCL_H
#define MCL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MCL_OK 0
#define MCL_ERR_ARG (-1)        /* bad argument: shape, level, null, range   */
#define MCL_ERR_CUDA (-2)       /* a CUDA runtime call failed                */
#define MCL_ERR_NONFINITE (-3)  /* (status word) non-finite particle loss    */
#define MCL_ERR_TIMEOUT (-4)    /* (status word) bounded device wait expired */
#define MCL_ERR_UNSUPPORTED (-5)/* configuration this build does not serve  */
#define MCL_ERR_DEGENERATE (-6) /* (status word) resampling weights all zero */

typedef struct mcl_map mcl_map;

/* NeRF MLP of the "basic NeRF model" (Sec. IV-A): positional encoding with
 * n_freq_xyz / n_freq_dir frequencies, a trunk of trunk_depth ReLU layers of
 * trunk_width units with gamma(x) concatenated after layer skip_layer, a
 * density head, a linear feature layer, and an RGB head of rgb_width ReLU
 * units fed with [feature, gamma(d)].  This build serves (10, 4, 8, 256, 5,
 * 128) and rejects other shapes with MCL_ERR_UNSUPPORTED. */
typedef struct {
    int n_freq_xyz, n_freq_dir, trunk_depth, trunk_width, skip_layer, rgb_width;
} mcl_arch;

/* Workspace bounds fixed at map creation. */
typedef struct {
    int max_rays;      /* largest N * B of any call (summed over queries)     */
    int max_samples;   /* largest n_coarse + n_fine                           */
    int max_particles; /* largest particle count (queries x stride for       */
                       /* mcl_localize)                                       */
    int max_queries;   /* largest query count of mcl_localize (<= 64)         */
} mcl_map_config;

/* Pinhole intrinsics K at FULL resolution (Eq. 4, "shared intrinsic camera
 * parameter K").  Level l uses R K with R = 2^(l - 2): focal length and
 * principal point divided by 4, 2, 1 for levels 0, 1, 2 (Alg. 1, "R_t K"). */
typedef struct {
    float fx, fy, cx, cy;
    int width, height;
} mcl_intrinsics;

enum { MCL_PREC_FP32 = 0, MCL_PREC_BF16 = 1, MCL_PREC_FP8 = 2 };

/* Options of one weight update. */
typedef struct {
    int n_coarse;       /* stratified samples per ray, 2..256                */
    int n_fine;         /* importance samples per ray, 0..256 (0: none)      */
    int precision;      /* MCL_PREC_*: arithmetic of the NeRF MLP            */
    int use_rejection;  /* 1: Eq. 6 (F from Eq. 5); 0: Eq. 4 (F = 1)         */
    int jitter;         /* 0: stratum midpoints; 1: SplitMix64 jitter drawn
                           from stream (seed, counter), value ray*n_coarse+k */
    float near_z, far_z;/* sample range along d (points x = o + z d)         */
    float alpha;        /* Eq. 5 threshold, 0 < alpha < 0.5                   */
    float tau;          /* lower bound of F (Eq. 6), > 0                      */
    double rho_reject;  /* mask_i = (w_i >= rho_reject / N)                   */
    double s_min;       /* floor of S_i before the logarithm (> 0)            */
    uint64_t seed, counter;
    int use_proposal;   /* 1: sample with the learned proposal (the project's
                           extension; see mcl_proposal_train): n_proposal
                           stratified proposal samples -> n_guided inverse-CDF
                           samples for the NeRF MLP -> n_fine importance
                           samples from those; n_coarse is then unused      */
    int n_proposal;     /* 2..256                                            */
    int n_guided;       /* 2..256                                            */
} mcl_opts;

/* Optional per-ray / per-particle outputs of mcl_update (any may be NULL). */
typedef struct {
    float* rgb;       /* [N*B, 3] rendered colour C(r(p_j, x_i))             */
    float* E;         /* [N*B]  squared RGB distance to the observed pixel   */
    float* F;         /* [N*B]  max(z_opaque - z_trans, tau), or 1           */
    float* z_trans;   /* [N*B]  Eq. 5                                        */
    float* z_opaque;  /* [N*B]  Eq. 5                                        */
    float* S;         /* [N]    sum_j E_ij F_ij                              */
} mcl_debug;

/* Upload the NeRF map M (Sec. III-A, "NeRF as a map"; the map is fixed for a
 * localisation run).  host_weights: n_floats FP32 values, per layer W[out][in]
 * then b[out], layers in the order trunk1..trunk_depth, sigma, feature,
 * rgb_hidden, rgb_out; trunk layer skip_layer+1 reads [h, gamma(x)] and
 * rgb_hidden reads [feature, gamma(d)].  The blob is copied (FP32, BF16 and
 * FP8 device forms are prepared here), so the caller keeps its buffer.
 * Allocates the workspace for cfg.  Synchronous.  *out_map is NULL on error. */
int mcl_init_map(const float* host_weights, size_t n_floats,
                 const mcl_arch* arch, const mcl_map_config* cfg,
                 mcl_map** out_map);

/* 1 if mcl_update / mcl_render on this map can run the NeRF MLP in
 * `precision` (MCL_PREC_*) on the current device, else 0.  FP32 is always
 * available; BF16 needs an sm_103 device. */
int mcl_map_supports(const mcl_map* map, int precision);

/* Free the map and its workspace (synchronises the device first). */
void mcl_destroy_map(mcl_map* map);

/* One particle-weight update (Alg. 1, loop over particles, with Eq. 6):
 *   for particle i (pose d_particles[i], row-major 3x4 camera-to-world [R|t],
 *   camera looking along -z with +y up) and query pixel p_j = d_pixels[j]
 *   (int32 (u, v) in the level image; the same B pixels for every particle):
 *     C_ij = volume render (Eq. 1) of the pixel-centre ray with R K, using
 *            n_coarse stratified and n_fine importance samples;
 *     E_ij = sum_c (I^R(p_j)_c - C_ij,c)^2, I^R = box downscale of d_image;
 *     F_ij = max(z_opaque - z_trans, tau) (Eq. 5) if use_rejection else 1;
 *   S_i = sum_j E_ij F_ij,  d_logw[i] = 4 (log B - log max(S_i, s_min)),
 *   d_w[i] = exp(logw_i - logsumexp(logw)) in FP64 (sums to 1),
 *   d_mask[i] = (d_w[i] >= rho_reject / N).
 * d_particles: [N,12] f32.  d_image: [H,W,3] f32 full resolution.  level:
 * 0, 1, 2 (R = 1/4, 1/2, 1; W and H divisible by the factor).  N*B <=
 * max_rays, N <= max_particles.  A particle whose S_i is not finite gets
 * logw = -inf, w = 0, mask = 0 and is counted in the status word. */
int mcl_update(mcl_map* map, const float* d_particles, int N,
               const float* d_image, const mcl_intrinsics* K, int level,
               const int32_t* d_pixels, int B, const mcl_opts* opts,
               float* d_logw, double* d_w, uint8_t* d_mask,
               const mcl_debug* dbg, void* stream);

/* Evaluate the map F(x, d) -> (c, sigma) of Sec. III-A at n points with the
 * NeRF MLP in `precision` (the arithmetic mcl_update uses):
 * d_out[i] = (sigma_raw_i, r_i, g_i, b_i), sigma_raw before the ReLU that
 * compositing applies, rgb after the sigmoid.  d_x [n,3] f32 points, d_dir
 * [n,3] f32 view directions (normalised here), d_out [n,4] f32, 16-byte
 * aligned.  1 <= n <= max_rays.  Uses the map workspace. */
int mcl_query(mcl_map* map, const float* d_x, const float* d_dir, int n,
              int precision, float* d_out, void* stream);

/* Render the colours C(r(p_j, x_i)) (Eq. 1 with the same sampling as
 * mcl_update) for n_poses poses x B pixels into d_rgb [n_poses*B, 3]; d_F
 * [n_poses*B] (optional) receives F of Eq. 6.  Used to synthesise
 * observations. */
int mcl_render(mcl_map* map, const float* d_poses, int n_poses,
               const mcl_intrinsics* K, int level, const int32_t* d_pixels,
               int B, const mcl_opts* opts, float* d_rgb, float* d_F,
               void* stream);

/* Systematic resampling (Alg. 1, "draw i with probability proportional to
 * w_i") on an exact integer CDF: with e the binary exponent of max w
 * (max w = m 2^e, m in [1/2, 1)) and s = 50 - e - ceil(log2 N_in),
 * q_i = floor(w_i 2^s), C_i = q_0 + .. + q_i, T = C_{N_in - 1},
 * U = floor(u0 2^53); d_idx[k] = smallest i with
 * C_i N_out 2^53 > (k 2^53 + U) T.  The same weights give the same indices
 * on every machine.  d_w: [N_in] f64 >= 0; d_idx: [N_out] int32.  N_in <=
 * max_particles, 1 <= N_out <= 65536, 0 <= u0 < 1.  Uses the map workspace.
 * Negative, non-finite or all-zero weights: every d_idx is -1 and the status
 * word records MCL_ERR_DEGENERATE. */
int mcl_resample(mcl_map* map, const double* d_w, int N_in, int N_out,
                 double u0, int32_t* d_idx, void* stream);

/* Largest N_in that mcl_resample_noalloc accepts. */
#define MCL_RESAMPLE_NOALLOC_MAX_IN 65536

/* Systematic resampling exactly as mcl_resample (same integer rule, same
 * indices for the same weights and u0), for callers that cannot allocate
 * device memory: a control loop that forbids allocation once it runs, code
 * executing while a stream is captured into a CUDA graph, or a filter that
 * has no map.  The paper has no counterpart; this entry point only changes
 * where the scratch lives.  It needs no map and allocates nothing: its
 * scratch (the integer CDF of up to MCL_RESAMPLE_NOALLOC_MAX_IN weights,
 * 512 KB) is a fixed array in the library image, present on every device
 * that loads the library until the process exits.  The first call on a
 * device looks up that array's device address (with that device current)
 * and caches it; make that first call before any stream capture, and do not
 * call this entry point on a device after cudaDeviceReset() (the cached
 * address would be stale).  Every call shares the array: calls that overlap
 * on the GPU (different streams, or different host threads on one device)
 * race and must be serialised by the caller.  d_w and d_idx must be device
 * memory of the current device (MCL_ERR_ARG otherwise).  N_in >
 * MCL_RESAMPLE_NOALLOC_MAX_IN is rejected with MCL_ERR_ARG.  Negative,
 * non-finite or all-zero weights give d_idx[k] = -1 for every k (there is
 * no status word).  d_w: [N_in] f64, d_idx: [N_out] int32, 1 <= N_out <=
 * 65536, 0 <= u0 < 1. */
int mcl_resample_noalloc(const double* d_w, int N_in, int N_out, double u0,
                         int32_t* d_idx, void* stream);

/* Prediction step (Sec. III-A): d_out[k] = d_in[idx[k]] * Exp(delta_k) with
 * O_t = I, delta_k = (rho, (0, yaw, 0)) in se(3), rho ~ N(0, sigma_t^2 I3),
 * yaw ~ N(0, sigma_yaw^2) in the body frame.  The normals are Box-Muller
 * pairs of SplitMix64 stream (seed, counter): normal m uses values 2m and
 * 2m+1, particle k takes normals 4k .. 4k+3.  d_in [N_in,12], d_out
 * [N_out,12] f32 (computed in FP64).  d_idx [N_out] may be NULL (identity,
 * N_out <= N_in); an index outside [0, N_in) yields a NaN pose. */
int mcl_predict(const float* d_in, int N_in, const int32_t* d_idx, int N_out,
                float sigma_t, float sigma_yaw, uint64_t seed,
                uint64_t counter, float* d_out, void* stream);

/* Prediction with odometry (Sec. III-A motion model x_t = x_{t-1} O_t
 * Exp(delta)): as mcl_predict, with d_odom the device 3x4 row-major relative
 * motion O_t between the two observations (NULL: O_t = I, mcl_predict). */
int mcl_predict_odom(const float* d_in, int N_in, const int32_t* d_idx, int N_out,
                     const float* d_odom, float sigma_t, float sigma_yaw, uint64_t seed,
                     uint64_t counter, float* d_out, void* stream);

/* Box downscale of Alg. 1 ("downscale(I_t, R_t)"): d_out[v][u] = mean of the
 * factor x factor block of d_image.  d_image [H,W,3] f32, d_out
 * [H/factor, W/factor, 3]. */
int mcl_downscale(const float* d_image, int W, int H, int factor,
                  float* d_out, void* stream);

/* Spread of the particle positions used by the refinement test of the
 * coarse-to-fine schedule (Sec. III-C, "Var({x_t}) < delta_refine"):
 * d_out[0..2] = mean position, d_out[3] = trace of the population covariance
 * (FP64).  d_poses [N,12] f32. */
int mcl_position_spread(const float* d_poses, int N, double* d_out,
                        void* stream);

/* Read and clear the map's status word (synchronises `stream`): MCL_OK or the
 * first MCL_ERR_* recorded by the device since the last read; *n_nonfinite
 * (optional) receives the number of particles masked for non-finite loss. */
int mcl_read_status(mcl_map* map, int* n_nonfinite, void* stream);

/* Draw the query pixel set of one update (Eq. 4 / Eq. 6 index p_j without a
 * particle index: one set for every particle): B distinct pixels of a W x H
 * level image, uniformly without replacement, by Floyd's sampling algorithm
 * on SplitMix64 stream (seed, counter): for j = n-B .. n-1 (n = W H), t =
 * floor(r (j+1) / 2^64) with r = value j-(n-B) of the stream; take t unless
 * already taken, else j; pixel index -> (u, v) = (index % W, index / W).
 * d_out: [B,2] int32.  1 <= B <= min(1024, W H). */
int mcl_draw_pixels(int W, int H, int B, uint64_t seed, uint64_t counter,
                    int32_t* d_out, void* stream);

/* Coarse-to-fine schedule of Sec. III-C for mcl_localize.  Stage s renders
 * level level[s] (R = 2^(level - 2)) with n_pixels[s] query pixels and at
 * most n_cap[s] particles.  After each iteration the particle count becomes
 * clamp(survivors, n_min, n_cap[stage]) (survivors = particles whose
 * normalised weight is at least rho_reject / N), and the run moves to the
 * next stage when the weighted variance (trace) of the positions falls below
 * refine[stage] or after stage_iter_cap[stage] iterations in the stage. */
#define MCL_MAX_STAGES 3
typedef struct {
    int n_stages;                         /* 1 .. 3                          */
    int level[MCL_MAX_STAGES];            /* image level of each stage       */
    int n_pixels[MCL_MAX_STAGES];         /* B of each stage, <= 256         */
    int n_cap[MCL_MAX_STAGES];            /* particle cap of each stage      */
    int n_min;                            /* lower clamp of the survivors    */
    int stage_iter_cap[MCL_MAX_STAGES];   /* forced refinement after this    */
    double refine[MCL_MAX_STAGES];        /* spread threshold per stage      */
    int iterations;                       /* MCL iterations of the run       */
    float sigma_t, sigma_yaw;             /* motion noise (mcl_predict)      */
} mcl_schedule;

/* One record per query and iteration of mcl_localize (weights of that
 * iteration, before resampling). */
typedef struct {
    int stage, level, n_particles, n_pixels, n_survivors;
    int status;            /* particles with a non-finite loss this iteration */
    double spread;         /* weighted trace of the position covariance       */
    double est[4];         /* weighted mean position (x, y, z), circular yaw  */
    uint64_t t_start_ns;   /* GPU global timer (ns) when the iteration began:
                              differences of consecutive records are the
                              per-update latencies of the run               */
} mcl_iter_record;

/* Run Monte Carlo localisation (Alg. 1 iterated, Sec. III-C schedule) on the
 * device for n_queries independent queries on one map.  Iteration t of query
 * q: draw the pixel set (mcl_draw_pixels, stream (seed, q 2^32 + 4t)), weight
 * the particles (as mcl_update), record, apply the schedule, resample
 * (mcl_resample with u0 = value 0 of stream (seed, q 2^32 + 4t + 1)) and
 * predict (mcl_predict with stream (seed, q 2^32 + 4t + 2)); jitter, when
 * enabled, uses stream (seed, q 2^32 + 4t + 3).  d_particles: [n_queries,
 * stride, 12] f32, query q's h_n0[q] initial particles at row q*stride; on
 * return its final particles (count in d_final_n[q]).  h_images: host array
 * of n_queries device pointers to [H,W,3] observations, all with intrinsics
 * K.  d_log: [n_queries, iterations].  All sizes that change during the run
 * stay on the device: with use_graph != 0 the run is captured into a CUDA
 * graph on the map's own stream (ordered after earlier work on `stream` and
 * before later work on it) and kept; later calls with the same shapes and
 * pointers relaunch it.  opts->precision selects the NeRF MLP's form (the
 * plain FP32 form or a tensor-core form); opts->use_proposal selects the
 * learned sampler.  The map must hold the largest iteration: n_queries * max(max_q
 * h_n0[q] * n_pixels[0], max_s min(n_cap[s], stride) * n_pixels[s]) <=
 * max_rays, and n_queries * stride <= max_particles. */
int mcl_localize(mcl_map* map, int n_queries, float* d_particles, int stride,
                 const int* h_n0, const float* const* h_images,
                 const mcl_intrinsics* K, const mcl_schedule* sch,
                 const mcl_opts* opts, mcl_iter_record* d_log, int* d_final_n,
                 int use_graph, void* stream);

/* ---- learned proposal sampler (a project extension; the paper has none) --
 * Network: gamma(x) with 6 frequencies (39 inputs) -> four ReLU layers of 64
 * units -> raw density s (linear head); density max(s, 0) composited over
 * n_proposal stratified midpoints as Eq. 1.  Weight blob (15105 floats):
 * P1 W[64][39] b[64], P2..P4 W[64][64] b[64], head w[64] b[1]. */
#define MCL_PROPOSAL_N_WEIGHTS 15105

typedef struct {
    int epochs;         /* passes over the training rays                     */
    int batch_rays;     /* rays per Adam step                                */
    int n_bins;         /* proposal samples = target histogram bins (<= 256) */
    float lr, beta1, beta2, eps;   /* Adam                                   */
    uint64_t seed;      /* shuffling of the rays                             */
    float lr_end;       /* learning rate of the last step; the rate decays
                           geometrically from lr (lr_end <= 0: constant lr)   */
} mcl_train_cfg;

/* Copy proposal weights in / out (host buffers of MCL_PROPOSAL_N_WEIGHTS). */
int mcl_proposal_set(mcl_map* map, const float* host_weights, size_t n);
int mcl_proposal_get(mcl_map* map, float* host_out, size_t n);

/* Raw proposal density at n points d_x [n,3] into d_sigma [n] (FP32 form:
 * the FP32 kernel; BF16 / FP8: the tensor-core kernel used by those forms,
 * BF16 operands).  1 <= n <= max_rays; uses the map workspace. */
int mcl_proposal_query(mcl_map* map, const float* d_x, int n, int precision, float* d_sigma,
                       void* stream);

/* Targets of the distillation: for n_poses poses x B pixels, render with the
 * full sampler of `opts` (n_coarse + n_fine, use_proposal ignored) and
 * re-bin the final weights onto n_bins equal intervals of [near_z, far_z]
 * (interval floor((z - near)/(far - near) n_bins), clamped), normalised
 * (uniform when a ray carries no weight).  d_hist: [n_poses*B, n_bins]. */
int mcl_render_histogram(mcl_map* map, const float* d_poses, int n_poses,
                         const mcl_intrinsics* K, int level,
                         const int32_t* d_pixels, int B, const mcl_opts* opts,
                         int n_bins, float* d_hist, void* stream);

/* Mean cross-entropy -sum_b h_b log(w_b / sum_k w_k + 1e-8) of the proposal
 * weights of n rays (origins d_o, directions d_d [n,3]; n_bins stratified
 * midpoints of [near_z, far_z]) against d_hist [n, n_bins] into *d_loss
 * (device double), and its gradient with respect to the proposal weights
 * into d_grad [MCL_PROPOSAL_N_WEIGHTS] (FP32).  Synchronous; allocates and
 * frees its scratch. */
int mcl_proposal_loss_grad(mcl_map* map, const float* d_o, const float* d_d,
                           int n, int n_bins, float near_z, float far_z,
                           const float* d_hist, double* d_loss, float* d_grad,
                           void* stream);

/* Distil the proposal from the full sampler: targets of n_poses x B rays
 * (mcl_render_histogram with sampler_opts), then cfg->epochs epochs of Adam
 * on shuffled batches of the mean cross-entropy, starting from the current
 * proposal weights (set them first).  d_loss_log (optional, [epochs])
 * receives the mean loss of every epoch.  Gradients are reduced in a fixed
 * order, so the same inputs give the same weights.  Synchronous; allocates
 * and frees its training scratch (targets, one batch of activations). */
int mcl_proposal_train(mcl_map* map, const float* d_poses, int n_poses,
                       const int32_t* d_pixels, int B, const mcl_intrinsics* K,
                       int level, const mcl_opts* sampler_opts,
                       const mcl_train_cfg* cfg, float* d_loss_log,
                       void* stream);

/* ---- fitting the map to samples of a field (a project extension) ---------
 * The paper takes the NeRF map as given (trained on images, Eq. 2, out of
 * scope here).  These entry points fit the map's FP32 weights to point
 * samples of a field instead -- points d_x [n,3], view directions d_dir
 * [n,3] (normalised here) and targets d_target [n,4] = (density, r, g, b) --
 * by minimising the mean of
 *   sigma_weight (sigma_raw(x) - density)^2 + |rgb(x, d) - (r, g, b)|^2
 * with the library's own FP32 forward (the plain form's kernels, every
 * layer's output kept), backward (SGEMMs on transposed weights with the
 * ReLU masks) and Adam.  Weight gradients are summed over each batch in a
 * fixed order, so the same inputs give the same weights. */
typedef struct {
    int steps;            /* Adam steps                                      */
    int batch;            /* points per step (the last epoch's tail is cut) */
    float lr, beta1, beta2, eps;
    float lr_end;         /* geometric decay from lr to lr_end (<= 0: none) */
    float sigma_weight;   /* weight of the density term                     */
    uint64_t seed;        /* shuffling of the points                        */
} mcl_fit_cfg;

/* Fit the map (starting from its current weights) with cfg->steps Adam
 * steps on shuffled batches; d_loss_log (optional, device [steps]) receives
 * each step's batch loss.  The tensor-core forms are rebuilt from the fitted
 * weights (their calibration and kernel-variant choices start afresh, and a
 * captured mcl_localize graph is dropped).  Synchronous; allocates and frees
 * its training scratch (about 8.5 KB per point of a batch).  1 <= batch,
 * 1 <= n, 1 <= steps. */
int mcl_fit_map(mcl_map* map, const float* d_x, const float* d_dir, const float* d_target, int n,
                const mcl_fit_cfg* cfg, float* d_loss_log, void* stream);

/* The fitting loss of n points (mean, into *d_loss, device double) and its
 * gradient with respect to the weights in the blob layout of mcl_init_map
 * (d_grad: device, as many floats as the blob).  Synchronous; allocates its
 * scratch. */
int mcl_map_loss_grad(mcl_map* map, const float* d_x, const float* d_dir, const float* d_target,
                      int n, float sigma_weight, double* d_loss, float* d_grad, void* stream);

/* Copy the map's FP32 weights, in the blob layout of mcl_init_map, into
 * host_out (n floats, the blob size).  Synchronous. */
int mcl_get_map_weights(mcl_map* map, float* host_out, size_t n);

/* Kernel variants of the tensor-core MLP (index: precision, epilogue warps
 * per 128-row tile, tile schedule):
 *   0 BF16 4 lockstep   1 BF16 8 lockstep   2 FP8 4 lockstep
 *   3 FP8 8 lockstep    4 FP8 4 staggered   5 FP8 8 staggered
 *   6 BF16 4 split      7 BF16 4 pipelined (one tile per CTA)
 *   8 BF16 4 lockstep, CTA pair   9 FP8 4 lockstep, CTA pair
 *  10 FP8 4 staggered, CTA pair   11 BF16 4 staggered   12 BF16 8 staggered
 *  13 BF16 4 staggered, CTA pair
 * Lockstep: each streamed weight block serves both tiles of a pair at once;
 * staggered: the second tile runs each part of a layer (the blocks the
 * weight ring holds: a whole FP8 layer, four BF16 blocks; with CTA pairs a
 * whole BF16 layer but the skip layer's, run as 2 + 8 blocks) after the first on
 * the same resident blocks, so one tile's epilogue overlaps the other's
 * MMAs; split: lockstep, each layer as two
 * 128-column halves whose epilogues overlap the MMAs of the other half and
 * of the next layer; pipelined: one tile per CTA with double-buffered
 * accumulators, the next layer's MMAs consuming the activations 64 columns
 * at a time as the epilogue writes them; CTA pair: clusters of two CTAs on
 * the two SMs of a TPC issue 256-row MMAs (tcgen05 cta_group::2), each CTA
 * streaming half of every weight block.  All variants of a precision give
 * bit-identical results.  Untuned defaults: 12 (BF16) and 5 (FP8). */
#define MCL_MLP_VARIANTS 14

/* Autotuner: time every variant of `precision` (MCL_PREC_BF16 or _FP8) on
 * `rows` synthetic samples (256 <= rows <= max_rays * min(64, max_samples);
 * uses the map workspace), keep the fastest for all later MLP launches of
 * the map, return its index in *chosen and the mean ms of each variant in
 * ms[MCL_MLP_VARIANTS] (-1 for variants of other precisions); either may be
 * NULL.  Synchronous; must not be called during stream capture.
 * mcl_localize runs it once per precision before its first graph capture. */
int mcl_autotune(mcl_map* map, int precision, long long rows, int* chosen, float* ms,
                 void* stream);

/* Failure detection test hook (no counterpart in the paper).  The next
 * n_launches launches of the tensor-core NeRF MLP on this map (any entry
 * point that runs it) use the untuned single-CTA kernel of their precision
 * with its weight stream held back and every bounded wait of the kernel
 * limited to wait_ms: the wait for the first weight block runs out, the
 * kernel's warps stop, release their tensor memory and exit, and the map's
 * status word records MCL_ERR_TIMEOUT (mcl_read_status).  The launching call
 * itself returns MCL_OK (the device sees the failure after the call has
 * returned); outputs of the stalled launches are undefined.  Later launches
 * run normally.  No GPU fault, trap or endless wait is involved.
 * 0 <= n_launches; 0.01 <= wait_ms <= 2000. */
int mcl_inject_weight_stall(mcl_map* map, int n_launches, double wait_ms);

/* Fused ray epilogues of the tensor-core forms (off by default): when the
 * pass shapes allow it (n_coarse -- or n_guided with the proposal -- and
 * n_fine divide 128, and a ray's merged samples fit the kernel's staging
 * buffer), the NeRF MLP kernel's epilogue draws the importance samples of
 * the first pass and, in the last pass, merges the samples, composites them
 * (Eq. 1), applies Eq. 5 / F and the photometric E (Eq. 6), so the fine
 * pass's per-sample outputs never leave the chip.  The arithmetic is that of
 * the separate kernels in another order (warp-shuffle scans instead of one
 * thread walking a ray), so results agree to FP32 rounding.  enable = 1
 * fuses, enable = 0 runs the separate kernels (mcl_update, mcl_render and
 * mcl_localize on this map).  The separate kernels are the default: on
 * GB300 the fused form moves less data but takes 4-17 % longer per update,
 * its ray tails running in the epilogue warps that the tensor pipe waits
 * for. */
int mcl_set_fused_epilogue(mcl_map* map, int enable);

/* Pin the MLP kernel variant of a precision (see MCL_MLP_VARIANTS). */
int mcl_set_mlp_variant(mcl_map* map, int precision, int variant);

/* Diagnostic of the tensor-core issue path the MLP kernel's schedule is
 * built around (no counterpart in the paper): one CTA per SM issues
 * n_groups groups of `group` back-to-back BF16 tcgen05 MMAs (128 x 256 x 16,
 * operands in shared memory in the MLP kernel's layouts, accumulators in
 * TMEM) from one thread, with a dependent chain of `gap` integer
 * multiply-adds in that thread after each group.  *clk_per_group receives
 * the median over SMs of SM clock cycles per group, *gap_clk (optional) the
 * cycles of one chain alone.  gap = 0 gives the per-SM MMA rate; gap > 0
 * shows how much work a group leaves queued while the thread is busy.
 * 1 <= group <= 64, 0 <= gap <= 4096, 1 <= n_groups <= 100000.
 * Synchronous, on the legacy default stream; sm_103 only
 * (MCL_ERR_UNSUPPORTED otherwise). */
int mcl_probe_mma_rate(int group, int gap, int n_groups, double* clk_per_group, double* gap_clk);

/* Phases timed when profiling is on (indices into the array of
 * mcl_profile_read). */
#define MCL_PHASE_RAYGEN 0     /* ray generation + stratified samples      */
#define MCL_PHASE_MLP_COARSE 1 /* NeRF MLP on the coarse samples           */
#define MCL_PHASE_SAMPLE 2     /* coarse composite + importance sampling   */
#define MCL_PHASE_MLP_FINE 3   /* NeRF MLP on the importance samples       */
#define MCL_PHASE_COMPOSITE 4  /* final composite, Eq. 5, photometric E    */
#define MCL_PHASE_WEIGHTS 5    /* Eq. 6 weights, FP64 normalisation        */
#define MCL_PHASE_RESAMPLE 6   /* systematic resampling                    */
#define MCL_N_PHASES 7

/* Turn per-phase GPU timing of mcl_update / mcl_render / mcl_resample on or
 * off for this map.  When on, CUDA events are recorded on the call's stream
 * around each phase (a few microseconds of overhead per phase). */
int mcl_profile_enable(mcl_map* map, int enable);

/* Synchronise on the recorded events and return the accumulated GPU time of
 * each phase in ms_out[MCL_N_PHASES] since the last reset; *n_launches
 * (optional) receives the number of kernels this library has launched in the
 * process so far (all maps and entry points).  reset != 0 clears the
 * accumulated times. */
int mcl_profile_read(mcl_map* map, double* ms_out, long long* n_launches, int reset);

/* Thread-local message of the last error, "" if none. */
const char* mcl_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* MCL_H */
