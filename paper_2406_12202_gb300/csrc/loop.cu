// loop.cu -- Monte Carlo localisation run on the device (Alg. 1 iterated with
// the coarse-to-fine schedule of Sec. III-C) for one or many independent
// queries on one map.
//
// Every size that changes during a run -- particles per query after
// rejection, pixels per query at the current stage, the level factor, the
// offsets of each query's rays in the flattened ray list -- lives in device
// memory and is decided by device kernels (k_plan, k_schedule_b).  The host
// enqueues a fixed sequence of launches per iteration whose grids cover the
// largest sizes, so the whole run can be captured into one CUDA graph and
// replayed with no host round trip; the persistent tensor-core MLP kernel
// reads its row count from device memory and balances all queries' rays over
// the SMs.
#include <string.h>

#include "stages.cuh"

namespace mcl {

constexpr int kLoopThreads = 1024;

// counter of SplitMix64 streams of query q at iteration t, purpose p
__host__ __device__ __forceinline__ uint64_t loop_ctr(int q, int t, int p) {
    return ((uint64_t)(uint32_t)q << 32) | ((uint64_t)(uint32_t)t << 2) | (uint64_t)p;
}

__device__ __forceinline__ int query_of_ray(const LoopPlan* pl, int nq, int r) {
    int q = 0;
    while (q + 1 < nq && pl->ray_off[q + 1] <= r) ++q;
    return q;
}

// Sizes of the coming iteration from each query's state.
__global__ void k_plan(LoopPlan* __restrict__ pl, const LoopQuery* __restrict__ qs, int nq,
                       mcl_schedule sch, int nc, int nf) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    pl->t_start = t;
    int off = 0;
    for (int q = 0; q < nq; ++q) {
        const int st = qs[q].stage;
        pl->N[q] = qs[q].N;
        pl->B[q] = sch.n_pixels[st];
        pl->factor[q] = 4 >> sch.level[st];
        pl->ray_off[q] = off;
        off += qs[q].N * sch.n_pixels[st];
    }
    pl->ray_off[nq] = off;
    pl->total_rays = off;
    pl->rows_c = off * nc;
    pl->rows_f = off * nf;
}

// Pixel set of each query (Floyd's algorithm on SplitMix64, as
// mcl_draw_pixels): one thread per query.
__global__ void k_pixels(const LoopPlan* __restrict__ pl, int nq, int W, int H, uint64_t seed,
                         int t, int32_t* __restrict__ pix) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nq) return;
    const int f = pl->factor[q];
    draw_pixel_set(W / f, H / f, pl->B[q], seed, loop_ctr(q, t, 0), pix + (size_t)q * kLoopMaxPixels * 2);
}

__global__ void k_raygen_b(const LoopPlan* __restrict__ pl, int nq, const float* __restrict__ P,
                           int stride, const int32_t* __restrict__ pix, float fx, float fy,
                           float cx, float cy, int nc, float near_z, float far_z, int jitter,
                           uint64_t seed, int t, int max_rays, Ray* __restrict__ rays,
                           float* __restrict__ gd, float* __restrict__ zc,
                           const float* const* __restrict__ imgs, int W, int H,
                           float4* __restrict__ obs) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= max_rays || r >= pl->total_rays) return;
    const int q = query_of_ray(pl, nq, r);
    const int B = pl->B[q], f = pl->factor[q];
    const int rl = r - pl->ray_off[q];
    const int i = rl / B, j = rl - (rl / B) * B;
    const int32_t* px = pix + (size_t)q * kLoopMaxPixels * 2;
    Ray ray;
    make_ray(P + 12 * ((size_t)q * stride + i), px[2 * j], px[2 * j + 1], fx / f, fy / f, cx / f,
             cy / f, ray, gd + (size_t)r * kGdPad);
    rays[r] = ray;
    coarse_samples(rl, nc, near_z, far_z, jitter, seed, loop_ctr(q, t, 3), zc + (size_t)r * nc);
    if (obs) obs[r] = observed_colour(imgs[q], W, H, f, px[2 * j], px[2 * j + 1]);
}

__global__ void k_final_b(const LoopPlan* __restrict__ pl, int nq, const float* const* __restrict__ imgs,
                          int W, const int32_t* __restrict__ pix, const Ray* __restrict__ rays,
                          const float* __restrict__ zc, const float4* __restrict__ oc, int nc,
                          const float* __restrict__ zf, const float4* __restrict__ of, int nf,
                          float alpha, float tau, int use_rej, int max_rays,
                          float* __restrict__ e_ray) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= max_rays || r >= pl->total_rays) return;
    const int q = query_of_ray(pl, nq, r);
    const int B = pl->B[q], f = pl->factor[q];
    const int j = (r - pl->ray_off[q]) % B;
    const int32_t* px = pix + (size_t)q * kLoopMaxPixels * 2;
    const float dn = rays[r].dnorm;
    const RayResult c = composite_ray(dn, zc + (size_t)r * nc, oc + (size_t)r * nc, nc,
                                      zf + (size_t)r * nf, of + (size_t)r * nf, nf, alpha, tau,
                                      use_rej);
    e_ray[r] = photometric_E(imgs[q], W, f, px[2 * j], px[2 * j + 1], c, dn) * c.F;
}

// Weights of each query (one block per query), survivors, weighted pose
// estimate and weighted position spread; one log record per query.
__global__ __launch_bounds__(kLoopThreads) void k_weights_b(
    const LoopPlan* __restrict__ pl, LoopQuery* __restrict__ qs, const float* __restrict__ P,
    int stride, const float* __restrict__ e_ray, double s_min, double rho,
    double* __restrict__ l64, double* __restrict__ w, uint8_t* __restrict__ mask,
    mcl_iter_record* __restrict__ log, int iterations, int t, mcl_schedule sch) {
    const int q = blockIdx.x;
    const int N = pl->N[q], B = pl->B[q];
    const size_t base = (size_t)q * stride;
    const int nbad = weights_block(e_ray + pl->ray_off[q], N, B, s_min, rho, nullptr, l64 + base,
                                   w + base, mask + base, nullptr);
    __shared__ double sh[32];
    double m[6];
    // survivors, weighted mean position, weighted yaw direction
    double acc_s = 0.0;
    double am[3] = {0.0, 0.0, 0.0}, ys = 0.0, yc = 0.0;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        const float* p = P + 12 * (base + i);
        const double wi = w[base + i];
        acc_s += mask[base + i] ? 1.0 : 0.0;
        if (wi > 0.0) {
            am[0] += wi * p[3]; am[1] += wi * p[7]; am[2] += wi * p[11];
            const double yaw = atan2((double)p[2], (double)p[0]);
            ys += wi * sin(yaw);
            yc += wi * cos(yaw);
        }
    }
    m[0] = block_sum_d(acc_s, sh);
    m[1] = block_sum_d(am[0], sh);
    m[2] = block_sum_d(am[1], sh);
    m[3] = block_sum_d(am[2], sh);
    m[4] = block_sum_d(ys, sh);
    m[5] = block_sum_d(yc, sh);
    double var = 0.0;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        const float* p = P + 12 * (base + i);
        const double wi = w[base + i];
        if (wi > 0.0) {
            const double d0 = p[3] - m[1], d1 = p[7] - m[2], d2 = p[11] - m[3];
            var += wi * (d0 * d0 + d1 * d1 + d2 * d2);
        }
    }
    var = block_sum_d(var, sh);
    if (threadIdx.x == 0) {
        qs[q].n_surv = (int)m[0];
        qs[q].wspread = var;
        if (nbad > 0) qs[q].nonfinite += nbad;
        mcl_iter_record rec;
        rec.stage = qs[q].stage;
        rec.level = sch.level[qs[q].stage];
        rec.n_particles = N;
        rec.n_pixels = B;
        rec.n_survivors = (int)m[0];
        rec.status = nbad;
        rec.spread = var;
        rec.est[0] = m[1]; rec.est[1] = m[2]; rec.est[2] = m[3];
        rec.est[3] = atan2(m[4], m[5]);
        rec.t_start_ns = pl->t_start;
        log[(size_t)q * iterations + t] = rec;
    }
}

// Stage transition (Sec. III-C: refine when the spread of the positions falls
// below the stage threshold, or after the stage's iteration cap) and the next
// particle count N = clamp(survivors, n_min, cap of the stage).
__global__ void k_schedule_b(LoopPlan* __restrict__ pl, LoopQuery* __restrict__ qs, int nq,
                             mcl_schedule sch, int stride) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nq) return;
    LoopQuery s = qs[q];
    if (s.stage < sch.n_stages - 1 &&
        (s.wspread < sch.refine[s.stage] || s.iter_at_stage + 1 >= sch.stage_iter_cap[s.stage])) {
        ++s.stage;
        s.iter_at_stage = 0;
    } else {
        ++s.iter_at_stage;
    }
    int n = s.n_surv;
    if (n < sch.n_min) n = sch.n_min;
    if (n > sch.n_cap[s.stage]) n = sch.n_cap[s.stage];
    if (n > stride) n = stride;
    s.N = n;
    qs[q] = s;
    pl->Nnext[q] = n;
}

__global__ __launch_bounds__(kLoopThreads) void k_resample_b(
    const LoopPlan* __restrict__ pl, int stride, const double* __restrict__ w,
    int32_t* __restrict__ idx, u64* __restrict__ cdf, uint64_t seed, int t) {
    const int q = blockIdx.x;
    const size_t base = (size_t)q * stride;
    const double u0 = cb_uniform(seed, loop_ctr(q, t, 1), 0);
    resample_block(w + base, pl->N[q], pl->Nnext[q], u0, idx + base, cdf + base);
}

__global__ void k_predict_b(const LoopPlan* __restrict__ pl, int nq, int stride,
                            const float* __restrict__ Pin, const int32_t* __restrict__ idx,
                            float sigma_t, float sigma_yaw, uint64_t seed, int t,
                            float* __restrict__ Pout) {
    const long g = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= (long)nq * stride) return;
    const int q = (int)(g / stride), k = (int)(g - (long)q * stride);
    if (k >= pl->Nnext[q]) return;
    const size_t base = (size_t)q * stride;
    const int src = idx[base + k];
    float* O = Pout + 12 * (base + k);
    if (src < 0 || src >= pl->N[q]) {
        for (int c = 0; c < 12; ++c) O[c] = __int_as_float(0x7fc00000);
        return;
    }
    double qn[4];
    motion_noise(seed, loop_ctr(q, t, 2), k, sigma_t, sigma_yaw, qn);
    predict_pose(Pin + 12 * (base + src), qn, O);
}

__global__ void k_loop_init(LoopQuery* __restrict__ qs, const int* __restrict__ n0, int nq) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nq) return;
    LoopQuery s;
    memset(&s, 0, sizeof(s));
    s.N = n0[q];
    qs[q] = s;
}

__global__ void k_loop_final(const LoopQuery* __restrict__ qs, int nq, int* __restrict__ n_out) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q < nq) n_out[q] = qs[q].N;
}

__global__ void k_draw_pixels(int W, int H, int B, uint64_t seed, uint64_t ctr,
                              int32_t* __restrict__ out) {
    if (blockIdx.x == 0 && threadIdx.x == 0) draw_pixel_set(W, H, B, seed, ctr, out);
}

cudaError_t launch_draw_pixels(int W, int H, int B, uint64_t seed, uint64_t ctr, int32_t* out,
                               cudaStream_t s) {
    note_launch();
    k_draw_pixels<<<1, 32, 0, s>>>(W, H, B, seed, ctr, out);
    return cudaGetLastError();
}

// One full run: n_iter iterations for nq queries (all launches on stream s).
int enqueue_localize(mcl_map* m, int nq, float* P_user, int stride, const mcl_intrinsics& K,
                     const mcl_schedule& sch, const mcl_opts& o, mcl_iter_record* d_log,
                     int* d_final_n, cudaStream_t s) {
    LoopWork& L = m->loop;
    int rc;
    const int max_rays_run = L.max_rays_run;
    const bool prop = o.use_proposal != 0;
    // sample sets: without the proposal, coarse (zc, out_c, nc) + fine (zf,
    // out_f, nf); with it, stratified proposal samples (zc, np) -> guided
    // (zf, out_c, ng) -> fine (zc, out_f, nf)
    const int np = prop ? o.n_proposal : o.n_coarse;
    const int nc = prop ? o.n_guided : o.n_coarse, nf = o.n_fine;
    float* const za = prop ? m->zf : m->zc;
    float* const zb = prop ? m->zc : m->zf;
    const int tb = 128;
    // the NeRF MLP of the precision, rows from the plan in device memory;
    // tensor-core forms with the fused ray epilogues where the shapes allow
    const bool fp32 = o.precision == MCL_PREC_FP32;
    const bool fused = !fp32 && m->fuse_epilogue &&
                       (nf > 0 ? mlp_tc_can_fuse(1, nc, 0) && mlp_tc_can_fuse(2, nf, nc)
                               : mlp_tc_can_fuse(2, nc, 0));
    FuseArgs fa1{}, fa2{};
    fa1.mode = 1;
    fa1.nf_out = nf;
    fa1.z_out = zb;
    fa2.mode = 2;
    fa2.z_first = za;
    fa2.out_first = m->out_c;
    fa2.S1 = nf > 0 ? nc : 0;
    fa2.alpha = o.alpha;
    fa2.tau = o.tau;
    fa2.use_rej = o.use_rejection;
    fa2.obs = m->obs;
    fa2.e_ray = m->e_ray;
    auto mlp = [&](const float* z, int S, const int* rows_dev, float4* dst,
                   const FuseArgs* fa) -> cudaError_t {
        if (fp32) return mlp_fp32(m, m->rays, m->gd, z, S, max_rays_run, dst, s, rows_dev);
        return mlp_tc(m, o.precision, m->rays, m->gd, z, S, max_rays_run, rows_dev, dst, s,
                      fused ? fa : nullptr);
    };
    float* Pc = P_user;
    float* Pn = L.P_next;
    note_launch();
    k_loop_init<<<1, 64, 0, s>>>(L.qs, L.n0, nq);
    for (int t = 0; t < sch.iterations; ++t) {
        note_launch(4);
        k_plan<<<1, 32, 0, s>>>(L.plan, L.qs, nq, sch, nc, nf);
        k_pixels<<<1, 64, 0, s>>>(L.plan, nq, K.width, K.height, o.seed, t, L.pix);
        k_raygen_b<<<(max_rays_run + tb - 1) / tb, tb, 0, s>>>(
            L.plan, nq, Pc, stride, L.pix, K.fx, K.fy, K.cx, K.cy, np, o.near_z, o.far_z,
            prop ? 0 : o.jitter, o.seed, t, max_rays_run, m->rays, m->gd, m->zc, L.imgs, K.width,
            K.height, fused ? m->obs : nullptr);
        if (!fp32 && (rc = cuda_check(mlp_tc_ray_bias(m, m->gd, max_rays_run, &L.plan->total_rays, s),
                                      "loop ray bias")))
            return rc;
        if (prop) {
            if ((rc = cuda_check(launch_prop_infer(m, o.precision, m->rays, m->zc, np, max_rays_run,
                                                   &L.plan->total_rays, m->out_f, s),
                                 "loop proposal")) ||
                (rc = cuda_check(launch_coarse_to_fine(m->rays, max_rays_run, &L.plan->total_rays,
                                                       m->zc, np, m->out_f, nc, m->zf, s),
                                 "loop proposal sampling")))
                return rc;
        }
        if ((rc = cuda_check(mlp(za, nc, &L.plan->rows_c, m->out_c, nf > 0 ? &fa1 : &fa2),
                             "loop mlp (coarse)")))
            return rc;
        if (nf > 0) {
            if (!fused &&
                (rc = cuda_check(launch_coarse_to_fine(m->rays, max_rays_run, &L.plan->total_rays,
                                                       za, nc, m->out_c, nf, zb, s),
                                 "loop importance sampling")))
                return rc;
            if ((rc = cuda_check(mlp(zb, nf, &L.plan->rows_f, m->out_f, &fa2), "loop mlp (fine)")))
                return rc;
        }
        if (!fused) {
            note_launch();
            k_final_b<<<(max_rays_run + tb - 1) / tb, tb, 0, s>>>(
                L.plan, nq, L.imgs, K.width, L.pix, m->rays, za, m->out_c, nc, zb, m->out_f, nf,
                o.alpha, o.tau, o.use_rejection, max_rays_run, m->e_ray);
        }
        note_launch(4);
        k_weights_b<<<nq, kLoopThreads, 0, s>>>(L.plan, L.qs, Pc, stride, m->e_ray, o.s_min,
                                                 o.rho_reject, m->logw64, L.w, L.mask, d_log,
                                                 sch.iterations, t, sch);
        k_schedule_b<<<1, 64, 0, s>>>(L.plan, L.qs, nq, sch, stride);
        k_resample_b<<<nq, kLoopThreads, 0, s>>>(L.plan, stride, L.w, L.idx, m->cdf, o.seed, t);
        k_predict_b<<<(unsigned)(((long)nq * stride + tb - 1) / tb), tb, 0, s>>>(
            L.plan, nq, stride, Pc, L.idx, sch.sigma_t, sch.sigma_yaw, o.seed, t, Pn);
        float* tmp = Pc;
        Pc = Pn;
        Pn = tmp;
    }
    if (Pc != P_user &&
        (rc = cuda_check(cudaMemcpyAsync(P_user, Pc, sizeof(float) * 12 * (size_t)nq * stride,
                                         cudaMemcpyDeviceToDevice, s),
                         "copy final particles")))
        return rc;
    note_launch();
    k_loop_final<<<1, 64, 0, s>>>(L.qs, nq, d_final_n);
    return cuda_check(cudaGetLastError(), "loop launch");
}

}  // namespace mcl
