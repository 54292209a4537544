// api.cu -- the extern "C" entry points of include/mcl.h: argument checks,
// map / workspace management, and the order of the stages of one update.
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>

#include <atomic>
#include <cmath>
#include <vector>

#include "internal.cuh"

namespace mcl {

static thread_local char g_err[512] = "";

int fail(int code, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return code;
}

void clear_error() { g_err[0] = 0; }

int cuda_check(cudaError_t e, const char* what) {
    if (e == cudaSuccess) return MCL_OK;
    return fail(MCL_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

static std::atomic<long long> g_launches{0};

void note_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

// Per-phase timing: an event pair recorded on the call's stream around a
// phase when the map's profiling flag is set.
static cudaEvent_t ev_get(mcl_map* m) {
    cudaEvent_t e = nullptr;
    if (!m->pool.empty()) {
        e = m->pool.back();
        m->pool.pop_back();
    } else {
        cudaEventCreate(&e);
    }
    return e;
}

struct PhaseScope {
    mcl_map* m;
    int phase;
    cudaStream_t s;
    cudaEvent_t a = nullptr;
    PhaseScope(mcl_map* m_, int ph, cudaStream_t s_) : m(m_), phase(ph), s(s_) {
        if (m && m->prof) {
            a = ev_get(m);
            cudaEventRecord(a, s);
        }
    }
    ~PhaseScope() {
        if (a) {
            cudaEvent_t b = ev_get(m);
            cudaEventRecord(b, s);
            m->marks.push_back({phase, a, b});
        }
    }
};

// Layer table of the fixed architecture: fan-in and fan-out in blob order.
static void layer_shapes(int* fin, int* fout) {
    for (int l = 0; l < kDepth; ++l) {
        fin[l] = (l == 0) ? kGx : (l == kSkip ? kWidth + kGx : kWidth);
        fout[l] = kWidth;
    }
    fin[8] = kWidth; fout[8] = 1;
    fin[9] = kWidth; fout[9] = kWidth;
    fin[10] = kWidth + kGd; fout[10] = kRgbW;
    fin[11] = kRgbW; fout[11] = 3;
}

void blob_layer_shapes(int* fin, int* fout) { layer_shapes(fin, fout); }

static size_t blob_size() {
    int fin[12], fout[12];
    layer_shapes(fin, fout);
    size_t n = 0;
    for (int l = 0; l < 12; ++l) n += (size_t)fin[l] * fout[l] + fout[l];
    return n;
}

static void free_map(mcl_map* m) {
    if (!m) return;
    mlp_tc_free(m);
    for (auto& mk : m->marks) {
        cudaEventDestroy(mk.a);
        cudaEventDestroy(mk.b);
    }
    for (auto e : m->pool) cudaEventDestroy(e);
    if (m->loop.exec) cudaGraphExecDestroy(m->loop.exec);
    if (m->loop.stream) cudaStreamDestroy(m->loop.stream);
    if (m->loop.ev_in) cudaEventDestroy(m->loop.ev_in);
    if (m->loop.ev_out) cudaEventDestroy(m->loop.ev_out);
    void* ptrs[] = {m->w32, m->rays, m->gd, m->zc, m->zf, m->out_c, m->out_f, m->obs, m->e_ray,
                    m->logw64, m->cdf, m->status, m->act0, m->act1, m->gxbuf,
                    m->loop.plan, m->loop.qs, m->loop.n0, (void*)m->loop.imgs, m->loop.pix,
                    m->loop.P_next, m->loop.w, m->loop.mask, m->loop.idx, m->prop_w,
                    m->prop_packed, m->prop_abort};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    delete m;
}

}  // namespace mcl

using namespace mcl;

extern "C" const char* mcl_last_error(void) { return g_err; }

extern "C" int mcl_init_map(const float* host_weights, size_t n_floats, const mcl_arch* arch,
                            const mcl_map_config* cfg, mcl_map** out_map) {
    g_err[0] = 0;
    if (!out_map) return fail(MCL_ERR_ARG, "mcl_init_map: out_map is NULL");
    *out_map = nullptr;
    if (!host_weights || !arch || !cfg) return fail(MCL_ERR_ARG, "mcl_init_map: NULL argument");
    if (arch->n_freq_xyz != kLxyz || arch->n_freq_dir != kLdir || arch->trunk_depth != kDepth ||
        arch->trunk_width != kWidth || arch->skip_layer != kSkip || arch->rgb_width != kRgbW)
        return fail(MCL_ERR_UNSUPPORTED,
                    "mcl_init_map: this build serves arch (10,4,8,256,5,128) only");
    if (n_floats != blob_size())
        return fail(MCL_ERR_ARG, "mcl_init_map: n_floats %zu, expected %zu", n_floats, blob_size());
    if (cfg->max_rays < 1 || cfg->max_samples < 2 || cfg->max_samples > kMaxSamples ||
        cfg->max_particles < 1 || cfg->max_queries < 1 || cfg->max_queries > kLoopMaxQueries)
        return fail(MCL_ERR_ARG,
                    "mcl_init_map: bad workspace config (rays %d samples %d particles %d queries %d)",
                    cfg->max_rays, cfg->max_samples, cfg->max_particles, cfg->max_queries);
    for (size_t i = 0; i < n_floats; ++i)
        if (!std::isfinite(host_weights[i]))
            return fail(MCL_ERR_ARG, "mcl_init_map: weight %zu is not finite", i);

    mcl_map* m = new mcl_map();
    m->cfg = *cfg;
    // ---- padded FP32 layers -------------------------------------------
    int fin[12], fout[12], kpad[12];
    layer_shapes(fin, fout);
    for (int l = 0; l < 12; ++l) kpad[l] = fin[l];
    kpad[0] = kGxPad;               // gamma(x) 63 -> 64
    kpad[kSkip] = kWidth + kGxPad;  // [h, gamma(x)] 319 -> 320
    kpad[10] = kWidth + kGdPad;     // [feature, gamma(d)] 283 -> 288
    std::vector<size_t> offW(12), offB(12);
    size_t tot = 0;
    for (int l = 0; l < 12; ++l) {
        offW[l] = tot; tot += (size_t)fout[l] * kpad[l];
        tot = (tot + 3) & ~(size_t)3;
        offB[l] = tot; tot += fout[l];
        tot = (tot + 3) & ~(size_t)3;
    }
    std::vector<float> h(tot, 0.0f);
    const float* src = host_weights;
    for (int l = 0; l < 12; ++l) {
        for (int o = 0; o < fout[l]; ++o)
            for (int i = 0; i < fin[l]; ++i) h[offW[l] + (size_t)o * kpad[l] + i] = src[(size_t)o * fin[l] + i];
        src += (size_t)fin[l] * fout[l];
        for (int o = 0; o < fout[l]; ++o) h[offB[l] + o] = src[o];
        src += fout[l];
    }
    int rc;
    if ((rc = cuda_check(cudaMalloc(&m->w32, tot * sizeof(float)), "cudaMalloc(weights)"))) {
        free_map(m);
        return rc;
    }
    if ((rc = cuda_check(cudaMemcpy(m->w32, h.data(), tot * sizeof(float), cudaMemcpyHostToDevice),
                         "cudaMemcpy(weights)"))) {
        free_map(m);
        return rc;
    }
    m->w32_n = tot;
    for (int l = 0; l < 12; ++l) {
        m->L[l].W = m->w32 + offW[l];
        m->L[l].b = m->w32 + offB[l];
        m->L[l].n = fout[l];
        m->L[l].k_pad = kpad[l];
    }
    // ---- workspace -------------------------------------------------------
    const size_t R = (size_t)cfg->max_rays, S = (size_t)cfg->max_samples;
    m->chunk_rows = 1 << 19;
    if ((size_t)m->chunk_rows > R * S) m->chunk_rows = (int)(((R * S) + 127) / 128 * 128);
    struct {
        void** p;
        size_t bytes;
        const char* what;
    } allocs[] = {
        {(void**)&m->rays, R * sizeof(Ray), "rays"},
        {(void**)&m->gd, R * kGdPad * sizeof(float), "gamma(d)"},
        {(void**)&m->zc, R * S * sizeof(float), "z coarse"},
        {(void**)&m->zf, R * S * sizeof(float), "z fine"},
        {(void**)&m->out_c, R * S * sizeof(float4), "coarse outputs"},
        {(void**)&m->out_f, R * S * sizeof(float4), "fine outputs"},
        {(void**)&m->obs, R * sizeof(float4), "observed colours"},
        {(void**)&m->e_ray, R * sizeof(float), "per-ray loss"},
        {(void**)&m->logw64, (size_t)cfg->max_particles * sizeof(double), "log weights"},
        {(void**)&m->cdf, (size_t)cfg->max_particles * sizeof(unsigned long long), "cdf"},
        {(void**)&m->status, sizeof(Status), "status"},
        {(void**)&m->act0, (size_t)m->chunk_rows * kWidth * sizeof(float), "act0"},
        {(void**)&m->act1, (size_t)m->chunk_rows * kWidth * sizeof(float), "act1"},
        {(void**)&m->gxbuf, (size_t)m->chunk_rows * kGxPad * sizeof(float), "gamma(x)"},
        {(void**)&m->loop.plan, sizeof(LoopPlan), "loop plan"},
        {(void**)&m->loop.qs, (size_t)cfg->max_queries * sizeof(LoopQuery), "loop state"},
        {(void**)&m->loop.n0, (size_t)cfg->max_queries * sizeof(int), "loop n0"},
        {(void**)&m->loop.imgs, (size_t)cfg->max_queries * sizeof(float*), "loop images"},
        {(void**)&m->loop.pix, (size_t)cfg->max_queries * kLoopMaxPixels * 2 * sizeof(int32_t),
         "loop pixels"},
        {(void**)&m->loop.P_next, (size_t)cfg->max_particles * 12 * sizeof(float), "loop particles"},
        {(void**)&m->loop.w, (size_t)cfg->max_particles * sizeof(double), "loop weights"},
        {(void**)&m->loop.mask, (size_t)cfg->max_particles, "loop mask"},
        {(void**)&m->loop.idx, (size_t)cfg->max_particles * sizeof(int32_t), "loop indices"},
    };
    for (auto& a : allocs) {
        if ((rc = cuda_check(cudaMalloc(a.p, a.bytes), a.what))) {
            free_map(m);
            return rc;
        }
    }
    cudaMemset(m->status, 0, sizeof(Status));
    if ((rc = cuda_check(cudaStreamCreateWithFlags(&m->loop.stream, cudaStreamNonBlocking),
                         "loop stream")) ||
        (rc = cuda_check(cudaEventCreateWithFlags(&m->loop.ev_in, cudaEventDisableTiming), "event")) ||
        (rc = cuda_check(cudaEventCreateWithFlags(&m->loop.ev_out, cudaEventDisableTiming), "event"))) {
        free_map(m);
        return rc;
    }
    if ((rc = proposal_alloc(m))) {
        free_map(m);
        return rc;
    }
    if ((rc = mlp_tc_prepare(m, host_weights))) {
        free_map(m);
        return rc;
    }
    if ((rc = cuda_check(cudaDeviceSynchronize(), "mcl_init_map"))) {
        free_map(m);
        return rc;
    }
    *out_map = m;
    return MCL_OK;
}

extern "C" void mcl_destroy_map(mcl_map* map) {
    if (!map) return;
    cudaDeviceSynchronize();
    free_map(map);
}

static int check_opts(const mcl_opts* o) {
    if (!o) return fail(MCL_ERR_ARG, "opts is NULL");
    if (o->n_coarse < 2 || o->n_coarse > kMaxCoarse || o->n_fine < 0 || o->n_fine > kMaxFine)
        return fail(MCL_ERR_ARG, "n_coarse %d / n_fine %d out of range", o->n_coarse, o->n_fine);
    if (o->precision < MCL_PREC_FP32 || o->precision > MCL_PREC_FP8)
        return fail(MCL_ERR_ARG, "precision %d unknown", o->precision);
    if (!(o->near_z < o->far_z) || !(o->alpha > 0.f && o->alpha < 0.5f) || !(o->tau > 0.f) ||
        !(o->rho_reject >= 0.0) || !(o->s_min > 0.0))
        return fail(MCL_ERR_ARG, "bad near/far/alpha/tau/rho/s_min");
    return MCL_OK;
}

// Sample counts against the workspace (both samplers).
static int check_samples(const mcl_map* m, const mcl_opts* o) {
    if (o->use_proposal) {
        if (!m->has_proposal) return fail(MCL_ERR_ARG, "use_proposal: no proposal weights set or trained");
        if (o->n_proposal < 2 || o->n_proposal > kMaxCoarse || o->n_guided < 2 ||
            o->n_guided > kMaxCoarse)
            return fail(MCL_ERR_ARG, "n_proposal %d / n_guided %d out of range", o->n_proposal,
                        o->n_guided);
        if (o->n_proposal > m->cfg.max_samples || o->n_guided + o->n_fine > m->cfg.max_samples)
            return fail(MCL_ERR_ARG, "proposal sample counts exceed max_samples %d", m->cfg.max_samples);
    } else if (o->n_coarse + o->n_fine > m->cfg.max_samples) {
        return fail(MCL_ERR_ARG, "n_coarse + n_fine > max_samples %d", m->cfg.max_samples);
    }
    return MCL_OK;
}

// The two sample sets the final composite merges (after render_passes);
// fused: the tensor-core MLP's last pass has already composited them.
struct Passes {
    const float* za;
    const float4* oa;
    int na;
    const float* zb;
    const float4* ob;
    int nb;
    int factor;
    bool fused;
};

// Per-ray outputs of the final stage (composite, Eq. 5 / F, E), produced by
// the fused epilogue of the tensor-core forms when the pass shapes allow it.
struct FinalOut {
    const float* image;   // observation [H, W, 3] (NULL: render only)
    float* e_ray;         // E * F per ray (with image)
    float* rgb;
    float* E;
    float* F;
    float* z_trans;
    float* z_opaque;
};

// Common front half of mcl_update, mcl_render and the training targets:
// rays, then either coarse + importance samples (the basic model's
// hierarchical sampler) or proposal + guided + importance samples.
static int render_passes(mcl_map* m, const float* d_poses, int N, const mcl_intrinsics* K,
                         int level, const int32_t* d_pixels, int B, const mcl_opts* o,
                         Passes* out, cudaStream_t s, const FinalOut* fin = nullptr) {
    int rc;
    if ((rc = check_opts(o))) return rc;
    if (!d_poses || !K || !d_pixels) return fail(MCL_ERR_ARG, "NULL pose / intrinsics / pixel set");
    if (N < 1 || B < 1 || (long)N * B > m->cfg.max_rays)
        return fail(MCL_ERR_ARG, "N*B = %ld outside [1, max_rays=%d]", (long)N * B, m->cfg.max_rays);
    if ((rc = check_samples(m, o))) return rc;
    const bool prop = o->use_proposal != 0;
    if (level < 0 || level > 2) return fail(MCL_ERR_ARG, "level %d not in 0..2", level);
    const int f = 4 >> level;
    if (K->width < 1 || K->height < 1 || K->width % f || K->height % f)
        return fail(MCL_ERR_ARG, "image %dx%d not divisible by level factor %d", K->width, K->height, f);
    if (!(K->fx > 0.f) || !(K->fy > 0.f)) return fail(MCL_ERR_ARG, "focal length must be > 0");
    const int nr = N * B;
    if (o->precision != MCL_PREC_FP32 && !mlp_tc_available(m, o->precision))
        return fail(MCL_ERR_UNSUPPORTED, "precision %d is not available on this device", o->precision);
    mcl_opts ro = *o;
    if (prop) {   // stratified midpoints of the proposal (the samples it was trained on)
        ro.n_coarse = o->n_proposal;
        ro.jitter = 0;
    }
    // fused ray epilogues: the first NeRF pass (coarse or guided samples, nA
    // per ray) draws the importance samples, the last composites
    const int nA = prop ? o->n_guided : o->n_coarse;
    const bool fused = fin && o->precision != MCL_PREC_FP32 && m->fuse_epilogue &&
                       (o->n_fine > 0 ? mlp_tc_can_fuse(1, nA, 0) && mlp_tc_can_fuse(2, o->n_fine, nA)
                                      : mlp_tc_can_fuse(2, nA, 0));
    out->fused = fused;
    FuseArgs fa1{}, fa2{};
    if (fused) {
        fa1.mode = 1;
        fa1.nf_out = o->n_fine;
        fa2.mode = 2;
        fa2.alpha = o->alpha;
        fa2.tau = o->tau;
        fa2.use_rej = o->use_rejection;
        fa2.obs = fin->image ? m->obs : nullptr;
        fa2.e_ray = fin->e_ray;
        fa2.rgb_out = fin->rgb;
        fa2.E_out = fin->E;
        fa2.F_out = fin->F;
        fa2.zt_out = fin->z_trans;
        fa2.zo_out = fin->z_opaque;
    }
    {
        PhaseScope ph(m, MCL_PHASE_RAYGEN, s);
        const bool with_obs = fused && fin->image;
        if ((rc = cuda_check(launch_raygen(d_poses, N, d_pixels, B, K->fx / f, K->fy / f,
                                           K->cx / f, K->cy / f, ro, m->rays, m->gd, m->zc, s,
                                           with_obs ? fin->image : nullptr, K->width, K->height, f,
                                           with_obs ? m->obs : nullptr),
                             "raygen")))
            return rc;
        if (o->precision != MCL_PREC_FP32 &&
            (rc = cuda_check(mlp_tc_ray_bias(m, m->gd, nr, nullptr, s), "per-ray bias")))
            return rc;
    }
    auto mlp = [&](const float* z, int S, float4* dst, const FuseArgs* fa) -> cudaError_t {
        if (o->precision == MCL_PREC_FP32) return mlp_fp32(m, m->rays, m->gd, z, S, nr, dst, s);
        return mlp_tc(m, o->precision, m->rays, m->gd, z, S, nr, nullptr, dst, s, fa);
    };
    out->factor = f;
    if (!prop) {
        if (fused) {
            // coarse pass: its epilogue draws the importance samples into zf
            // (or, without them, composites); fine pass: final composite
            fa1.z_out = m->zf;
            fa2.z_first = m->zc;
            fa2.out_first = m->out_c;
            fa2.S1 = o->n_fine > 0 ? o->n_coarse : 0;
            {
                PhaseScope ph(m, MCL_PHASE_MLP_COARSE, s);
                if ((rc = cuda_check(mlp(m->zc, o->n_coarse, m->out_c, o->n_fine > 0 ? &fa1 : &fa2),
                                     "mlp (coarse, fused)")))
                    return rc;
            }
            if (o->n_fine > 0) {
                PhaseScope ph(m, MCL_PHASE_MLP_FINE, s);
                if ((rc = cuda_check(mlp(m->zf, o->n_fine, m->out_f, &fa2), "mlp (fine, fused)")))
                    return rc;
            }
            return MCL_OK;
        }
        {
            PhaseScope ph(m, MCL_PHASE_MLP_COARSE, s);
            if ((rc = cuda_check(mlp(m->zc, o->n_coarse, m->out_c, nullptr), "mlp (coarse)"))) return rc;
        }
        if (o->n_fine > 0) {
            {
                PhaseScope ph(m, MCL_PHASE_SAMPLE, s);
                if ((rc = cuda_check(launch_coarse_to_fine(m->rays, nr, nullptr, m->zc, o->n_coarse,
                                                           m->out_c, o->n_fine, m->zf, s),
                                     "importance sampling")))
                    return rc;
            }
            PhaseScope ph(m, MCL_PHASE_MLP_FINE, s);
            if ((rc = cuda_check(mlp(m->zf, o->n_fine, m->out_f, nullptr), "mlp (fine)"))) return rc;
        }
        *out = Passes{m->zc, m->out_c, o->n_coarse, m->zf, m->out_f, o->n_fine, f, false};
        return MCL_OK;
    }
    // proposal: densities at the stratified samples (into out_f), guided
    // samples from their weights (into zf), NeRF MLP there (into out_c),
    // importance samples from those (into zc), NeRF MLP (into out_f)
    {
        PhaseScope ph(m, MCL_PHASE_SAMPLE, s);
        if ((rc = cuda_check(launch_prop_infer(m, o->precision, m->rays, m->zc, o->n_proposal, nr, nullptr,
                                               m->out_f, s),
                             "proposal")))
            return rc;
        if ((rc = cuda_check(launch_coarse_to_fine(m->rays, nr, nullptr, m->zc, o->n_proposal,
                                                   m->out_f, o->n_guided, m->zf, s),
                             "proposal sampling")))
            return rc;
    }
    if (fused) {
        // guided pass: its epilogue draws the importance samples into zc (or,
        // without them, composites); importance pass: final composite
        fa1.z_out = m->zc;
        fa2.z_first = m->zf;
        fa2.out_first = m->out_c;
        fa2.S1 = o->n_fine > 0 ? o->n_guided : 0;
        {
            PhaseScope ph(m, MCL_PHASE_MLP_COARSE, s);
            if ((rc = cuda_check(mlp(m->zf, o->n_guided, m->out_c, o->n_fine > 0 ? &fa1 : &fa2),
                                 "mlp (guided, fused)")))
                return rc;
        }
        if (o->n_fine > 0) {
            PhaseScope ph(m, MCL_PHASE_MLP_FINE, s);
            if ((rc = cuda_check(mlp(m->zc, o->n_fine, m->out_f, &fa2), "mlp (fine, fused)")))
                return rc;
        }
        return MCL_OK;
    }
    {
        PhaseScope ph(m, MCL_PHASE_MLP_COARSE, s);
        if ((rc = cuda_check(mlp(m->zf, o->n_guided, m->out_c, nullptr), "mlp (guided)"))) return rc;
    }
    if (o->n_fine > 0) {
        {
            PhaseScope ph(m, MCL_PHASE_SAMPLE, s);
            if ((rc = cuda_check(launch_coarse_to_fine(m->rays, nr, nullptr, m->zf, o->n_guided,
                                                       m->out_c, o->n_fine, m->zc, s),
                                 "importance sampling")))
                return rc;
        }
        PhaseScope ph(m, MCL_PHASE_MLP_FINE, s);
        if ((rc = cuda_check(mlp(m->zc, o->n_fine, m->out_f, nullptr), "mlp (fine)"))) return rc;
    }
    *out = Passes{m->zf, m->out_c, o->n_guided, m->zc, m->out_f, o->n_fine, f, false};
    return MCL_OK;
}

// Full-sampler render used for the distillation targets (proposal off).
static int render_full(mcl_map* m, const float* d_poses, int N, const mcl_intrinsics* K, int level,
                       const int32_t* d_pixels, int B, const mcl_opts* o, cudaStream_t s) {
    mcl_opts full = *o;
    full.use_proposal = 0;
    Passes ps;
    return render_passes(m, d_poses, N, K, level, d_pixels, B, &full, &ps, s);
}

extern "C" int mcl_update(mcl_map* m, const float* d_particles, int N, const float* d_image,
                          const mcl_intrinsics* K, int level, const int32_t* d_pixels, int B,
                          const mcl_opts* o, float* d_logw, double* d_w, uint8_t* d_mask,
                          const mcl_debug* dbg, void* stream) {
    g_err[0] = 0;
    if (!m) return fail(MCL_ERR_ARG, "mcl_update: map is NULL");
    if (!d_image || !d_logw || !d_w || !d_mask) return fail(MCL_ERR_ARG, "mcl_update: NULL output/image");
    if (N > m->cfg.max_particles) return fail(MCL_ERR_ARG, "N %d > max_particles %d", N, m->cfg.max_particles);
    cudaStream_t s = (cudaStream_t)stream;
    int rc;
    Passes ps;
    const FinalOut fin{d_image, m->e_ray, dbg ? dbg->rgb : nullptr, dbg ? dbg->E : nullptr,
                       dbg ? dbg->F : nullptr, dbg ? dbg->z_trans : nullptr,
                       dbg ? dbg->z_opaque : nullptr};
    if ((rc = render_passes(m, d_particles, N, K, level, d_pixels, B, o, &ps, s, &fin))) return rc;
    const int nr = N * B;
    if (!ps.fused) {
        PhaseScope ph(m, MCL_PHASE_COMPOSITE, s);
        if ((rc = cuda_check(launch_final_composite(m->rays, nr, ps.za, ps.oa, ps.na, ps.zb, ps.ob,
                                                    ps.nb, d_image, K->width, K->height, ps.factor,
                                                    d_pixels, B, *o, m->e_ray, dbg, nullptr,
                                                    nullptr, s),
                             "composite")))
            return rc;
    }
    PhaseScope ph(m, MCL_PHASE_WEIGHTS, s);
    return cuda_check(launch_weights(m->e_ray, N, B, *o, d_logw, m->logw64, d_w, d_mask,
                                     dbg ? dbg->S : nullptr, m->status, s),
                      "weights");
}

extern "C" int mcl_query(mcl_map* m, const float* d_x, const float* d_dir, int n, int precision,
                         float* d_out, void* stream) {
    g_err[0] = 0;
    if (!m || !d_x || !d_dir || !d_out) return fail(MCL_ERR_ARG, "mcl_query: NULL argument");
    if (n < 1 || n > m->cfg.max_rays) return fail(MCL_ERR_ARG, "mcl_query: n %d outside [1, %d]", n, m->cfg.max_rays);
    if (((uintptr_t)d_out) % 16) return fail(MCL_ERR_ARG, "mcl_query: d_out must be 16-byte aligned");
    if (precision != MCL_PREC_FP32 && !mlp_tc_available(m, precision))
        return fail(MCL_ERR_UNSUPPORTED, "precision %d is not available on this device", precision);
    cudaStream_t s = (cudaStream_t)stream;
    int rc;
    if ((rc = cuda_check(launch_query_setup(d_x, d_dir, n, m->rays, m->gd, m->zc, s), "query setup")))
        return rc;
    if (precision == MCL_PREC_FP32)
        return cuda_check(mlp_fp32(m, m->rays, m->gd, m->zc, 1, n, (float4*)d_out, s), "query mlp");
    if ((rc = cuda_check(mlp_tc_ray_bias(m, m->gd, n, nullptr, s), "query ray bias"))) return rc;
    return cuda_check(mlp_tc(m, precision, m->rays, m->gd, m->zc, 1, n, nullptr, (float4*)d_out, s),
                      "query mlp");
}

extern "C" int mcl_proposal_query(mcl_map* m, const float* d_x, int n, int precision,
                                  float* d_sigma, void* stream) {
    g_err[0] = 0;
    if (!m || !d_x || !d_sigma) return fail(MCL_ERR_ARG, "mcl_proposal_query: NULL argument");
    if (n < 1 || n > m->cfg.max_rays)
        return fail(MCL_ERR_ARG, "mcl_proposal_query: n %d outside [1, %d]", n, m->cfg.max_rays);
    if (!m->has_proposal) return fail(MCL_ERR_ARG, "mcl_proposal_query: no proposal weights set or trained");
    if (precision != MCL_PREC_FP32 && !mlp_tc_available(m, precision))
        return fail(MCL_ERR_UNSUPPORTED, "precision %d is not available on this device", precision);
    cudaStream_t s = (cudaStream_t)stream;
    int rc;
    // rays from the points with zero-length steps (z = 0), one sample each
    if ((rc = cuda_check(launch_query_setup(d_x, d_x, n, m->rays, m->gd, m->zc, s), "query setup")) ||
        (rc = cuda_check(launch_prop_infer(m, precision, m->rays, m->zc, 1, n, nullptr, m->out_c, s),
                         "proposal")))
        return rc;
    return cuda_check(cudaMemcpy2DAsync(d_sigma, sizeof(float), m->out_c, sizeof(float4), sizeof(float),
                                        n, cudaMemcpyDeviceToDevice, s),
                      "copy densities");
}

extern "C" int mcl_render(mcl_map* m, const float* d_poses, int n_poses, const mcl_intrinsics* K,
                          int level, const int32_t* d_pixels, int B, const mcl_opts* o,
                          float* d_rgb, float* d_F, void* stream) {
    g_err[0] = 0;
    if (!m || !d_rgb) return fail(MCL_ERR_ARG, "mcl_render: NULL map / output");
    cudaStream_t s = (cudaStream_t)stream;
    int rc;
    Passes ps;
    const FinalOut fin{nullptr, nullptr, d_rgb, nullptr, d_F, nullptr, nullptr};
    if ((rc = render_passes(m, d_poses, n_poses, K, level, d_pixels, B, o, &ps, s, &fin))) return rc;
    if (ps.fused) return MCL_OK;
    PhaseScope ph(m, MCL_PHASE_COMPOSITE, s);
    return cuda_check(launch_final_composite(m->rays, n_poses * B, ps.za, ps.oa, ps.na, ps.zb,
                                             ps.ob, ps.nb, nullptr, K->width, K->height, ps.factor,
                                             d_pixels, B, *o, nullptr, nullptr, d_rgb, d_F, s),
                      "composite");
}

extern "C" int mcl_resample(mcl_map* m, const double* d_w, int N_in, int N_out, double u0,
                            int32_t* d_idx, void* stream) {
    g_err[0] = 0;
    if (!m || !d_w || !d_idx) return fail(MCL_ERR_ARG, "mcl_resample: NULL argument");
    if (N_in < 1 || N_in > m->cfg.max_particles)
        return fail(MCL_ERR_ARG, "mcl_resample: N_in %d outside [1, %d]", N_in, m->cfg.max_particles);
    if (N_out < 1 || N_out > 65536) return fail(MCL_ERR_ARG, "mcl_resample: N_out %d outside [1, 65536]", N_out);
    if (!(u0 >= 0.0 && u0 < 1.0)) return fail(MCL_ERR_ARG, "mcl_resample: u0 must be in [0, 1)");
    PhaseScope ph(m, MCL_PHASE_RESAMPLE, (cudaStream_t)stream);
    return cuda_check(launch_resample(d_w, N_in, N_out, u0, d_idx, m->cdf, m->status,
                                      (cudaStream_t)stream),
                      "resample");
}

extern "C" int mcl_predict_odom(const float* d_in, int N_in, const int32_t* d_idx, int N_out,
                                const float* d_odom, float sigma_t, float sigma_yaw, uint64_t seed,
                                uint64_t counter, float* d_out, void* stream) {
    g_err[0] = 0;
    if (!d_in || !d_out || N_out < 1 || N_in < 1) return fail(MCL_ERR_ARG, "mcl_predict: bad argument");
    if (!d_idx && N_out > N_in) return fail(MCL_ERR_ARG, "mcl_predict: N_out > N_in without an index");
    if (!(sigma_t >= 0.f) || !(sigma_yaw >= 0.f)) return fail(MCL_ERR_ARG, "mcl_predict: negative sigma");
    if (d_in == d_out && d_idx) return fail(MCL_ERR_ARG, "mcl_predict: in-place gather is not allowed");
    return cuda_check(launch_predict(d_in, N_in, d_idx, N_out, d_odom, sigma_t, sigma_yaw, seed, counter,
                                     d_out, (cudaStream_t)stream),
                      "predict");
}

extern "C" int mcl_predict(const float* d_in, int N_in, const int32_t* d_idx, int N_out,
                           float sigma_t, float sigma_yaw, uint64_t seed, uint64_t counter,
                           float* d_out, void* stream) {
    return mcl_predict_odom(d_in, N_in, d_idx, N_out, nullptr, sigma_t, sigma_yaw, seed, counter,
                            d_out, stream);
}

extern "C" int mcl_downscale(const float* d_image, int W, int H, int factor, float* d_out,
                             void* stream) {
    g_err[0] = 0;
    if (!d_image || !d_out || W < 1 || H < 1 || factor < 1 || W % factor || H % factor)
        return fail(MCL_ERR_ARG, "mcl_downscale: bad argument");
    return cuda_check(launch_downscale(d_image, W, H, factor, d_out, (cudaStream_t)stream), "downscale");
}

extern "C" int mcl_position_spread(const float* d_poses, int N, double* d_out, void* stream) {
    g_err[0] = 0;
    if (!d_poses || !d_out || N < 1) return fail(MCL_ERR_ARG, "mcl_position_spread: bad argument");
    return cuda_check(launch_position_spread(d_poses, N, d_out, (cudaStream_t)stream), "spread");
}

extern "C" int mcl_read_status(mcl_map* m, int* n_nonfinite, void* stream) {
    g_err[0] = 0;
    if (!m) return fail(MCL_ERR_ARG, "mcl_read_status: map is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    Status st;
    int rc;
    if ((rc = cuda_check(cudaMemcpyAsync(&st, m->status, sizeof(Status), cudaMemcpyDeviceToHost, s),
                         "status read")))
        return rc;
    if ((rc = cuda_check(cudaStreamSynchronize(s), "status sync"))) return rc;
    if ((rc = cuda_check(cudaMemsetAsync(m->status, 0, sizeof(Status), s), "status clear"))) return rc;
    if (n_nonfinite) *n_nonfinite = st.n_nonfinite;
    return st.code;
}

extern "C" int mcl_profile_enable(mcl_map* m, int enable) {
    g_err[0] = 0;
    if (!m) return fail(MCL_ERR_ARG, "mcl_profile_enable: map is NULL");
    m->prof = enable != 0;
    return MCL_OK;
}

extern "C" int mcl_profile_read(mcl_map* m, double* ms_out, long long* n_launches, int reset) {
    g_err[0] = 0;
    if (!m) return fail(MCL_ERR_ARG, "mcl_profile_read: map is NULL");
    for (auto& mk : m->marks) {
        int rc;
        if ((rc = cuda_check(cudaEventSynchronize(mk.b), "profile sync"))) return rc;
        float ms = 0.f;
        if ((rc = cuda_check(cudaEventElapsedTime(&ms, mk.a, mk.b), "profile elapsed"))) return rc;
        m->phase_ms[mk.phase] += ms;
        m->pool.push_back(mk.a);
        m->pool.push_back(mk.b);
    }
    m->marks.clear();
    if (ms_out)
        for (int i = 0; i < MCL_N_PHASES; ++i) ms_out[i] = m->phase_ms[i];
    if (n_launches) *n_launches = g_launches.load();
    if (reset)
        for (int i = 0; i < MCL_N_PHASES; ++i) m->phase_ms[i] = 0.0;
    return MCL_OK;
}

extern "C" int mcl_map_supports(const mcl_map* m, int precision) {
    if (!m) return 0;
    if (precision == MCL_PREC_FP32) return 1;
    if (precision == MCL_PREC_BF16 || precision == MCL_PREC_FP8)
        return mlp_tc_available(m, precision) ? 1 : 0;
    return 0;
}

extern "C" int mcl_draw_pixels(int W, int H, int B, uint64_t seed, uint64_t counter,
                               int32_t* d_out, void* stream) {
    g_err[0] = 0;
    if (!d_out || W < 1 || H < 1 || B < 1 || B > 1024 || (long)B > (long)W * H)
        return fail(MCL_ERR_ARG, "mcl_draw_pixels: bad argument (W %d H %d B %d)", W, H, B);
    return cuda_check(launch_draw_pixels(W, H, B, seed, counter, d_out, (cudaStream_t)stream),
                      "draw pixels");
}

static unsigned long long mix_key(unsigned long long h, const void* p, size_t n) {
    const unsigned char* b = (const unsigned char*)p;
    for (size_t i = 0; i < n; ++i) h = (h ^ b[i]) * 0x100000001B3ull;  // FNV-1a
    return h;
}

extern "C" int mcl_localize(mcl_map* m, int nq, float* d_particles, int stride, const int* h_n0,
                            const float* const* h_images, const mcl_intrinsics* K,
                            const mcl_schedule* sch, const mcl_opts* o, mcl_iter_record* d_log,
                            int* d_final_n, int use_graph, void* stream) {
    g_err[0] = 0;
    int rc;
    if (!m || !d_particles || !h_n0 || !h_images || !K || !sch || !o || !d_log || !d_final_n)
        return fail(MCL_ERR_ARG, "mcl_localize: NULL argument");
    if ((rc = check_opts(o))) return rc;
    if (o->precision != MCL_PREC_FP32 && !mlp_tc_available(m, o->precision))
        return fail(MCL_ERR_UNSUPPORTED, "mcl_localize: precision %d is not available on this device",
                    o->precision);
    if (nq < 1 || nq > m->cfg.max_queries) return fail(MCL_ERR_ARG, "mcl_localize: n_queries %d", nq);
    if (stride < 1 || (long)nq * stride > m->cfg.max_particles)
        return fail(MCL_ERR_ARG, "mcl_localize: n_queries * stride > max_particles");
    if (sch->n_stages < 1 || sch->n_stages > MCL_MAX_STAGES || sch->iterations < 1 || sch->n_min < 1)
        return fail(MCL_ERR_ARG, "mcl_localize: bad schedule");
    int maxB = 0, maxf = 1;
    for (int st = 0; st < sch->n_stages; ++st) {
        if (sch->level[st] < 0 || sch->level[st] > 2 || sch->n_pixels[st] < 1 ||
            sch->n_pixels[st] > kLoopMaxPixels || sch->n_cap[st] < 1 || sch->n_cap[st] > stride ||
            sch->stage_iter_cap[st] < 1)
            return fail(MCL_ERR_ARG, "mcl_localize: bad stage %d", st);
        const int f = 4 >> sch->level[st];
        if (sch->n_pixels[st] > maxB) maxB = sch->n_pixels[st];
        if (f > maxf) maxf = f;
        if ((long)(K->width / f) * (K->height / f) < sch->n_pixels[st])
            return fail(MCL_ERR_ARG, "mcl_localize: stage %d asks for more pixels than its level has", st);
    }
    if (!(sch->sigma_t >= 0.f) || !(sch->sigma_yaw >= 0.f))
        return fail(MCL_ERR_ARG, "mcl_localize: negative motion noise");
    if (K->width < 1 || K->height < 1 || K->width % maxf || K->height % maxf || !(K->fx > 0.f) ||
        !(K->fy > 0.f))
        return fail(MCL_ERR_ARG, "mcl_localize: bad intrinsics for the schedule's levels");
    for (int q = 0; q < nq; ++q) {
        if (h_n0[q] < 1 || h_n0[q] > stride) return fail(MCL_ERR_ARG, "mcl_localize: n0[%d]", q);
        if (!h_images[q]) return fail(MCL_ERR_ARG, "mcl_localize: image %d is NULL", q);
    }
    // largest rays of one iteration: a query has its n0 particles in the
    // first iteration and at most its stage's cap afterwards
    int max_n0 = 0;
    for (int q = 0; q < nq; ++q) max_n0 = std::max(max_n0, h_n0[q]);
    long per_query = (long)max_n0 * sch->n_pixels[0];
    for (int st = 0; st < sch->n_stages; ++st)
        per_query = std::max(per_query, (long)std::min(sch->n_cap[st], stride) * sch->n_pixels[st]);
    const long max_rays_run = (long)nq * per_query;
    (void)maxB;
    if (max_rays_run > m->cfg.max_rays)
        return fail(MCL_ERR_ARG, "mcl_localize: %ld rays in the largest iteration > max_rays %d",
                    max_rays_run, m->cfg.max_rays);
    if ((rc = check_samples(m, o))) return rc;
    cudaStream_t caller = (cudaStream_t)stream;
    // the first graph-mode run of a precision picks the MLP kernel variant
    // (synchronous; never inside a capture)
    if (use_graph && o->precision != MCL_PREC_FP32 && !mlp_tc_tuned(m, o->precision)) {
        const int S = std::min(64, m->cfg.max_samples);
        const long long rows = std::min((long long)max_rays_run * S, (long long)m->cfg.max_rays * S);
        if (rows >= 256 && (rc = mlp_tc_autotune(m, o->precision, rows, nullptr, nullptr, caller)))
            return rc;
    }
    // graph mode captures on the map's own stream, ordered after the caller's
    // work and before the caller's later work by two events
    cudaStream_t s = use_graph ? m->loop.stream : caller;
    if (use_graph) {
        if ((rc = cuda_check(cudaEventRecord(m->loop.ev_in, caller), "event record")) ||
            (rc = cuda_check(cudaStreamWaitEvent(s, m->loop.ev_in, 0), "stream wait")))
            return rc;
    }
    // per-call inputs read by the run's kernels
    if ((rc = cuda_check(cudaMemcpyAsync(m->loop.n0, h_n0, sizeof(int) * nq, cudaMemcpyHostToDevice, s),
                         "upload n0")))
        return rc;
    if ((rc = cuda_check(cudaMemcpyAsync((void*)m->loop.imgs, h_images, sizeof(float*) * nq,
                                         cudaMemcpyHostToDevice, s),
                         "upload image pointers")))
        return rc;
    m->loop.max_rays_run = (int)max_rays_run;
    if (!use_graph)
        return enqueue_localize(m, nq, d_particles, stride, *K, *sch, *o, d_log, d_final_n, s);
    unsigned long long key = 1469598103934665603ull;
    const void* ptrs[] = {d_particles, d_log, d_final_n};
    key = mix_key(key, &nq, sizeof(nq));
    key = mix_key(key, &stride, sizeof(stride));
    key = mix_key(key, ptrs, sizeof(ptrs));
    key = mix_key(key, K, sizeof(*K));
    key = mix_key(key, sch, sizeof(*sch));
    key = mix_key(key, o, sizeof(*o));
    key = mix_key(key, &max_rays_run, sizeof(max_rays_run));
    if (!m->loop.exec || m->loop.key != key) {
        if (m->loop.exec) {
            cudaGraphExecDestroy(m->loop.exec);
            m->loop.exec = nullptr;
        }
        if ((rc = cuda_check(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal),
                             "begin capture")))
            return rc;
        const int erc = enqueue_localize(m, nq, d_particles, stride, *K, *sch, *o, d_log, d_final_n, s);
        cudaGraph_t g = nullptr;
        const cudaError_t ce = cudaStreamEndCapture(s, &g);
        if (erc) {
            if (g) cudaGraphDestroy(g);
            return erc;
        }
        if ((rc = cuda_check(ce, "end capture"))) return rc;
        rc = cuda_check(cudaGraphInstantiate(&m->loop.exec, g, 0), "instantiate graph");
        cudaGraphDestroy(g);
        if (rc) return rc;
        m->loop.key = key;
    }
    if ((rc = cuda_check(cudaGraphLaunch(m->loop.exec, s), "launch graph"))) return rc;
    if ((rc = cuda_check(cudaEventRecord(m->loop.ev_out, s), "event record"))) return rc;
    return cuda_check(cudaStreamWaitEvent(caller, m->loop.ev_out, 0), "stream wait");
}

extern "C" int mcl_autotune(mcl_map* m, int precision, long long rows, int* chosen, float* ms,
                            void* stream) {
    g_err[0] = 0;
    if (!m) return fail(MCL_ERR_ARG, "mcl_autotune: NULL map");
    if (precision != MCL_PREC_BF16 && precision != MCL_PREC_FP8)
        return fail(MCL_ERR_ARG, "mcl_autotune: precision %d has no kernel variants", precision);
    return mlp_tc_autotune(m, precision, rows, chosen, ms, (cudaStream_t)stream);
}

extern "C" int mcl_inject_weight_stall(mcl_map* m, int n_launches, double wait_ms) {
    g_err[0] = 0;
    if (!m) return fail(MCL_ERR_ARG, "mcl_inject_weight_stall: NULL map");
    if (n_launches < 0 || !(wait_ms >= 0.01 && wait_ms <= 2000.0))
        return fail(MCL_ERR_ARG, "mcl_inject_weight_stall: n_launches >= 0, 0.01 <= wait_ms <= 2000");
    return mlp_tc_hold_weights(m, n_launches, (unsigned long long)(wait_ms * 1e6));
}

extern "C" int mcl_set_fused_epilogue(mcl_map* m, int enable) {
    g_err[0] = 0;
    if (!m) return fail(MCL_ERR_ARG, "mcl_set_fused_epilogue: NULL map");
    m->fuse_epilogue = enable != 0;
    m->loop.key = 0;   // a captured loop holds the old launch sequence
    return MCL_OK;
}

extern "C" int mcl_fit_map(mcl_map* m, const float* d_x, const float* d_dir, const float* d_target,
                           int n, const mcl_fit_cfg* cfg, float* d_loss_log, void* stream) {
    g_err[0] = 0;
    if (!m || !d_x || !d_dir || !d_target || !cfg || n < 1)
        return fail(MCL_ERR_ARG, "mcl_fit_map: bad argument");
    if (cfg->steps < 1 || cfg->batch < 1 || !(cfg->lr > 0.f) || !(cfg->beta1 >= 0.f && cfg->beta1 < 1.f) ||
        !(cfg->beta2 >= 0.f && cfg->beta2 < 1.f) || !(cfg->eps > 0.f) || !(cfg->sigma_weight >= 0.f))
        return fail(MCL_ERR_ARG, "mcl_fit_map: bad fitting configuration");
    cudaStream_t s = (cudaStream_t)stream;
    int rc;
    if ((rc = fit_map(m, d_x, d_dir, d_target, n, *cfg, d_loss_log, s))) return rc;
    // rebuild the tensor-core forms from the fitted weights
    std::vector<float> blob(blob_size());
    if ((rc = map_download(m, blob.data()))) return rc;
    if (m->loop.exec) {
        cudaGraphExecDestroy(m->loop.exec);
        m->loop.exec = nullptr;
    }
    m->loop.key = 0;
    mlp_tc_free(m);
    if ((rc = mlp_tc_prepare(m, blob.data()))) return rc;
    return cuda_check(cudaDeviceSynchronize(), "mcl_fit_map");
}

extern "C" int mcl_map_loss_grad(mcl_map* m, const float* d_x, const float* d_dir,
                                 const float* d_target, int n, float sigma_weight, double* d_loss,
                                 float* d_grad, void* stream) {
    g_err[0] = 0;
    if (!m || !d_x || !d_dir || !d_target || !d_loss || !d_grad || n < 1 || !(sigma_weight >= 0.f))
        return fail(MCL_ERR_ARG, "mcl_map_loss_grad: bad argument");
    return map_loss_grad(m, d_x, d_dir, d_target, n, sigma_weight, d_loss, d_grad, (cudaStream_t)stream);
}

extern "C" int mcl_get_map_weights(mcl_map* m, float* host_out, size_t n) {
    g_err[0] = 0;
    if (!m || !host_out || n != blob_size())
        return fail(MCL_ERR_ARG, "mcl_get_map_weights: need %zu floats", blob_size());
    return map_download(m, host_out);
}

extern "C" int mcl_set_mlp_variant(mcl_map* m, int precision, int variant) {
    g_err[0] = 0;
    if (!m) return fail(MCL_ERR_ARG, "mcl_set_mlp_variant: NULL map");
    return mlp_tc_set_variant(m, precision, variant);
}

extern "C" int mcl_proposal_set(mcl_map* m, const float* host, size_t n) {
    g_err[0] = 0;
    if (!m || !host || n != MCL_PROPOSAL_N_WEIGHTS)
        return fail(MCL_ERR_ARG, "mcl_proposal_set: need %d weights", MCL_PROPOSAL_N_WEIGHTS);
    for (size_t i = 0; i < n; ++i)
        if (!std::isfinite(host[i])) return fail(MCL_ERR_ARG, "mcl_proposal_set: weight %zu not finite", i);
    int rc;
    if ((rc = cuda_check(cudaMemcpy(m->prop_w, host, sizeof(float) * n, cudaMemcpyHostToDevice),
                         "upload proposal")))
        return rc;
    // fresh optimiser state for the new weights; BF16 copy for inference
    if ((rc = cuda_check(cudaMemset(m->prop_m, 0, sizeof(float) * 2 * n), "clear moments")) ||
        (rc = cuda_check(prop_tc_pack(m, 0), "pack proposal")) ||
        (rc = cuda_check(cudaDeviceSynchronize(), "pack proposal")))
        return rc;
    m->prop_step = 0;
    m->has_proposal = true;
    return MCL_OK;
}

extern "C" int mcl_proposal_get(mcl_map* m, float* host, size_t n) {
    g_err[0] = 0;
    if (!m || !host || n != MCL_PROPOSAL_N_WEIGHTS)
        return fail(MCL_ERR_ARG, "mcl_proposal_get: need %d weights", MCL_PROPOSAL_N_WEIGHTS);
    return cuda_check(cudaMemcpy(host, m->prop_w, sizeof(float) * n, cudaMemcpyDeviceToHost),
                      "download proposal");
}

extern "C" int mcl_render_histogram(mcl_map* m, const float* d_poses, int n_poses,
                                    const mcl_intrinsics* K, int level, const int32_t* d_pixels,
                                    int B, const mcl_opts* o, int n_bins, float* d_hist,
                                    void* stream) {
    g_err[0] = 0;
    if (!m || !d_hist || !o) return fail(MCL_ERR_ARG, "mcl_render_histogram: NULL argument");
    if (n_bins < 2 || n_bins > kMaxCoarse) return fail(MCL_ERR_ARG, "n_bins %d out of range", n_bins);
    cudaStream_t s = (cudaStream_t)stream;
    int rc;
    mcl_opts full = *o;
    full.use_proposal = 0;
    Passes ps;
    if ((rc = render_passes(m, d_poses, n_poses, K, level, d_pixels, B, &full, &ps, s))) return rc;
    return cuda_check(launch_histogram(m->rays, n_poses * B, ps.za, ps.oa, ps.na, ps.zb, ps.ob,
                                       ps.nb, n_bins, o->near_z, o->far_z, d_hist, s),
                      "histogram");
}

extern "C" int mcl_proposal_loss_grad(mcl_map* m, const float* d_o, const float* d_d, int n,
                                      int n_bins, float near_z, float far_z, const float* d_hist,
                                      double* d_loss, float* d_grad, void* stream) {
    g_err[0] = 0;
    if (!m || !d_o || !d_d || !d_hist || !d_loss || !d_grad || n < 1)
        return fail(MCL_ERR_ARG, "mcl_proposal_loss_grad: bad argument");
    if (n_bins < 2 || n_bins > kMaxCoarse || !(near_z < far_z))
        return fail(MCL_ERR_ARG, "mcl_proposal_loss_grad: bad bins / range");
    return proposal_loss_grad(m, d_o, d_d, n, n_bins, near_z, far_z, d_hist, d_loss, d_grad,
                              (cudaStream_t)stream);
}

extern "C" int mcl_proposal_train(mcl_map* m, const float* d_poses, int n_poses,
                                  const int32_t* d_pixels, int B, const mcl_intrinsics* K,
                                  int level, const mcl_opts* o, const mcl_train_cfg* cfg,
                                  float* d_loss_log, void* stream) {
    g_err[0] = 0;
    if (!m || !d_poses || !d_pixels || !K || !o || !cfg || n_poses < 1 || B < 1)
        return fail(MCL_ERR_ARG, "mcl_proposal_train: bad argument");
    if (cfg->epochs < 1 || cfg->batch_rays < 1 || cfg->n_bins < 2 || cfg->n_bins > kMaxCoarse ||
        !(cfg->lr > 0.f) || !(cfg->beta1 >= 0.f && cfg->beta1 < 1.f) ||
        !(cfg->beta2 >= 0.f && cfg->beta2 < 1.f) || !(cfg->eps > 0.f))
        return fail(MCL_ERR_ARG, "mcl_proposal_train: bad training configuration");
    if (B > m->cfg.max_rays) return fail(MCL_ERR_ARG, "mcl_proposal_train: B > max_rays");
    if (!m->has_proposal) return fail(MCL_ERR_ARG, "mcl_proposal_train: set initial proposal weights first");
    return proposal_train(m, d_poses, n_poses, d_pixels, B, *K, level, *o, *cfg, d_loss_log,
                          (cudaStream_t)stream, render_full);
}
