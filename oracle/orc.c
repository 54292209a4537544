/*
 * orc.c -- plain FP64 CPU oracle of the Fast Loc-NeRF particle-weight update
 * (Kong, Lee, Lee, Kim, "Fast Global Localization on Neural Radiance Field",
 * arXiv 2406.12202).
 *
 * TEST INFRASTRUCTURE.  This file is the slow, obviously correct statement of
 * what the GPU library must compute.  Only the test-suite, the smoke check and
 * the CPU-baseline leg of the benchmark may load it.  It shares no code,
 * header, table or helper with the CUDA library, and the library never calls
 * it.
 *
 * Everything is computed in double precision with plain loops, in the order
 * the paper states the method:
 *   Sec. III-A, Eq. 1   volume rendering by a sampled Riemann sum
 *   Sec. III-A, Eq. 3/4 particle set and the Loc-NeRF likelihood
 *   Sec. III-B, Eq. 5   transparent / opaque points of a ray
 *   Sec. III-B, Eq. 6   rejection weight with F = max(z_opaque - z_trans, tau)
 *   Sec. III-C, Alg. 1  downscale, render, weight, normalise, resample
 * together with the parts of the "basic NeRF model" (Sec. IV-A) that the paper
 * takes as given: positional encoding, the MLP, hierarchical (importance)
 * sampling.  The readings taken where the paper is silent are listed at each
 * function.
 *
 * OpenMP is used only to run independent rays side by side; every ray is
 * evaluated exactly as the single-threaded loop would evaluate it.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_MAX_LAYERS 16
#define ORC_MAX_WIDTH 512

/* ------------------------------------------------------------------------ */
/* Architecture: arch[6] = {L_xyz, L_dir, depth, width, skip, rgb_width}.    */
/* Blob order: trunk1..trunk_depth, sigma, feature, rgb_hidden, rgb_out.     */
/* Each layer is W[out][in] (row-major) followed by b[out].                  */
/* Trunk layer skip+1 reads [h_skip, gamma(x)]; rgb_hidden reads             */
/* [feature, gamma(d)].                                                      */
/* ------------------------------------------------------------------------ */
static int layer_table(const int* a, int* fin, int* fout) {
    int gx = 3 + 6 * a[0], gd = 3 + 6 * a[1];
    int D = a[2], W = a[3], skip = a[4], Wr = a[5];
    int n = 0;
    if (D < 1 || D + 4 > ORC_MAX_LAYERS || W < 1 || W > ORC_MAX_WIDTH ||
        Wr < 1 || Wr > ORC_MAX_WIDTH || skip < 1 || skip >= D)
        return -1;
    for (int l = 1; l <= D; ++l) {
        fin[n] = (l == 1) ? gx : (l == skip + 1 ? W + gx : W);
        fout[n] = W;
        ++n;
    }
    fin[n] = W;      fout[n] = 1;  ++n;   /* sigma head            */
    fin[n] = W;      fout[n] = W;  ++n;   /* feature (linear)      */
    fin[n] = W + gd; fout[n] = Wr; ++n;   /* rgb hidden (ReLU)     */
    fin[n] = Wr;     fout[n] = 3;  ++n;   /* rgb out (sigmoid)     */
    return n;
}

long orc_n_weights(const int* arch) {
    int fin[ORC_MAX_LAYERS], fout[ORC_MAX_LAYERS];
    int n = layer_table(arch, fin, fout);
    if (n < 0) return -1;
    long tot = 0;
    for (int i = 0; i < n; ++i) tot += (long)fin[i] * fout[i] + fout[i];
    return tot;
}

/* ------------------------------------------------------------------------ */
/* Positional encoding of the basic NeRF model:                              */
/*   gamma(p) = [p, sin(2^0 p), cos(2^0 p), ..., sin(2^(L-1) p), cos(...)]   */
/* where each sin / cos acts on the 3-vector p (3 + 6L outputs).             */
/* Reading: frequencies 2^k without a factor pi, identity term included.     */
/* ------------------------------------------------------------------------ */
void orc_pe(const double* p, int L, double* out) {
    out[0] = p[0]; out[1] = p[1]; out[2] = p[2];
    for (int k = 0; k < L; ++k) {
        double f = ldexp(1.0, k);
        for (int c = 0; c < 3; ++c) {
            out[3 + 6 * k + c] = sin(f * p[c]);
            out[3 + 6 * k + 3 + c] = cos(f * p[c]);
        }
    }
}

/* y = W x + b, optionally followed by ReLU (max(., 0)). */
static void dense(const double* W, const double* b, int fin, int fout,
                  const double* x, double* y, int relu) {
    for (int o = 0; o < fout; ++o) {
        double s = b[o];
        const double* w = W + (long)o * fin;
        for (int i = 0; i < fin; ++i) s += w[i] * x[i];
        y[o] = (relu && s < 0.0) ? 0.0 : s;
    }
}

/* The NeRF MLP F(x, d) -> (c, sigma) (Sec. III-A, "Neural Radiance Fields").
 * Returns the raw density (before the ReLU that compositing applies) and the
 * sigmoid RGB.  wd is the blob widened to double. */
static int mlp_eval(const double* wd, const int* arch, const double* x,
                    const double* dhat, double* sigma_raw, double* rgb) {
    int fin[ORC_MAX_LAYERS], fout[ORC_MAX_LAYERS];
    int n = layer_table(arch, fin, fout);
    if (n < 0) return -1;
    int D = arch[2], W = arch[3], skip = arch[4];
    int gxn = 3 + 6 * arch[0], gdn = 3 + 6 * arch[1];
    double gx[3 + 6 * 64], gd[3 + 6 * 64];
    double h[ORC_MAX_WIDTH + 3 + 6 * 64], t[ORC_MAX_WIDTH + 3 + 6 * 64];
    if (arch[0] > 64 || arch[1] > 64) return -1;
    orc_pe(x, arch[0], gx);
    orc_pe(dhat, arch[1], gd);

    const double* p = wd;
    /* trunk layer 1 reads gamma(x) */
    memcpy(t, gx, sizeof(double) * gxn);
    for (int l = 0; l < D; ++l) {
        const double* Wl = p;
        const double* bl = p + (long)fin[l] * fout[l];
        dense(Wl, bl, fin[l], fout[l], t, h, 1);
        p = bl + fout[l];
        /* input of the next layer: h, with gamma(x) appended after layer skip */
        memcpy(t, h, sizeof(double) * W);
        if (l + 1 == skip) memcpy(t + W, gx, sizeof(double) * gxn);
    }
    /* sigma head on the trunk output */
    double s;
    dense(p, p + W, W, 1, t, &s, 0);
    p += W + 1;
    /* feature layer (linear) */
    double feat[ORC_MAX_WIDTH + 3 + 6 * 64];
    dense(p, p + (long)W * W, W, W, t, feat, 0);
    p += (long)W * W + W;
    /* rgb hidden reads [feature, gamma(d)] */
    memcpy(feat + W, gd, sizeof(double) * gdn);
    int Wr = arch[5];
    double hr[ORC_MAX_WIDTH];
    dense(p, p + (long)Wr * (W + gdn), W + gdn, Wr, feat, hr, 1);
    p += (long)Wr * (W + gdn) + Wr;
    double o3[3];
    dense(p, p + 3 * Wr, Wr, 3, hr, o3, 0);
    *sigma_raw = s;
    for (int c = 0; c < 3; ++c) rgb[c] = 1.0 / (1.0 + exp(-o3[c]));
    return 0;
}

static double* widen(const float* blob, long n) {
    double* wd = (double*)malloc(sizeof(double) * (size_t)n);
    if (!wd) return NULL;
    for (long i = 0; i < n; ++i) wd[i] = (double)blob[i];
    return wd;
}

/* Batch MLP evaluation (for pins): x, dhat [n,3] -> sigma_raw [n], rgb [n,3]. */
int orc_mlp(const float* blob, const int* arch, int n, const double* x,
            const double* dhat, double* sigma_raw, double* rgb) {
    long nw = orc_n_weights(arch);
    if (nw < 0) return -1;
    double* wd = widen(blob, nw);
    if (!wd) return -2;
    int err = 0;
#pragma omp parallel for schedule(static) reduction(| : err)
    for (int i = 0; i < n; ++i)
        err |= mlp_eval(wd, arch, x + 3 * i, dhat + 3 * i, sigma_raw + i, rgb + 3 * i);
    free(wd);
    return err ? -1 : 0;
}

/* ------------------------------------------------------------------------ */
/* Ray through the centre of pixel (u, v) for camera-to-world pose P (row-   */
/* major 3x4 [R | t]).  Camera looks along -z with +y up (NeRF convention):  */
/*   d_cam = ((u + 1/2 - cx)/fx, -(v + 1/2 - cy)/fy, -1),  d = R d_cam,      */
/*   o = t.  d is not normalised; points are x = o + z d.                    */
/* ------------------------------------------------------------------------ */
void orc_ray(const double* P, double fx, double fy, double cx, double cy,
             double u, double v, double* o, double* d) {
    double dc[3] = {(u + 0.5 - cx) / fx, -(v + 0.5 - cy) / fy, -1.0};
    for (int r = 0; r < 3; ++r) {
        d[r] = P[4 * r + 0] * dc[0] + P[4 * r + 1] * dc[1] + P[4 * r + 2] * dc[2];
        o[r] = P[4 * r + 3];
    }
}

/* ------------------------------------------------------------------------ */
/* Eq. 1 by the Riemann sum of the basic NeRF model, on sorted samples z:    */
/*   delta_k = (z_{k+1} - z_k) |d|,  delta_last = 1e10,                      */
/*   alpha_k = 1 - exp(-max(sigma_k, 0) delta_k),                            */
/*   T_k = prod_{m<k} (1 - alpha_m),  w_k = T_k alpha_k,  C = sum_k w_k c_k. */
/* No background colour.                                                     */
/* ------------------------------------------------------------------------ */
void orc_composite(int n, const double* z, const double* sigma_raw,
                   const double* rgb, double dnorm, double* w, double* T,
                   double* C) {
    double trans = 1.0;
    C[0] = C[1] = C[2] = 0.0;
    for (int k = 0; k < n; ++k) {
        double delta = (k < n - 1) ? (z[k + 1] - z[k]) * dnorm : 1e10;
        double s = sigma_raw[k] > 0.0 ? sigma_raw[k] : 0.0;
        double a = 1.0 - exp(-s * delta);
        if (T) T[k] = trans;
        w[k] = trans * a;
        for (int c = 0; c < 3; ++c) C[c] += w[k] * rgb[3 * k + c];
        trans *= (1.0 - a);
    }
}

/* ------------------------------------------------------------------------ */
/* Hierarchical sampling of the basic NeRF model (inverse transform):        */
/* bin edges are the midpoints of consecutive coarse samples; the pdf over   */
/* the interior bins is proportional to the interior coarse weights plus     */
/* 1e-5; for each u the first CDF entry strictly greater than u selects the  */
/* bin, and z is linearly interpolated inside it.                            */
/* ------------------------------------------------------------------------ */
void orc_sample_pdf(int n_c, const double* z_c, const double* w_c, int n_f,
                    const double* u, double* z_f) {
    int ne = n_c - 1;             /* number of edges   */
    int nb = n_c - 2;             /* number of bins    */
    double* edge = (double*)malloc(sizeof(double) * (size_t)(ne > 0 ? ne : 1));
    double* pdf = (double*)malloc(sizeof(double) * (size_t)(nb > 0 ? nb : 1));
    double* cdf = (double*)malloc(sizeof(double) * (size_t)(ne > 0 ? ne : 1));
    for (int i = 0; i < ne; ++i) edge[i] = 0.5 * (z_c[i] + z_c[i + 1]);
    double tot = 0.0;
    for (int i = 0; i < nb; ++i) { pdf[i] = w_c[i + 1] + 1e-5; tot += pdf[i]; }
    for (int i = 0; i < nb; ++i) pdf[i] /= tot;
    cdf[0] = 0.0;
    for (int i = 0; i < nb; ++i) cdf[i + 1] = cdf[i] + pdf[i];
    for (int j = 0; j < n_f; ++j) {
        int idx = 0;
        while (idx < ne && cdf[idx] <= u[j]) ++idx;
        int below = idx - 1 < 0 ? 0 : idx - 1;
        int above = idx > ne - 1 ? ne - 1 : idx;
        double denom = cdf[above] - cdf[below];
        if (denom < 1e-5) denom = 1.0;
        double t = (u[j] - cdf[below]) / denom;
        z_f[j] = edge[below] + t * (edge[above] - edge[below]);
    }
    free(edge); free(pdf); free(cdf);
}

/* ------------------------------------------------------------------------ */
/* Eq. 5 on discrete samples, and F of Eq. 6.  W_k = sum_{m<=k} w_m.         */
/*   z_trans  = z_k for the smallest k with W_k >= alpha (else z_0);         */
/*   z_opaque = z_k for the largest  k with W_k <= 1 - alpha (else z_0);     */
/*   F = max(z_opaque - z_trans, tau).                                       */
/* tie: how far the running sum is from flipping either decision, i.e. the   */
/* distance to alpha of W at the chosen k_trans and at k_trans - 1, and the  */
/* distance to 1 - alpha of W at k_opaque and k_opaque + 1; step: the widest */
/* sample spacing next to either decision (how far z_trans or z_opaque move  */
/* if a decision flips by one sample).  Both are reported for parity tests   */
/* and are not part of the method.                                           */
/* ------------------------------------------------------------------------ */
void orc_uncertainty(int n, const double* z, const double* w, double alpha,
                     double tau, double* z_trans, double* z_opaque, double* F,
                     double* tie, double* step) {
    double Wc = 0.0;
    int kt = -1, ko = -1;
    double* W = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    for (int k = 0; k < n; ++k) {
        Wc += w[k];
        W[k] = Wc;
        if (kt < 0 && Wc >= alpha) kt = k;
        if (Wc <= 1.0 - alpha) ko = k;
    }
    *z_trans = kt >= 0 ? z[kt] : z[0];
    *z_opaque = ko >= 0 ? z[ko] : z[0];
    double g = *z_opaque - *z_trans;
    *F = g > tau ? g : tau;
    if (tie) {
        double m = INFINITY, d;
        if (kt >= 0) {
            d = W[kt] - alpha; if (d < m) m = d;
            d = alpha - (kt > 0 ? W[kt - 1] : 0.0); if (d < m) m = d;
        } else if (n > 0) {
            d = alpha - W[n - 1]; if (d < m) m = d;
        }
        if (ko >= 0) {
            d = (1.0 - alpha) - W[ko]; if (d < m) m = d;
            if (ko + 1 < n) { d = W[ko + 1] - (1.0 - alpha); if (d < m) m = d; }
        } else if (n > 0) {
            d = W[0] - (1.0 - alpha); if (d < m) m = d;
        }
        *tie = m;
    }
    if (step) {
        double st = 0.0;
        int ks[2] = {kt >= 0 ? kt : 0, ko >= 0 ? ko : 0};
        for (int i = 0; i < 2; ++i) {
            int k = ks[i];
            if (k > 0 && z[k] - z[k - 1] > st) st = z[k] - z[k - 1];
            if (k + 1 < n && z[k + 1] - z[k] > st) st = z[k + 1] - z[k];
        }
        *step = st;
    }
    free(W);
}

/* Options of one update (mirrored by a ctypes Structure in oracle/__init__). */
typedef struct {
    double near_z, far_z, alpha, tau, rho, s_min;
    int n_coarse, n_fine, use_rejection, pad;
} orc_opts;

/* Render one ray: coarse stratified samples, MLP, composite, importance
 * samples from the coarse weights, MLP on the new samples only (the same MLP
 * serves both passes, so the coarse outputs are reused), stable merge by z,
 * composite, Eq. 5 / F.  uj: n_coarse jitter uniforms or NULL (midpoints).
 * out[0..2] rgb, out[3] z_trans, out[4] z_opaque, out[5] F, out[6] tie,
 * out[7] raw density of the last sample, out[8] transmittance before it
 * (the last interval is 1e10 long, so the colour jumps by about
 * out[8] * c_last when that density crosses 0), out[9] decision step (see
 * orc_uncertainty); out[6..9] are reported for parity tests. */
static int render_ray(const double* wd, const int* arch, const double* o,
                      const double* d, const orc_opts* op, const double* uj,
                      double* out, double* z_dbg, double* w_dbg) {
    int nc = op->n_coarse, nf = op->n_fine, n = nc + nf;
    double dn = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    double dh[3] = {d[0] / dn, d[1] / dn, d[2] / dn};
    double* z = (double*)malloc(sizeof(double) * (size_t)n);
    double* sg = (double*)malloc(sizeof(double) * (size_t)n);
    double* cl = (double*)malloc(sizeof(double) * 3 * (size_t)n);
    double* w = (double*)malloc(sizeof(double) * (size_t)n);
    double* uf = (double*)malloc(sizeof(double) * (size_t)(nf > 0 ? nf : 1));
    int* ord = (int*)malloc(sizeof(int) * (size_t)n);
    double* zs = (double*)malloc(sizeof(double) * (size_t)n);
    double* ss = (double*)malloc(sizeof(double) * (size_t)n);
    double* cs = (double*)malloc(sizeof(double) * 3 * (size_t)n);
    int err = 0;
    /* coarse: z_k = near + (far - near) (k + u_k) / n_c */
    for (int k = 0; k < nc; ++k) {
        double uk = uj ? uj[k] : 0.5;
        z[k] = op->near_z + (op->far_z - op->near_z) * (k + uk) / nc;
    }
    for (int k = 0; k < nc; ++k) {
        double x[3] = {o[0] + z[k] * d[0], o[1] + z[k] * d[1], o[2] + z[k] * d[2]};
        err |= mlp_eval(wd, arch, x, dh, sg + k, cl + 3 * k);
    }
    double C[3];
    if (nf > 0) {
        orc_composite(nc, z, sg, cl, dn, w, NULL, C);
        for (int j = 0; j < nf; ++j) uf[j] = nf > 1 ? (double)j / (nf - 1) : 0.0;
        orc_sample_pdf(nc, z, w, nf, uf, z + nc);
        for (int k = nc; k < n; ++k) {
            double x[3] = {o[0] + z[k] * d[0], o[1] + z[k] * d[1], o[2] + z[k] * d[2]};
            err |= mlp_eval(wd, arch, x, dh, sg + k, cl + 3 * k);
        }
    }
    /* stable sort of all samples by z (insertion sort: equal z keep their
       order, coarse before fine) */
    for (int k = 0; k < n; ++k) ord[k] = k;
    for (int k = 1; k < n; ++k) {
        int v = ord[k], m = k - 1;
        while (m >= 0 && z[ord[m]] > z[v]) { ord[m + 1] = ord[m]; --m; }
        ord[m + 1] = v;
    }
    for (int k = 0; k < n; ++k) {
        zs[k] = z[ord[k]];
        ss[k] = sg[ord[k]];
        for (int c = 0; c < 3; ++c) cs[3 * k + c] = cl[3 * ord[k] + c];
    }
    double* Tk = (double*)malloc(sizeof(double) * (size_t)n);
    orc_composite(n, zs, ss, cs, dn, w, Tk, C);
    out[0] = C[0]; out[1] = C[1]; out[2] = C[2];
    orc_uncertainty(n, zs, w, op->alpha, op->tau, out + 3, out + 4, out + 5, out + 6, out + 9);
    out[7] = ss[n - 1];
    out[8] = Tk[n - 1];
    free(Tk);
    if (z_dbg) memcpy(z_dbg, zs, sizeof(double) * (size_t)n);
    if (w_dbg) memcpy(w_dbg, w, sizeof(double) * (size_t)n);
    free(z); free(sg); free(cl); free(w); free(uf); free(ord);
    free(zs); free(ss); free(cs);
    return err;
}

/* Render arbitrary rays (for pins and for oracle-rendered observations).
 * o, d: [n,3].  uj: [n, n_coarse] or NULL.  out: [n,10] as render_ray.
 * z_dbg, w_dbg: [n, n_coarse + n_fine] or NULL. */
int orc_render_rays(const float* blob, const int* arch, int n, const double* o,
                    const double* d, const orc_opts* op, const double* uj,
                    double* out, double* z_dbg, double* w_dbg) {
    long nw = orc_n_weights(arch);
    if (nw < 0 || op->n_coarse < 2 || op->n_fine < 0) return -1;
    double* wd = widen(blob, nw);
    if (!wd) return -2;
    int ns = op->n_coarse + op->n_fine, err = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : err)
    for (int r = 0; r < n; ++r)
        err |= render_ray(wd, arch, o + 3 * r, d + 3 * r, op,
                          uj ? uj + (long)r * op->n_coarse : NULL, out + 10 * r,
                          z_dbg ? z_dbg + (long)r * ns : NULL,
                          w_dbg ? w_dbg + (long)r * ns : NULL);
    free(wd);
    return err ? -1 : 0;
}

/* ------------------------------------------------------------------------ */
/* downscale(I_t, R_t) of Alg. 1: box average over factor x factor blocks    */
/* (reading: the paper does not name the filter).  img [H,W,3] -> out        */
/* [H/f, W/f, 3].                                                            */
/* ------------------------------------------------------------------------ */
int orc_downscale(const double* img, int W, int H, int f, double* out) {
    if (f < 1 || W % f || H % f) return -1;
    int Wl = W / f, Hl = H / f;
    for (int v = 0; v < Hl; ++v)
        for (int u = 0; u < Wl; ++u)
            for (int c = 0; c < 3; ++c) {
                double s = 0.0;
                for (int dy = 0; dy < f; ++dy)
                    for (int dx = 0; dx < f; ++dx)
                        s += img[((long)(v * f + dy) * W + (u * f + dx)) * 3 + c];
                out[((long)v * Wl + u) * 3 + c] = s / (f * f);
            }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* One weight update (Alg. 1, inner loop over particles, with Eq. 6):        */
/*   I^R = downscale(I, R), K^R = R K (focal and centre divided by factor);  */
/*   for particle i and query pixel p_j (shared by all particles):           */
/*     C_ij = render(r(p_j, x_i), K^R);                                      */
/*     E_ij = sum_c (I^R(p_j)_c - C_ij,c)^2   (Eq. 6 read with exponent 2);  */
/*     F_ij = max(z_opaque - z_trans, tau)   (F = 1 without rejection, Eq.4);*/
/*   S_i = sum_j E_ij F_ij,                                                  */
/*   log w_i = 4 (log B - log max(S_i, s_min))   (Eq. 6 in logs),            */
/*   w_i = exp(log w_i - logsumexp_k log w_k)   (weights normalised to 1),   */
/*   mask_i = (w_i >= rho / N).                                              */
/* particles [N,12]; image [H,W,3] full resolution; K4 = {fx, fy, cx, cy}    */
/* at full resolution; pixels [B,2] (u, v) in the level image; uj           */
/* [N*B, n_coarse] or NULL.  Per-ray outputs are [N*B] in (i, j) order.      */
/* ------------------------------------------------------------------------ */
int orc_update(const float* blob, const int* arch, const double* particles,
               int N, const double* image, int W, int H, const double* K4,
               int factor, const int32_t* pixels, int B, const orc_opts* op,
               const double* uj, double* rgb, double* E, double* Fr,
               double* zt, double* zo, double* tie, double* sig_last,
               double* t_last, double* step, double* S, double* logw, double* w,
               uint8_t* mask) {
    if (N < 1 || B < 1 || factor < 1 || W % factor || H % factor) return -1;
    long nw = orc_n_weights(arch);
    if (nw < 0) return -1;
    int Wl = W / factor, Hl = H / factor;
    for (int j = 0; j < B; ++j)
        if (pixels[2 * j] < 0 || pixels[2 * j] >= Wl || pixels[2 * j + 1] < 0 ||
            pixels[2 * j + 1] >= Hl)
            return -1;
    double* lvl = (double*)malloc(sizeof(double) * 3 * (size_t)Wl * Hl);
    double* wd = widen(blob, nw);
    double* ef = (double*)malloc(sizeof(double) * (size_t)N * B);
    if (!lvl || !wd || !ef) { free(lvl); free(wd); free(ef); return -2; }
    orc_downscale(image, W, H, factor, lvl);
    double fx = K4[0] / factor, fy = K4[1] / factor;
    double cx = K4[2] / factor, cy = K4[3] / factor;
    int err = 0;
    long nr = (long)N * B;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : err)
    for (long r = 0; r < nr; ++r) {
        int i = (int)(r / B), j = (int)(r % B);
        double o[3], d[3], out[10];
        orc_ray(particles + 12 * (long)i, fx, fy, cx, cy, pixels[2 * j],
                pixels[2 * j + 1], o, d);
        err |= render_ray(wd, arch, o, d, op,
                          uj ? uj + r * op->n_coarse : NULL, out, NULL, NULL);
        const double* obs = lvl + ((long)pixels[2 * j + 1] * Wl + pixels[2 * j]) * 3;
        double e = 0.0;
        for (int c = 0; c < 3; ++c) {
            double df = obs[c] - out[c];
            e += df * df;
            if (rgb) rgb[3 * r + c] = out[c];
        }
        double f = op->use_rejection ? out[5] : 1.0;
        ef[r] = e * f;
        if (E) E[r] = e;
        if (zt) zt[r] = out[3];
        if (zo) zo[r] = out[4];
        if (Fr) Fr[r] = f;
        if (tie) tie[r] = out[6];
        if (sig_last) sig_last[r] = out[7];
        if (t_last) t_last[r] = out[8];
        if (step) step[r] = out[9];
    }
    /* per-particle sums and log weights */
    double mx = -INFINITY;
    for (int i = 0; i < N; ++i) {
        double s = 0.0;
        for (int j = 0; j < B; ++j) s += ef[(long)i * B + j];
        S[i] = s;
        if (isfinite(s)) {
            double sc = s > op->s_min ? s : op->s_min;
            logw[i] = 4.0 * (log((double)B) - log(sc));
        } else {
            /* a particle whose loss is not a number carries no weight */
            logw[i] = -INFINITY;
        }
        if (logw[i] > mx) mx = logw[i];
    }
    double acc = 0.0;
    if (mx > -INFINITY)
        for (int i = 0; i < N; ++i) acc += exp(logw[i] - mx);
    double lse = mx + log(acc);
    for (int i = 0; i < N; ++i) {
        w[i] = mx > -INFINITY ? exp(logw[i] - lse) : 0.0;
        mask[i] = (uint8_t)(w[i] >= op->rho / N && w[i] > 0.0);
    }
    free(lvl); free(wd); free(ef);
    return err ? -1 : 0;
}

/* ------------------------------------------------------------------------ */
/* Systematic resampling (Alg. 1: draw i with probability proportional to   */
/* w_i) on an exact integer CDF:                                             */
/*   e: max w = m 2^e with m in [1/2, 1);  s = 50 - e - ceil(log2 N_in);     */
/*   q_i = floor(w_i 2^s) (exact), C_i = q_0 + ... + q_i, T = C_{N_in-1};    */
/*   U = floor(u0 2^53);                                                     */
/*   idx_k = smallest i with C_i N_out 2^53 > (k 2^53 + U) T  (128-bit).     */
/* This is the systematic rule "smallest i with CDF_i > (k + u0)/N_out"     */
/* evaluated without rounding.  Returns -1 for bad arguments or T = 0.       */
/* ------------------------------------------------------------------------ */
int orc_resample(const double* w, int n_in, int n_out, double u0, int32_t* idx) {
    if (n_in < 1 || n_out < 1 || n_out > 65536 || !(u0 >= 0.0 && u0 < 1.0))
        return -1;
    double mx = 0.0;
    for (int i = 0; i < n_in; ++i) {
        if (!(w[i] >= 0.0) || isinf(w[i])) return -1;
        if (w[i] > mx) mx = w[i];
    }
    if (mx <= 0.0) return -1;
    int e;
    frexp(mx, &e);
    int lg = 0;
    while ((1L << lg) < n_in) ++lg;
    int sh = 50 - e - lg;
    uint64_t* C = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)n_in);
    if (!C) return -2;
    uint64_t run = 0;
    for (int i = 0; i < n_in; ++i) {
        run += (uint64_t)floor(ldexp(w[i], sh));
        C[i] = run;
    }
    uint64_t T = run;
    if (T == 0) { free(C); return -1; }
    uint64_t U = (uint64_t)floor(ldexp(u0, 53));
    for (int k = 0; k < n_out; ++k) {
        /* (k 2^53 + U) needs up to 69 bits: form it in 128 bits */
        unsigned __int128 rhs =
            ((((unsigned __int128)(uint64_t)k) << 53) + U) * (unsigned __int128)T;
        int found = n_in - 1;
        for (int i = 0; i < n_in; ++i) {
            unsigned __int128 lhs =
                ((unsigned __int128)C[i] * (uint64_t)n_out) << 53;
            if (lhs > rhs) { found = i; break; }
        }
        idx[k] = found;
    }
    free(C);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Counter-based random numbers: SplitMix64 (Steele, Lea, Flood, OOPSLA      */
/* 2014).  The generator adds gamma = 0x9E3779B97F4A7C15 to its state and    */
/* returns mix(state).  Stream (seed, ctr): initial state                    */
/*   s0 = seed XOR mix(ctr + gamma);  value idx = mix(s0 + (idx + 1) gamma). */
/* ------------------------------------------------------------------------ */
static uint64_t sm_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

uint64_t orc_splitmix64_next(uint64_t* state) {
    *state += 0x9E3779B97F4A7C15ULL;
    return sm_mix(*state);
}

uint64_t orc_cbrng(uint64_t seed, uint64_t ctr, uint64_t idx) {
    uint64_t s0 = seed ^ sm_mix(ctr + 0x9E3779B97F4A7C15ULL);
    return sm_mix(s0 + (idx + 1) * 0x9E3779B97F4A7C15ULL);
}

/* uniform in [0, 1) with 53 random bits */
double orc_uniform(uint64_t seed, uint64_t ctr, uint64_t idx) {
    return (double)(orc_cbrng(seed, ctr, idx) >> 11) * 0x1.0p-53;
}

/* standard normal number m of stream (seed, ctr): Box-Muller on the
 * uniforms 2m (shifted into (0, 1]) and 2m + 1. */
double orc_normal(uint64_t seed, uint64_t ctr, uint64_t m) {
    double u1 = ((double)(orc_cbrng(seed, ctr, 2 * m) >> 11) + 1.0) * 0x1.0p-53;
    double u2 = orc_uniform(seed, ctr, 2 * m + 1);
    return sqrt(-2.0 * log(u1)) * cos(2.0 * M_PI * u2);
}

/* ------------------------------------------------------------------------ */
/* Query pixel set {p_j} of one update (Alg. 1; Eq. 4 and Eq. 6 index p_j    */
/* without a particle index, so one set serves every particle): B distinct  */
/* pixels of a W x H level image, uniformly without replacement, by Floyd's  */
/* sampling algorithm (Bentley & Floyd, CACM 1987): for j = n-B .. n-1 draw  */
/* t uniform in [0, j]; take t unless already taken, else take j.  The       */
/* uniform integer is floor(r (j + 1) / 2^64) with r = value j-(n-B) of      */
/* SplitMix64 stream (seed, ctr).  Pixel index q -> (u, v) = (q % W, q / W). */
/* ------------------------------------------------------------------------ */
int orc_pixel_set(int W, int H, int B, uint64_t seed, uint64_t ctr, int32_t* out) {
    long n = (long)W * H;
    if (W < 1 || H < 1 || B < 1 || B > n) return -1;
    long* chosen = (long*)malloc(sizeof(long) * (size_t)B);
    if (!chosen) return -2;
    int m = 0;
    for (long j = n - B; j < n; ++j) {
        uint64_t r = orc_cbrng(seed, ctr, (uint64_t)(j - (n - B)));
        long t = (long)(((unsigned __int128)r * (unsigned __int128)(uint64_t)(j + 1)) >> 64);
        int dup = 0;
        for (int i = 0; i < m; ++i)
            if (chosen[i] == t) { dup = 1; break; }
        chosen[m++] = dup ? j : t;
    }
    for (int i = 0; i < B; ++i) {
        out[2 * i] = (int32_t)(chosen[i] % W);
        out[2 * i + 1] = (int32_t)(chosen[i] / W);
    }
    free(chosen);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Prediction step (Sec. III-A): x_t = x_{t-1} O_t Exp(delta), O_t = I for   */
/* global localisation.  delta = (rho, omega) in se(3); the SE(3)            */
/* exponential is R = Rodrigues(omega), t = V rho with                       */
/*   V = I + (1 - cos th)/th^2 [w]x + (th - sin th)/th^3 [w]x^2.             */
/* ------------------------------------------------------------------------ */
void orc_se3_exp(const double* rho, const double* om, double* M /*3x4*/) {
    double th2 = om[0] * om[0] + om[1] * om[1] + om[2] * om[2];
    double th = sqrt(th2);
    double K[9] = {0, -om[2], om[1], om[2], 0, -om[0], -om[1], om[0], 0};
    double K2[9];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            double s = 0.0;
            for (int m = 0; m < 3; ++m) s += K[3 * r + m] * K[3 * m + c];
            K2[3 * r + c] = s;
        }
    double a, b, cc;
    if (th < 1e-8) {
        a = 1.0; b = 0.5; cc = 1.0 / 6.0;
    } else {
        a = sin(th) / th;
        b = (1.0 - cos(th)) / th2;
        cc = (th - sin(th)) / (th2 * th);
    }
    double R[9], V[9];
    for (int i = 0; i < 9; ++i) {
        double I = (i % 4 == 0) ? 1.0 : 0.0;
        R[i] = I + a * K[i] + b * K2[i];
        V[i] = I + b * K[i] + cc * K2[i];
    }
    for (int r = 0; r < 3; ++r) {
        for (int c = 0; c < 3; ++c) M[4 * r + c] = R[3 * r + c];
        M[4 * r + 3] = V[3 * r + 0] * rho[0] + V[3 * r + 1] * rho[1] + V[3 * r + 2] * rho[2];
    }
}

/* out = pose * Exp(rho, (0, yaw, 0)) for n poses [n,12]; noise [n,4] =
 * (rho_x, rho_y, rho_z, yaw) in the body frame. */
/* Prediction with odometry (Sec. III-A motion model x_t = x_{t-1} O_t
 * Exp(delta)): odom is the 3x4 relative motion O_t, or NULL for O_t = I. */
void orc_predict_odom(int n, const double* pose, const double* odom, const double* noise,
                      double* out) {
    for (int i = 0; i < n; ++i) {
        const double* P0 = pose + 12 * (long)i;
        double PO[12];
        if (odom) {
            for (int r = 0; r < 3; ++r)
                for (int c = 0; c < 4; ++c) {
                    double s = (c == 3) ? P0[4 * r + 3] : 0.0;
                    for (int m = 0; m < 3; ++m) s += P0[4 * r + m] * odom[4 * m + c];
                    PO[4 * r + c] = s;
                }
        } else {
            for (int k = 0; k < 12; ++k) PO[k] = P0[k];
        }
        const double* P = PO;
        const double* q = noise + 4 * (long)i;
        double om[3] = {0.0, q[3], 0.0}, E[12];
        orc_se3_exp(q, om, E);
        double* O = out + 12 * (long)i;
        for (int r = 0; r < 3; ++r) {
            for (int c = 0; c < 4; ++c) {
                double s = 0.0;
                for (int m = 0; m < 3; ++m) s += P[4 * r + m] * E[4 * m + c];
                if (c == 3) s += P[4 * r + 3];
                O[4 * r + c] = s;
            }
        }
    }
}

void orc_predict(int n, const double* pose, const double* noise, double* out) {
    orc_predict_odom(n, pose, NULL, noise, out);
}

/* Motion noise of particle k drawn from stream (seed, ctr): normals 4k..4k+3
 * scaled by (sigma_t, sigma_t, sigma_t, sigma_yaw). */
void orc_motion_noise(int n, uint64_t seed, uint64_t ctr, double sigma_t,
                      double sigma_yaw, double* noise) {
    for (int k = 0; k < n; ++k)
        for (int c = 0; c < 4; ++c)
            noise[4 * (long)k + c] = (c < 3 ? sigma_t : sigma_yaw) *
                                     orc_normal(seed, ctr, 4 * (uint64_t)k + c);
}

/* ------------------------------------------------------------------------ */
/* Refinement test of the coarse-to-fine schedule (Sec. III-C, "Detailed     */
/* Structure"): Var({x_t}) read as the trace of the population covariance of */
/* the particle positions.  out[0..2] mean, out[3] trace.                    */
/* ------------------------------------------------------------------------ */
void orc_position_spread(int n, const double* pose, double* out) {
    double m[3] = {0, 0, 0};
    for (int i = 0; i < n; ++i)
        for (int c = 0; c < 3; ++c) m[c] += pose[12 * (long)i + 4 * c + 3];
    for (int c = 0; c < 3; ++c) m[c] /= n;
    double tr = 0.0;
    for (int i = 0; i < n; ++i)
        for (int c = 0; c < 3; ++c) {
            double dd = pose[12 * (long)i + 4 * c + 3] - m[c];
            tr += dd * dd;
        }
    out[0] = m[0]; out[1] = m[1]; out[2] = m[2];
    out[3] = tr / n;
}

/* ------------------------------------------------------------------------ */
/* Statistics of one weighted particle set, as the coarse-to-fine loop uses */
/* them after the weights of an iteration (Sec. III-C, "Detailed            */
/* Structure"; Alg. 1).  The paper's refinement test compares Var({x_t})    */
/* with a threshold; the set it states it on is the resampled one, whose    */
/* expected spread is the weighted spread of the set before resampling.     */
/* This reading evaluates it on the weighted set (no resampling noise):     */
/*   mean      m = sum_i w_i t_i / sum_i w_i        (t_i = position of x_i) */
/*   spread    V = sum_i w_i |t_i - m|^2 / sum_i w_i                        */
/*   yaw       atan2(sum_i w_i sin(yaw_i), sum_i w_i cos(yaw_i)),           */
/*             yaw_i = atan2(R_i[0][2], R_i[0][0]) (rotation about +y)      */
/*   survivors n_s = number of particles with mask_i = 1                    */
/* out[0..2] = m, out[3] = yaw, out[4] = V, out[5] = n_s.  Particles with   */
/* w_i = 0 (or all weights zero: out[0..4] = NaN) take no part.             */
/* ------------------------------------------------------------------------ */
void orc_loop_statistics(int n, const double* pose, const double* w, const uint8_t* mask,
                         double* out) {
    double W = 0.0, m[3] = {0, 0, 0}, ys = 0.0, yc = 0.0;
    long ns = 0;
    for (int i = 0; i < n; ++i) {
        const double* p = pose + 12 * (long)i;
        if (mask[i]) ++ns;
        if (!(w[i] > 0.0)) continue;
        W += w[i];
        for (int c = 0; c < 3; ++c) m[c] += w[i] * p[4 * c + 3];
        double yaw = atan2(p[2], p[0]);
        ys += w[i] * sin(yaw);
        yc += w[i] * cos(yaw);
    }
    for (int c = 0; c < 3; ++c) m[c] /= W;
    double V = 0.0;
    for (int i = 0; i < n; ++i) {
        const double* p = pose + 12 * (long)i;
        if (!(w[i] > 0.0)) continue;
        for (int c = 0; c < 3; ++c) {
            double dd = p[4 * c + 3] - m[c];
            V += w[i] * dd * dd;
        }
    }
    out[0] = m[0]; out[1] = m[1]; out[2] = m[2];
    out[3] = atan2(ys, yc);
    out[4] = V / W;
    out[5] = (double)ns;
}

/* ------------------------------------------------------------------------ */
/* One step of the coarse-to-fine schedule (Sec. III-C): the paper moves to */
/* the next resolution level when Var({x_t}) falls below delta_refine; this */
/* reading also moves after a per-stage iteration cap, and sets the next    */
/* particle count from the survivors of the rejection weighting:            */
/*   refine  = stage < n_stages - 1 and (V < refine[stage] or               */
/*             iter_at_stage + 1 >= iter_cap[stage])                        */
/*   stage'  = stage + 1, iter' = 0   if refine                             */
/*             stage,     iter + 1    otherwise                             */
/*   N'      = min(max(n_s, n_min), n_cap[stage'], stride)                  */
/* state[0..2] = (stage, iter_at_stage, N) in, (stage', iter', N') out.     */
/* ------------------------------------------------------------------------ */
void orc_loop_schedule(int* state, int n_stages, const double* refine, const int* iter_cap,
                       const int* n_cap, int n_min, int stride, double V, int n_s) {
    int stage = state[0], it = state[1];
    if (stage < n_stages - 1 && (V < refine[stage] || it + 1 >= iter_cap[stage])) {
        stage += 1;
        it = 0;
    } else {
        it += 1;
    }
    int N = n_s;
    if (N < n_min) N = n_min;
    if (N > n_cap[stage]) N = n_cap[stage];
    if (N > stride) N = stride;
    state[0] = stage;
    state[1] = it;
    state[2] = N;
}

/* ======================================================================== */
/* Learned proposal sampler (not in the paper; a project extension that     */
/* replaces the coarse pass).  Network: gamma(x) with 6 frequencies (39     */
/* inputs) -> 4 ReLU layers of 64 units -> raw density s (linear head);     */
/* density = max(s, 0), composited over n_b stratified midpoints exactly as  */
/* Eq. 1 (delta_last = 1e10).  Blob: P1 W[64][39] b[64], P2..P4 W[64][64]    */
/* b[64], head w[64] b[1] (15105 floats).  Target: the full sampler's final  */
/* weights re-binned onto the same n_b equal intervals of [near, far] and    */
/* normalised (uniform when the ray carries no weight).  Loss of a ray:      */
/*   L = -sum_b h_b log(w_b / sum_k w_k + 1e-8).                             */
/* ======================================================================== */
#define PROP_L 6
#define PROP_IN (3 + 6 * PROP_L)
#define PROP_W 64
#define PROP_DEPTH 4

long orc_prop_n_weights(void) {
    return (long)PROP_W * PROP_IN + PROP_W + (PROP_DEPTH - 1) * ((long)PROP_W * PROP_W + PROP_W) +
           PROP_W + 1;
}

/* Forward of one point; a[l][j] pre-activations, h[l][j] = max(a, 0). */
static double prop_forward(const double* wd, const double* x, double* g,
                           double a[PROP_DEPTH][PROP_W], double h[PROP_DEPTH][PROP_W]) {
    orc_pe(x, PROP_L, g);
    const double* p = wd;
    const double* in = g;
    int fin = PROP_IN;
    for (int l = 0; l < PROP_DEPTH; ++l) {
        const double* W = p;
        const double* b = p + (long)PROP_W * fin;
        for (int o = 0; o < PROP_W; ++o) {
            double s = b[o];
            for (int i = 0; i < fin; ++i) s += W[(long)o * fin + i] * in[i];
            a[l][o] = s;
            h[l][o] = s > 0.0 ? s : 0.0;
        }
        p = b + PROP_W;
        in = h[l];
        fin = PROP_W;
    }
    double s = p[PROP_W];
    for (int i = 0; i < PROP_W; ++i) s += p[i] * h[PROP_DEPTH - 1][i];
    return s;
}

int orc_prop_forward(const float* blob, int n, const double* x, double* s_out) {
    long nw = orc_prop_n_weights();
    double* wd = widen(blob, nw);
    if (!wd) return -2;
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; ++i) {
        double g[PROP_IN], a[PROP_DEPTH][PROP_W], h[PROP_DEPTH][PROP_W];
        s_out[i] = prop_forward(wd, x + 3 * i, g, a, h);
    }
    free(wd);
    return 0;
}

/* Re-bin weights w of sorted samples z onto nb equal intervals of
 * [near, far] (interval floor((z - near) / (far - near) nb), clamped) and
 * normalise; a ray without weight gets the uniform histogram. */
void orc_histogram(int n, const double* z, const double* w, int nb, double near_z,
                   double far_z, double* hist) {
    for (int b = 0; b < nb; ++b) hist[b] = 0.0;
    for (int k = 0; k < n; ++k) {
        int b = (int)floor((z[k] - near_z) / (far_z - near_z) * nb);
        if (b < 0) b = 0;
        if (b > nb - 1) b = nb - 1;
        hist[b] += w[k];
    }
    double t = 0.0;
    for (int b = 0; b < nb; ++b) t += hist[b];
    for (int b = 0; b < nb; ++b) hist[b] = t > 0.0 ? hist[b] / t : 1.0 / nb;
}

/* Loss of one ray and (if grad != NULL) its gradient added to grad (blob
 * layout), by the chain rule: with g_k = dL/dw_k and w_k = T_k alpha_k,
 *   dL/dsigma_j = delta_j (g_j T_j (1 - alpha_j) - sum_{k>j} g_k w_k),
 * masked by s_j > 0, then back through the ReLU layers. */
static double prop_ray(const double* wd, const double* o, const double* d, int nb,
                       double near_z, double far_z, const double* hist, double* grad) {
    double dn = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    double* z = (double*)malloc(sizeof(double) * nb);
    double* sr = (double*)malloc(sizeof(double) * nb);
    double* al = (double*)malloc(sizeof(double) * nb);
    double* T = (double*)malloc(sizeof(double) * nb);
    double* w = (double*)malloc(sizeof(double) * nb);
    double* gw = (double*)malloc(sizeof(double) * nb);
    double* ds = (double*)malloc(sizeof(double) * nb);
    double (*A)[PROP_DEPTH][PROP_W] = malloc(sizeof(double) * nb * PROP_DEPTH * PROP_W);
    double (*Hh)[PROP_DEPTH][PROP_W] = malloc(sizeof(double) * nb * PROP_DEPTH * PROP_W);
    double (*G)[PROP_IN] = malloc(sizeof(double) * nb * PROP_IN);
    for (int k = 0; k < nb; ++k) {
        z[k] = near_z + (far_z - near_z) * (k + 0.5) / nb;
        double x[3] = {o[0] + z[k] * d[0], o[1] + z[k] * d[1], o[2] + z[k] * d[2]};
        sr[k] = prop_forward(wd, x, G[k], A[k], Hh[k]);
    }
    double trans = 1.0, W = 0.0;
    for (int k = 0; k < nb; ++k) {
        double delta = (k < nb - 1) ? (z[k + 1] - z[k]) * dn : 1e10;
        double sg = sr[k] > 0.0 ? sr[k] : 0.0;
        al[k] = 1.0 - exp(-sg * delta);
        T[k] = trans;
        w[k] = trans * al[k];
        trans *= (1.0 - al[k]);
        W += w[k];
    }
    double L = 0.0;
    if (!(W > 0.0)) {
        /* no density anywhere on the ray: every p_b = 1e-8, no gradient */
        for (int b = 0; b < nb; ++b) L -= hist[b] * log(1e-8);
    } else {
        for (int b = 0; b < nb; ++b) L -= hist[b] * log(w[b] / W + 1e-8);
    }
    if (grad && W > 0.0) {
        /* g_j = -h_j / (p_j W) + sum_b h_b w_b / (p_b W^2) */
        double c = 0.0;
        for (int b = 0; b < nb; ++b) c += hist[b] * w[b] / ((w[b] / W + 1e-8) * W * W);
        for (int j = 0; j < nb; ++j) gw[j] = -hist[j] / ((w[j] / W + 1e-8) * W) + c;
        double tail = 0.0; /* sum_{k>j} g_k w_k */
        for (int j = nb - 1; j >= 0; --j) {
            double delta = (j < nb - 1) ? (z[j + 1] - z[j]) * dn : 1e10;
            double dsig = delta * (gw[j] * T[j] * (1.0 - al[j]) - tail);
            ds[j] = sr[j] > 0.0 ? dsig : 0.0;
            tail += gw[j] * w[j];
        }
        /* back through the network, parameters in blob order */
        long off[PROP_DEPTH + 1];
        off[0] = 0;
        for (int l = 0; l < PROP_DEPTH; ++l)
            off[l + 1] = off[l] + (long)PROP_W * (l == 0 ? PROP_IN : PROP_W) + PROP_W;
        const double* head = wd + off[PROP_DEPTH];
        for (int k = 0; k < nb; ++k) {
            double dh[PROP_W], da[PROP_W];
            for (int i = 0; i < PROP_W; ++i) {
                grad[off[PROP_DEPTH] + i] += ds[k] * Hh[k][PROP_DEPTH - 1][i];
                dh[i] = ds[k] * head[i];
            }
            grad[off[PROP_DEPTH] + PROP_W] += ds[k];
            for (int l = PROP_DEPTH - 1; l >= 0; --l) {
                int fin = (l == 0) ? PROP_IN : PROP_W;
                const double* in = (l == 0) ? G[k] : Hh[k][l - 1];
                const double* Wl = wd + off[l];
                for (int o2 = 0; o2 < PROP_W; ++o2) da[o2] = A[k][l][o2] > 0.0 ? dh[o2] : 0.0;
                for (int o2 = 0; o2 < PROP_W; ++o2) {
                    for (int i = 0; i < fin; ++i) grad[off[l] + (long)o2 * fin + i] += da[o2] * in[i];
                    grad[off[l] + (long)PROP_W * fin + o2] += da[o2];
                }
                if (l > 0)
                    for (int i = 0; i < PROP_W; ++i) {
                        double s = 0.0;
                        for (int o2 = 0; o2 < PROP_W; ++o2) s += Wl[(long)o2 * fin + i] * da[o2];
                        dh[i] = s;
                    }
            }
        }
    }
    free(z); free(sr); free(al); free(T); free(w); free(gw); free(ds);
    free(A); free(Hh); free(G);
    return L;
}

/* Mean loss and mean gradient over n rays (o, d [n,3], hist [n, nb]). */
int orc_prop_loss_grad(const float* blob, int n, const double* o, const double* d, int nb,
                       double near_z, double far_z, const double* hist, double* loss,
                       double* grad) {
    long nw = orc_prop_n_weights();
    double* wd = widen(blob, nw);
    if (!wd) return -2;
    if (grad) for (long i = 0; i < nw; ++i) grad[i] = 0.0;
    double L = 0.0;
    for (int r = 0; r < n; ++r)
        L += prop_ray(wd, o + 3 * r, d + 3 * r, nb, near_z, far_z, hist + (long)r * nb, grad);
    *loss = L / n;
    if (grad) for (long i = 0; i < nw; ++i) grad[i] /= n;
    free(wd);
    return 0;
}

/* Proposal weights of n rays over nb stratified midpoints (for pins). */
int orc_prop_weights(const float* blob, int n, const double* o, const double* d, int nb,
                     double near_z, double far_z, double* wout) {
    long nw = orc_prop_n_weights();
    double* wd = widen(blob, nw);
    if (!wd) return -2;
    for (int r = 0; r < n; ++r) {
        const double* oo = o + 3 * r;
        const double* dd = d + 3 * r;
        double dn = sqrt(dd[0] * dd[0] + dd[1] * dd[1] + dd[2] * dd[2]);
        double* z = (double*)malloc(sizeof(double) * nb);
        double* sg = (double*)malloc(sizeof(double) * nb);
        double* col = (double*)calloc(3 * (size_t)nb, sizeof(double));
        for (int k = 0; k < nb; ++k) {
            double g[PROP_IN], a[PROP_DEPTH][PROP_W], h[PROP_DEPTH][PROP_W];
            z[k] = near_z + (far_z - near_z) * (k + 0.5) / nb;
            double x[3] = {oo[0] + z[k] * dd[0], oo[1] + z[k] * dd[1], oo[2] + z[k] * dd[2]};
            sg[k] = prop_forward(wd, x, g, a, h);
        }
        double C[3];
        orc_composite(nb, z, sg, col, dn, wout + (long)r * nb, NULL, C);
        free(z); free(sg); free(col);
    }
    free(wd);
    return 0;
}

/* Render with the proposal sampler: n_p proposal samples (stratified
 * midpoints) -> proposal weights -> n_g importance samples (as the basic
 * model's inverse CDF, with the proposal weights as the coarse weights) ->
 * main MLP -> composite -> n_f importance samples from those -> main MLP ->
 * composite of the n_g + n_f samples; Eq. 5 / F as render_ray.  out as
 * orc_render_rays (rgb, z_trans, z_opaque, F, ...). */
int orc_render_rays_proposal(const float* blob, const int* arch, const float* pblob, int n,
                             const double* o, const double* d, const orc_opts* op, int n_p,
                             int n_g, double* out) {
    long nw = orc_n_weights(arch);
    if (nw < 0) return -1;
    double* wd = widen(blob, nw);
    if (!wd) return -2;
    double* pw = (double*)malloc(sizeof(double) * (size_t)n * n_p);
    int err = orc_prop_weights(pblob, n, o, d, n_p, op->near_z, op->far_z, pw);
    int nf = op->n_fine;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : err)
    for (int r = 0; r < n; ++r) {
        const double* oo = o + 3 * r;
        const double* dd = d + 3 * r;
        double dn = sqrt(dd[0] * dd[0] + dd[1] * dd[1] + dd[2] * dd[2]);
        double dh[3] = {dd[0] / dn, dd[1] / dn, dd[2] / dn};
        int ntot = n_g + nf;
        double* zp = (double*)malloc(sizeof(double) * n_p);
        double* z = (double*)malloc(sizeof(double) * ntot);
        double* sg = (double*)malloc(sizeof(double) * ntot);
        double* cl = (double*)malloc(sizeof(double) * 3 * ntot);
        double* w = (double*)malloc(sizeof(double) * ntot);
        double* u = (double*)malloc(sizeof(double) * (n_g > nf ? n_g : nf) + 8);
        int* ord = (int*)malloc(sizeof(int) * ntot);
        double* zs = (double*)malloc(sizeof(double) * ntot);
        double* ss = (double*)malloc(sizeof(double) * ntot);
        double* cs = (double*)malloc(sizeof(double) * 3 * ntot);
        for (int k = 0; k < n_p; ++k) zp[k] = op->near_z + (op->far_z - op->near_z) * (k + 0.5) / n_p;
        for (int j = 0; j < n_g; ++j) u[j] = n_g > 1 ? (double)j / (n_g - 1) : 0.0;
        orc_sample_pdf(n_p, zp, pw + (long)r * n_p, n_g, u, z);
        for (int k = 0; k < n_g; ++k) {
            double x[3] = {oo[0] + z[k] * dd[0], oo[1] + z[k] * dd[1], oo[2] + z[k] * dd[2]};
            err |= mlp_eval(wd, arch, x, dh, sg + k, cl + 3 * k);
        }
        if (nf > 0) {
            double C0[3];
            orc_composite(n_g, z, sg, cl, dn, w, NULL, C0);
            for (int j = 0; j < nf; ++j) u[j] = nf > 1 ? (double)j / (nf - 1) : 0.0;
            orc_sample_pdf(n_g, z, w, nf, u, z + n_g);
            for (int k = n_g; k < ntot; ++k) {
                double x[3] = {oo[0] + z[k] * dd[0], oo[1] + z[k] * dd[1], oo[2] + z[k] * dd[2]};
                err |= mlp_eval(wd, arch, x, dh, sg + k, cl + 3 * k);
            }
        }
        for (int k = 0; k < ntot; ++k) ord[k] = k;
        for (int k = 1; k < ntot; ++k) {
            int v = ord[k], m = k - 1;
            while (m >= 0 && z[ord[m]] > z[v]) { ord[m + 1] = ord[m]; --m; }
            ord[m + 1] = v;
        }
        for (int k = 0; k < ntot; ++k) {
            zs[k] = z[ord[k]];
            ss[k] = sg[ord[k]];
            for (int c = 0; c < 3; ++c) cs[3 * k + c] = cl[3 * ord[k] + c];
        }
        double C[3];
        double* oout = out + 10 * (long)r;
        double* Tk = (double*)malloc(sizeof(double) * ntot);
        orc_composite(ntot, zs, ss, cs, dn, w, Tk, C);
        oout[0] = C[0]; oout[1] = C[1]; oout[2] = C[2];
        orc_uncertainty(ntot, zs, w, op->alpha, op->tau, oout + 3, oout + 4, oout + 5, oout + 6,
                        oout + 9);
        oout[7] = ss[ntot - 1];
        oout[8] = Tk[ntot - 1];
        free(Tk); free(zp); free(z); free(sg); free(cl); free(w); free(u); free(ord);
        free(zs); free(ss); free(cs);
    }
    free(pw); free(wd);
    return err ? -1 : 0;
}

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
