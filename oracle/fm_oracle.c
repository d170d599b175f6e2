/*
 * fm_oracle.c -- plain, slow FP64 CPU oracle for the regularised 3-D field-map
 * estimator of Lin & Fessler, "Efficient Regularized Field Map Estimation in 3D
 * MRI" (arXiv 2005.08661).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library's product path may link, load
 * or call this file: only the tests, the package's smoke check and the benchmark's
 * CPU-baseline leg use it.  It shares no code, header, table or constant with the
 * CUDA path.
 *
 * What it computes, in the paper's order and notation (units: t in the caller's
 * unit, w in radians per that unit):
 *   Eq. 3  r_cdmnj = Gamma_mn / (sum_c' |s_c'j|^2) * s_cj * conj(s_dj) * conj(y_cmj) * y_dnj,
 *          Gamma_mn = 1/L (field-map case), or the complex L x L projector
 *          gamma (gamma^H gamma)^{-1} gamma^H of the water-fat model (Eq. gamma), set by
 *          orc_set_gamma.  Precomputed once (Algorithm box).
 *   Eq. 2  Phi(w) = sum_j sum_{c,d,m,n} |r| (1 - cos(angle(r) + w_j (t_m - t_n))), literal
 *          (all ordered tuples, including m = n).
 *   Eq. 5  Psi = Phi + beta/2 ||C w||^2, C = non-periodic first-order differences between
 *          6-neighbours that are both inside the support mask.
 *   Eq. 8  grad Psi = grad Phi + beta C'C w, with (grad Phi)_j =
 *          sum |r| (t_m - t_n) sin(angle(r) + w_j (t_m - t_n)) (first power of t_m - t_n:
 *          the derivative of Eq. 2).
 *   Eq. 9-11  d_j = sum |r| (t_m - t_n)^2 sin(u)/u, u = angle(r) + w_j (t_m - t_n) wrapped
 *          into [-pi, pi] by removing the nearest multiple of 2 pi (Huber's optimal
 *          curvature for 1 - cos).
 *   Eq. 9  H = diag(d) + beta C'C over the mask voxels.
 *   Eq. 12 IC(0): a generic incomplete Cholesky on H's nonzero pattern, textbook
 *          right-looking k,i,j loop, natural (x fastest, then y, then z) order.
 *   Sec. III-B  IC with a drop tolerance (the paper's L_t): the same factorisation with
 *          fill-in allowed, where every off-diagonal factor entry smaller in magnitude
 *          than tau = droptol * H_max (H_max: the largest |H_jk|, recomputed for every
 *          outer iteration) is set to zero; generic left-looking column code (orc_ict).
 *   Eq. 6  w0_j = angle(conj(sum_c conj(s_c) y_c1) * sum_d conj(s_d) y_d2) / (t_2 - t_1).
 *   Algorithm box + Eq. 13-16: preconditioned Polak-Ribiere NCG, z = -p + mu z with
 *          mu^0 = 0, mu^i = (g^i - g^{i-1})'p^i / ((g^{i-1})'p^{i-1}); monotonic line
 *          search alpha_{k+1} = alpha_k - f'(alpha_k) / (d^(k) + beta ||C z||^2),
 *          d^(k) = sum_j z_j^2 d_j(w + alpha_k z), alpha_0 = 0, N_ls fixed steps.
 * Reductions over voxels are taken in fixed chunks of ORC_CHUNK consecutive voxels: each
 * chunk is summed sequentially in voxel order and the chunk sums are added in chunk order.
 * With OpenMP (orc_set_threads) the chunks and the per-voxel loops are spread over
 * threads; the fixed chunking makes every result bitwise independent of the thread count.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_CHUNK 8192
static int g_threads = 1;

/* Number of host threads for the per-voxel loops and chunked sums (>= 1; 1 = serial).
 * Returns the count in effect (1 when built without OpenMP). */
int orc_set_threads(int n) {
#ifdef _OPENMP
    g_threads = n < 1 ? 1 : n;
#else
    (void)n;
    g_threads = 1;
#endif
    return g_threads;
}

int orc_get_threads(void) { return g_threads; }

/* sum_{j in [0, n)} of a per-index term, chunked as stated in the header */
typedef double (*orc_range_sum)(const void *arg, long j0, long j1);
static double chunked_sum(long n, orc_range_sum f, const void *arg) {
    long nch = (n + ORC_CHUNK - 1) / ORC_CHUNK;
    double stack_part[64];
    double *part = nch <= 64 ? stack_part : (double *)malloc(sizeof(double) * nch);
    double acc = 0.0;
    if (!part) return NAN;
#pragma omp parallel for schedule(static) if (g_threads > 1) num_threads(g_threads)
    for (long c = 0; c < nch; ++c) {
        long j0 = c * ORC_CHUNK, j1 = j0 + ORC_CHUNK < n ? j0 + ORC_CHUNK : n;
        part[c] = f(arg, j0, j1);
    }
    for (long c = 0; c < nch; ++c) acc += part[c];
    if (part != stack_part) free(part);
    return acc;
}

/* sum_j a_j b_j over [0, n) */
typedef struct { const double *a, *b; } dot_arg;
static double dot_range(const void *p, long j0, long j1) {
    const dot_arg *d = (const dot_arg *)p;
    double acc = 0.0;
    for (long j = j0; j < j1; ++j) acc += d->a[j] * d->b[j];
    return acc;
}
static double dot(long n, const double *a, const double *b) {
    dot_arg d = {a, b};
    return chunked_sum(n, dot_range, &d);
}

/* sum_j a_j over [0, n) */
static double sum_range(const void *p, long j0, long j1) {
    const double *a = (const double *)p;
    double acc = 0.0;
    for (long j = j0; j < j1; ++j) acc += a[j];
    return acc;
}
static double sum(long n, const double *a) { return chunked_sum(n, sum_range, a); }

#define ORC_OK 0
#define ORC_ERR_ARG (-1)
#define ORC_ERR_NOT_PD (-4)
#define ORC_ERR_OOM (-7)
#define ORC_MAXL 32

typedef struct {
    int nx, ny, nz, nc, L;
    long nv;
    double beta;
    double te[ORC_MAXL];
    unsigned char *mask; /* [nv], 1 = unknown */
    double *y;           /* [L][nc][nv][2] */
    double *s;           /* [nc][nv][2] or NULL (s = 1) */
    long T;              /* tuples per voxel: nc*nc*L*L */
    long *slot;          /* [nv] -> index among mask voxels, -1 outside */
    long nm;             /* number of mask voxels */
    double *rabs, *rang; /* [nm][T] modulus and angle of r_cdmnj */
    double *dt;          /* [T] t_m - t_n of each tuple */
    int curv_mode;       /* 0: literal Eq. 10 sum; 1: coil-combined pair weights (labelled variant) */
    double droptol;      /* drop tolerance of the thresholded IC, relative to H_max (default 1e-3) */
    int has_gam;         /* 0: Gamma_mn = 1/L; 1: gam holds a complex L x L Gamma */
    double gam[2 * ORC_MAXL * ORC_MAXL];
} orc_t;

static const double TWO_PI = 6.283185307179586476925286766559;

/* wrap an angle into [-pi, pi] by removing the nearest multiple of 2 pi */
static double wrap_angle(double th) { return th - TWO_PI * nearbyint(th / TWO_PI); }

static double sinc(double u) { return u == 0.0 ? 1.0 : sin(u) / u; }

/* Gamma_mn (Eq. 3, Eq. gamma): 1/L, or the stored complex projector entry */
static void gamma_mn(const double *gam, int L, int m, int n, double *gr, double *gi) {
    if (gam) {
        *gr = gam[2 * (m * L + n)];
        *gi = gam[2 * (m * L + n) + 1];
    } else {
        *gr = 1.0 / (double)L;
        *gi = 0.0;
    }
}

/* Eq. 3 for one voxel: y_vox[(l*nc + c)*2 + {0,1}], s_vox[c*2 + {0,1}] (NULL: s = 1);
 * gam: complex L x L Gamma or NULL (1/L). */
static void pair_weights(int nc, int L, const double *y_vox, long ystride, const double *s_vox,
                         long sstride, const double *gam, double *rabs, double *rang) {
    double S = 0.0;
    for (int c = 0; c < nc; ++c) {
        double sr = s_vox ? s_vox[c * sstride] : 1.0, si = s_vox ? s_vox[c * sstride + 1] : 0.0;
        S += sr * sr + si * si;
    }
    long t = 0;
    for (int c = 0; c < nc; ++c)
        for (int d = 0; d < nc; ++d)
            for (int m = 0; m < L; ++m)
                for (int n = 0; n < L; ++n, ++t) {
                    if (S == 0.0) { rabs[t] = 0.0; rang[t] = 0.0; continue; }
                    double Gr, Gi;
                    gamma_mn(gam, L, m, n, &Gr, &Gi);
                    double scr = s_vox ? s_vox[c * sstride] : 1.0, sci = s_vox ? s_vox[c * sstride + 1] : 0.0;
                    double sdr = s_vox ? s_vox[d * sstride] : 1.0, sdi = s_vox ? -s_vox[d * sstride + 1] : 0.0; /* conj(s_d) */
                    const double *ycm = y_vox + (long)(m * nc + c) * ystride;
                    const double *ydn = y_vox + (long)(n * nc + d) * ystride;
                    double ar = ycm[0], ai = -ycm[1]; /* conj(y_cm) */
                    double br = ydn[0], bi = ydn[1];
                    /* s_c * conj(s_d) */
                    double pr = scr * sdr - sci * sdi, pi_ = scr * sdi + sci * sdr;
                    /* * conj(y_cm) */
                    double qr = pr * ar - pi_ * ai, qi = pr * ai + pi_ * ar;
                    /* * y_dn */
                    double ur = qr * br - qi * bi, ui = qr * bi + qi * br;
                    /* * Gamma_mn / S */
                    double rr = (Gr * ur - Gi * ui) / S, ri = (Gr * ui + Gi * ur) / S;
                    rabs[t] = hypot(rr, ri);
                    rang[t] = atan2(ri, rr);
                }
}

static void tuple_dt(int nc, int L, const double *te, double *dt) {
    long t = 0;
    for (int c = 0; c < nc; ++c)
        for (int d = 0; d < nc; ++d)
            for (int m = 0; m < L; ++m)
                for (int n = 0; n < L; ++n, ++t) dt[t] = te[m] - te[n];
}

/* per-voxel data-term pieces at w: phi (Eq. 2 term), dphi (Eq. 8 term), curvature (Eq. 10) */
static void voxel_terms(long T, const double *rabs, const double *rang, const double *dt, double w,
                        double *phi, double *dphi, double *curv) {
    double a = 0.0, b = 0.0, c = 0.0;
    for (long t = 0; t < T; ++t) {
        double th = rang[t] + w * dt[t];
        if (phi) a += rabs[t] * (1.0 - cos(th));
        if (dphi) b += rabs[t] * dt[t] * sin(th);
        if (curv) c += rabs[t] * dt[t] * dt[t] * sinc(wrap_angle(th));
    }
    if (phi) *phi = a;
    if (dphi) *dphi = b;
    if (curv) *curv = c;
}

void orc_destroy(orc_t *h) {
    if (!h) return;
    free(h->mask); free(h->y); free(h->s); free(h->slot); free(h->rabs); free(h->rang); free(h->dt);
    free(h);
}

/* y: [L][nc][nv] complex (interleaved re,im); s: [nc][nv] complex or NULL; mask: [nv] or NULL */
int orc_create(orc_t **out, int nx, int ny, int nz, int nc, int L, const double *y, const double *s,
               const double *te, const unsigned char *mask, double beta) {
    if (!out || nx < 1 || ny < 1 || nz < 1 || nc < 1 || L < 2 || L > ORC_MAXL || !y || !te) return ORC_ERR_ARG;
    if (!s && nc != 1) return ORC_ERR_ARG;
    orc_t *h = (orc_t *)calloc(1, sizeof(orc_t));
    if (!h) return ORC_ERR_OOM;
    h->nx = nx; h->ny = ny; h->nz = nz; h->nc = nc; h->L = L;
    h->nv = (long)nx * ny * nz;
    h->beta = beta;
    h->droptol = 1e-3;
    for (int l = 0; l < L; ++l) h->te[l] = te[l];
    h->T = (long)nc * nc * L * L;
    h->mask = (unsigned char *)malloc(h->nv);
    h->y = (double *)malloc(sizeof(double) * 2 * L * nc * h->nv);
    h->s = s ? (double *)malloc(sizeof(double) * 2 * nc * h->nv) : NULL;
    h->slot = (long *)malloc(sizeof(long) * h->nv);
    h->dt = (double *)malloc(sizeof(double) * h->T);
    if (!h->mask || !h->y || (s && !h->s) || !h->slot || !h->dt) { orc_destroy(h); return ORC_ERR_OOM; }
    for (long j = 0; j < h->nv; ++j) h->mask[j] = mask ? (mask[j] != 0) : 1;
    memcpy(h->y, y, sizeof(double) * 2 * L * nc * h->nv);
    if (s) memcpy(h->s, s, sizeof(double) * 2 * nc * h->nv);
    tuple_dt(nc, L, h->te, h->dt);
    h->nm = 0;
    for (long j = 0; j < h->nv; ++j) h->slot[j] = h->mask[j] ? h->nm++ : -1;
    h->rabs = (double *)malloc(sizeof(double) * (h->nm ? h->nm : 1) * h->T);
    h->rang = (double *)malloc(sizeof(double) * (h->nm ? h->nm : 1) * h->T);
    if (!h->rabs || !h->rang) { orc_destroy(h); return ORC_ERR_OOM; }
    /* precompute r_cdmnj (Eq. 3) once, as the Algorithm box does */
#pragma omp parallel for schedule(dynamic, 256) if (g_threads > 1) num_threads(g_threads)
    for (long j = 0; j < h->nv; ++j) {
        long k = h->slot[j];
        if (k < 0) continue;
        pair_weights(nc, L, h->y + 2 * j, 2 * h->nv, h->s ? h->s + 2 * j : NULL, 2 * h->nv, NULL,
                     h->rabs + k * h->T, h->rang + k * h->T);
    }
    *out = h;
    return ORC_OK;
}

long orc_num_unknowns(const orc_t *h) { return h->nm; }

/* Phi (Eq. 2) over the mask voxels */
typedef struct { const orc_t *h; const double *w; } hw_arg;
static double phi_range(const void *p, long j0, long j1) {
    const orc_t *h = ((const hw_arg *)p)->h;
    const double *w = ((const hw_arg *)p)->w;
    double acc = 0.0;
    for (long j = j0; j < j1; ++j) {
        long k = h->slot[j];
        if (k < 0) continue;
        double ph;
        voxel_terms(h->T, h->rabs + k * h->T, h->rang + k * h->T, h->dt, w[j], &ph, NULL, NULL);
        acc += ph;
    }
    return acc;
}
double orc_phi(const orc_t *h, const double *w) {
    hw_arg a = {h, w};
    return chunked_sum(h->nv, phi_range, &a);
}

/* neighbour helpers: forward neighbours (+x, +y, +z) of voxel j, -1 if outside grid or mask */
static long fwd_nbr(const orc_t *h, long j, int axis) {
    long x = j % h->nx, y = (j / h->nx) % h->ny, z = j / ((long)h->nx * h->ny);
    long k = -1;
    if (axis == 0 && x + 1 < h->nx) k = j + 1;
    if (axis == 1 && y + 1 < h->ny) k = j + h->nx;
    if (axis == 2 && z + 1 < h->nz) k = j + (long)h->nx * h->ny;
    return (k >= 0 && h->mask[k]) ? k : -1;
}

static long bwd_nbr(const orc_t *h, long j, int axis) {
    long x = j % h->nx, y = (j / h->nx) % h->ny, z = j / ((long)h->nx * h->ny);
    long k = -1;
    if (axis == 0 && x > 0) k = j - 1;
    if (axis == 1 && y > 0) k = j - h->nx;
    if (axis == 2 && z > 0) k = j - (long)h->nx * h->ny;
    return (k >= 0 && h->mask[k]) ? k : -1;
}

/* sum over edges (both ends in the mask) of (a_j - a_k)(b_j - b_k), each edge counted at
 * its lower voxel j */
typedef struct { const orc_t *h; const double *a, *b; } edge_arg;
static double edge_range(const void *p, long j0, long j1) {
    const edge_arg *e = (const edge_arg *)p;
    double acc = 0.0;
    for (long j = j0; j < j1; ++j) {
        if (!e->h->mask[j]) continue;
        for (int ax = 0; ax < 3; ++ax) {
            long k = fwd_nbr(e->h, j, ax);
            if (k >= 0) acc += (e->a[j] - e->a[k]) * (e->b[j] - e->b[k]);
        }
    }
    return acc;
}
static double edge_dot(const orc_t *h, const double *a, const double *b) {
    edge_arg e = {h, a, b};
    return chunked_sum(h->nv, edge_range, &e);
}

/* beta/2 ||C w||^2 */
double orc_reg(const orc_t *h, const double *w) { return 0.5 * h->beta * edge_dot(h, w, w); }

double orc_cost(const orc_t *h, const double *w) { return orc_phi(h, w) + orc_reg(h, w); }

/* grad Psi (Eq. 8); zero outside the mask */
void orc_grad(const orc_t *h, const double *w, double *g) {
#pragma omp parallel for schedule(dynamic, 256) if (g_threads > 1) num_threads(g_threads)
    for (long j = 0; j < h->nv; ++j) {
        long k = h->slot[j];
        if (k < 0) { g[j] = 0.0; continue; }
        double dp;
        voxel_terms(h->T, h->rabs + k * h->T, h->rang + k * h->T, h->dt, w[j], NULL, &dp, NULL);
        double lap = 0.0;
        for (int ax = 0; ax < 3; ++ax) {
            long a = fwd_nbr(h, j, ax), b = bwd_nbr(h, j, ax);
            if (a >= 0) lap += w[j] - w[a];
            if (b >= 0) lap += w[j] - w[b];
        }
        g[j] = dp + h->beta * lap;
    }
}

/* gradient of the data term alone */
void orc_grad_phi(const orc_t *h, const double *w, double *g) {
#pragma omp parallel for schedule(dynamic, 256) if (g_threads > 1) num_threads(g_threads)
    for (long j = 0; j < h->nv; ++j) {
        long k = h->slot[j];
        if (k < 0) { g[j] = 0.0; continue; }
        voxel_terms(h->T, h->rabs + k * h->T, h->rang + k * h->T, h->dt, w[j], NULL, g + j, NULL);
    }
}

/* Labelled variant of the curvature: Huber's curvature of the coil-combined pair terms,
 * sum_{m,n} |R_mn| (t_m - t_n)^2 sinc(wrap(angle R_mn + w (t_m - t_n))), R_mn = sum_{c,d} r_cdmn.
 * Because Phi_j = const + sum_{m,n} |R_mn| (1 - cos(angle R_mn + w (t_m - t_n))) exactly, it is
 * also a majoriser curvature.  Identical to Eq. 10 for one coil. */
static double voxel_curv_combined(const orc_t *h, const double *rabs, const double *rang, double w) {
    int L = h->L, nc = h->nc;
    double acc = 0.0;
    for (int m = 0; m < L; ++m)
        for (int n = 0; n < L; ++n) {
            double rr = 0.0, ri = 0.0;
            for (int c = 0; c < nc; ++c)
                for (int d = 0; d < nc; ++d) {
                    long t = (((long)c * nc + d) * L + m) * L + n;
                    rr += rabs[t] * cos(rang[t]);
                    ri += rabs[t] * sin(rang[t]);
                }
            double dt = h->te[m] - h->te[n];
            double Ra = hypot(rr, ri), Rg = atan2(ri, rr);
            acc += Ra * dt * dt * sinc(wrap_angle(Rg + w * dt));
        }
    return acc;
}

void orc_set_curvature(orc_t *h, int mode) { h->curv_mode = mode; }

/* curvature d_j of Eq. 10 at w (or the combined variant); zero outside the mask */
void orc_curv(const orc_t *h, const double *w, double *d) {
#pragma omp parallel for schedule(dynamic, 256) if (g_threads > 1) num_threads(g_threads)
    for (long j = 0; j < h->nv; ++j) {
        long k = h->slot[j];
        if (k < 0) { d[j] = 0.0; continue; }
        if (h->curv_mode == 1) d[j] = voxel_curv_combined(h, h->rabs + k * h->T, h->rang + k * h->T, w[j]);
        else voxel_terms(h->T, h->rabs + k * h->T, h->rang + k * h->T, h->dt, w[j], NULL, NULL, d + j);
    }
}

/* Second derivative of Phi_j (Eq. 2) at w: sum |r| (t_m - t_n)^2 cos(angle r + w (t_m - t_n)),
 * the diagonal of the true Hessian of the data term (used for implicit differentiation of the
 * converged field map, not by the solver).  Zero outside the mask. */
void orc_hess_diag(const orc_t *h, const double *w, double *out) {
#pragma omp parallel for schedule(dynamic, 256) if (g_threads > 1) num_threads(g_threads)
    for (long j = 0; j < h->nv; ++j) {
        long k = h->slot[j];
        if (k < 0) { out[j] = 0.0; continue; }
        const double *ra = h->rabs + k * h->T, *rg = h->rang + k * h->T;
        double acc = 0.0;
        for (long t = 0; t < h->T; ++t) acc += ra[t] * h->dt[t] * h->dt[t] * cos(rg[t] + w[j] * h->dt[t]);
        out[j] = acc;
    }
}

/* Directional derivative of (grad Phi)_j (Eq. 8) with respect to the images y in the complex
 * direction dy ([L][nc][nv], interleaved): product rule on Eq. 3,
 * d r_cdmn = Gamma_mn/S s_c conj(s_d) (conj(dy_cm) y_dn + conj(y_cm) dy_dn), and
 * d (grad Phi)_j = sum (t_m - t_n) Im(d r e^{i w (t_m - t_n)}).  Zero outside the mask. */
void orc_dgrad_dy(const orc_t *h, const double *w, const double *dy, double *out) {
    const int nc = h->nc, L = h->L;
    const double *gam = h->has_gam ? h->gam : NULL;
    for (long j = 0; j < h->nv; ++j) {
        if (!h->mask[j]) { out[j] = 0.0; continue; }
        double S = 0.0;
        for (int c = 0; c < nc; ++c) {
            double sr = h->s ? h->s[2 * (c * h->nv + j)] : 1.0, si = h->s ? h->s[2 * (c * h->nv + j) + 1] : 0.0;
            S += sr * sr + si * si;
        }
        if (S == 0.0) { out[j] = 0.0; continue; }
        double acc = 0.0;
        for (int c = 0; c < nc; ++c)
            for (int d = 0; d < nc; ++d)
                for (int m = 0; m < L; ++m)
                    for (int n = 0; n < L; ++n) {
                        double scr = h->s ? h->s[2 * (c * h->nv + j)] : 1.0, sci = h->s ? h->s[2 * (c * h->nv + j) + 1] : 0.0;
                        double sdr = h->s ? h->s[2 * (d * h->nv + j)] : 1.0, sdi = h->s ? -h->s[2 * (d * h->nv + j) + 1] : 0.0;
                        double pr = scr * sdr - sci * sdi, pi_ = scr * sdi + sci * sdr; /* s_c conj(s_d) */
                        const double *ycm = h->y + 2 * ((long)(m * nc + c) * h->nv + j);
                        const double *ydn = h->y + 2 * ((long)(n * nc + d) * h->nv + j);
                        const double *dcm = dy + 2 * ((long)(m * nc + c) * h->nv + j);
                        const double *ddn = dy + 2 * ((long)(n * nc + d) * h->nv + j);
                        /* conj(dy_cm) y_dn + conj(y_cm) dy_dn */
                        double ar = dcm[0] * ydn[0] + dcm[1] * ydn[1], ai = dcm[0] * ydn[1] - dcm[1] * ydn[0];
                        double br = ycm[0] * ddn[0] + ycm[1] * ddn[1], bi = ycm[0] * ddn[1] - ycm[1] * ddn[0];
                        double qr = ar + br, qi = ai + bi;
                        double Gr, Gi;
                        gamma_mn(gam, L, m, n, &Gr, &Gi);
                        double er = pr * Gr - pi_ * Gi, ei = pr * Gi + pi_ * Gr; /* Gamma_mn s_c conj(s_d) */
                        double rr = (er * qr - ei * qi) / S, ri = (er * qi + ei * qr) / S;
                        double dt = h->te[m] - h->te[n];
                        double th = w[j] * dt;
                        acc += dt * (rr * sin(th) + ri * cos(th)); /* Im(dr e^{i th}) */
                    }
        out[j] = acc;
    }
}

/* Adjoint of orc_dgrad_dy: out = sum_j lam_j grad_y (grad Phi)_j as a complex array
 * [L][nc][nv] (interleaved), in the convention out = d/dRe y + i d/dIm y.  Each term
 * f = (t_m - t_n) Im(A conj(y_cm) y_dn), A = Gamma/S s_c conj(s_d) e^{i w (t_m - t_n)},
 * contributes -i (t_m - t_n) A y_dn to y_cm and i (t_m - t_n) conj(A) y_cm to y_dn. */
void orc_dgrad_dy_adj(const orc_t *h, const double *w, const double *lam, double *out) {
    const int nc = h->nc, L = h->L;
    const double *gam = h->has_gam ? h->gam : NULL;
    for (long i = 0; i < 2L * L * nc * h->nv; ++i) out[i] = 0.0;
    for (long j = 0; j < h->nv; ++j) {
        if (!h->mask[j] || lam[j] == 0.0) continue;
        double S = 0.0;
        for (int c = 0; c < nc; ++c) {
            double sr = h->s ? h->s[2 * (c * h->nv + j)] : 1.0, si = h->s ? h->s[2 * (c * h->nv + j) + 1] : 0.0;
            S += sr * sr + si * si;
        }
        if (S == 0.0) continue;
        for (int c = 0; c < nc; ++c)
            for (int d = 0; d < nc; ++d)
                for (int m = 0; m < L; ++m)
                    for (int n = 0; n < L; ++n) {
                        double dt = h->te[m] - h->te[n];
                        if (dt == 0.0) continue;
                        double scr = h->s ? h->s[2 * (c * h->nv + j)] : 1.0, sci = h->s ? h->s[2 * (c * h->nv + j) + 1] : 0.0;
                        double sdr = h->s ? h->s[2 * (d * h->nv + j)] : 1.0, sdi = h->s ? -h->s[2 * (d * h->nv + j) + 1] : 0.0;
                        double pr = scr * sdr - sci * sdi, pi_ = scr * sdi + sci * sdr; /* s_c conj(s_d) */
                        double th = w[j] * dt, ct = cos(th), st = sin(th);
                        double Gr, Gi;
                        gamma_mn(gam, L, m, n, &Gr, &Gi);
                        double er = pr * Gr - pi_ * Gi, ei = pr * Gi + pi_ * Gr; /* Gamma_mn s_c conj(s_d) */
                        double Ar = (er * ct - ei * st) / S, Ai = (er * st + ei * ct) / S;
                        const double *ycm = h->y + 2 * ((long)(m * nc + c) * h->nv + j);
                        const double *ydn = h->y + 2 * ((long)(n * nc + d) * h->nv + j);
                        double *ocm = out + 2 * ((long)(m * nc + c) * h->nv + j);
                        double *odn = out + 2 * ((long)(n * nc + d) * h->nv + j);
                        double k = lam[j] * dt;
                        /* -i A y_dn */
                        double ur = Ar * ydn[0] - Ai * ydn[1], ui = Ar * ydn[1] + Ai * ydn[0];
                        ocm[0] += k * ui;
                        ocm[1] -= k * ur;
                        /* i conj(A) y_cm */
                        double vr = Ar * ycm[0] + Ai * ycm[1], vi = Ar * ycm[1] - Ai * ycm[0];
                        odn[0] -= k * vi;
                        odn[1] += k * vr;
                    }
    }
}

/* Water-fat model (Eq. gamma): replace Gamma_mn = 1/L by the complex L x L matrix gam
 * (interleaved, row m, column n) and recompute every r_cdmnj (Eq. 3). */
int orc_set_gamma(orc_t *h, const double *gam) {
    if (!h || !gam) return ORC_ERR_ARG;
    const int L = h->L;
    for (int i = 0; i < 2 * L * L; ++i) h->gam[i] = gam[i];
    h->has_gam = 1;
    for (long j = 0; j < h->nv; ++j) {
        long k = h->slot[j];
        if (k < 0) continue;
        pair_weights(h->nc, L, h->y + 2 * j, 2 * h->nv, h->s ? h->s + 2 * j : NULL, 2 * h->nv, h->gam,
                     h->rabs + k * h->T, h->rang + k * h->T);
    }
    return ORC_OK;
}

/* Phi_j(w_j) (Eq. 2) of every voxel (0 outside the mask). */
void orc_phi_vox(const orc_t *h, const double *w, double *out) {
#pragma omp parallel for schedule(dynamic, 256) if (g_threads > 1) num_threads(g_threads)
    for (long j = 0; j < h->nv; ++j) {
        long k = h->slot[j];
        double phi = 0.0;
        if (k >= 0) voxel_terms(h->T, h->rabs + k * h->T, h->rang + k * h->T, h->dt, w[j], &phi, NULL, NULL);
        out[j] = phi;
    }
}

/* Spatial weights of the PWLS initialisation (Eq. w0_wf): rho_j = sum_{c,d,m,n} |r_cdmnj|. */
void orc_rho(const orc_t *h, double *out) {
    for (long j = 0; j < h->nv; ++j) {
        long k = h->slot[j];
        double acc = 0.0;
        if (k >= 0)
            for (long t = 0; t < h->T; ++t) acc += h->rabs[k * h->T + t];
        out[j] = acc;
    }
}

/* Voxel-wise initialisation of the water-fat case (Sec. III-A): evaluate Phi_j (Eq. 2) at
 * nsweep equally spaced values from wlo to whi (both included) and keep the first value
 * with the smallest cost.  Zero outside the mask. */
void orc_wf_sweep(const orc_t *h, int nsweep, double wlo, double whi, double *out) {
#pragma omp parallel for schedule(dynamic, 256) if (g_threads > 1) num_threads(g_threads)
    for (long j = 0; j < h->nv; ++j) {
        long k = h->slot[j];
        if (k < 0) { out[j] = 0.0; continue; }
        double best = 0.0, best_phi = 0.0;
        for (int q = 0; q < nsweep; ++q) {
            double w = nsweep > 1 ? wlo + (whi - wlo) * (double)q / (double)(nsweep - 1) : wlo;
            double phi;
            voxel_terms(h->T, h->rabs + k * h->T, h->rang + k * h->T, h->dt, w, &phi, NULL, NULL);
            if (q == 0 || phi < best_phi) { best_phi = phi; best = w; }
        }
        out[j] = best;
    }
}

/* A x with A = 2 diag(rho) + beta C'C on the mask (the Hessian of Eq. w0_wf); 0 outside. */
static void pwls_apply(const orc_t *h, const double *rho, const double *x, double *ax) {
    for (long j = 0; j < h->nv; ++j) {
        if (!h->mask[j]) { ax[j] = 0.0; continue; }
        double lap = 0.0;
        for (int axis = 0; axis < 3; ++axis) {
            long f = fwd_nbr(h, j, axis), b = bwd_nbr(h, j, axis);
            if (f >= 0) lap += x[j] - x[f];
            if (b >= 0) lap += x[j] - x[b];
        }
        ax[j] = 2.0 * rho[j] * x[j] + h->beta * lap;
    }
}

/* PWLS initialisation (Eq. w0_wf): niter iterations of conjugate gradients on
 * (2 diag(rho) + beta C'C) w = 2 rho wt, starting from w = wt (the sweep's map). */
int orc_pwls(const orc_t *h, const double *wt, int niter, double *out) {
    const long nv = h->nv;
    double *rho = (double *)malloc(sizeof(double) * nv), *r = (double *)malloc(sizeof(double) * nv);
    double *p = (double *)malloc(sizeof(double) * nv), *q = (double *)malloc(sizeof(double) * nv);
    if (!rho || !r || !p || !q) { free(rho); free(r); free(p); free(q); return ORC_ERR_OOM; }
    orc_rho(h, rho);
    for (long j = 0; j < nv; ++j) out[j] = h->mask[j] ? wt[j] : 0.0;
    pwls_apply(h, rho, out, q);
    double rr = 0.0;
    for (long j = 0; j < nv; ++j) {
        r[j] = h->mask[j] ? 2.0 * rho[j] * wt[j] - q[j] : 0.0;
        p[j] = r[j];
        rr += r[j] * r[j];
    }
    for (int it = 0; it < niter && rr > 0.0; ++it) {
        pwls_apply(h, rho, p, q);
        double pq = 0.0;
        for (long j = 0; j < nv; ++j) pq += p[j] * q[j];
        if (!(pq > 0.0)) break;
        double alpha = rr / pq, rr_new = 0.0;
        for (long j = 0; j < nv; ++j) {
            out[j] += alpha * p[j];
            r[j] -= alpha * q[j];
            rr_new += r[j] * r[j];
        }
        double b = rr_new / rr;
        for (long j = 0; j < nv; ++j) p[j] = r[j] + b * p[j];
        rr = rr_new;
    }
    free(rho); free(r); free(p); free(q);
    return ORC_OK;
}

/* Eq. 6: initial field map from the first two echoes; zero outside the mask */
void orc_init(const orc_t *h, double *w) {
    for (long j = 0; j < h->nv; ++j) {
        if (!h->mask[j]) { w[j] = 0.0; continue; }
        double z1r = 0, z1i = 0, z2r = 0, z2i = 0;
        for (int c = 0; c < h->nc; ++c) {
            double sr = h->s ? h->s[2 * (c * h->nv + j)] : 1.0;
            double si = h->s ? -h->s[2 * (c * h->nv + j) + 1] : 0.0; /* conj(s_c) */
            const double *y1 = h->y + 2 * ((long)(0 * h->nc + c) * h->nv + j);
            const double *y2 = h->y + 2 * ((long)(1 * h->nc + c) * h->nv + j);
            z1r += sr * y1[0] - si * y1[1]; z1i += sr * y1[1] + si * y1[0];
            z2r += sr * y2[0] - si * y2[1]; z2i += sr * y2[1] + si * y2[0];
        }
        /* conj(z1) * z2 */
        double pr = z1r * z2r + z1i * z2i, pi_ = z1r * z2i - z1i * z2r;
        double ang = (pr == 0.0 && pi_ == 0.0) ? 0.0 : atan2(pi_, pr);
        w[j] = ang / (h->te[1] - h->te[0]);
    }
}

/* ---------------------------------------------------------------------------------
 * IC(0) of H = diag(d) + beta C'C (Eq. 9, Eq. 12) on the mask voxels, generic sparse
 * code: H's lower triangle in compressed-column form (diagonal first in each column,
 * rows ascending), factorised in place by the textbook right-looking loop that only
 * updates entries inside the pattern.  order 0: unknowns in natural voxel order (the
 * paper's); order 1: red-black, every voxel with x + y + z even (natural order among
 * them) before every voxel with x + y + z odd (the labelled multicolour variant, an
 * IC(0) of P H P' for that permutation P).
 * colptr: [n+1], rowidx/val: capacity 4 nv, umap: [nv] voxel of each unknown.
 * ------------------------------------------------------------------------------- */
int orc_ic0_ordered(int nx, int ny, int nz, const unsigned char *mask, const double *d, double beta, int order,
                    long *colptr, long *rowidx, double *val, long *umap, long *n_out, long *nnz_out) {
    long nv = (long)nx * ny * nz, nxy = (long)nx * ny;
    long *uidx = (long *)malloc(sizeof(long) * nv);
    if (!uidx) return ORC_ERR_OOM;
    long n = 0;
    for (int pass = 0; pass < (order == 1 ? 2 : 1); ++pass)
        for (long j = 0; j < nv; ++j) {
            if (order == 1 && (int)((j % nx + (j / nx) % ny + j / nxy) % 2) != pass) continue;
            if (mask == NULL || mask[j]) {
                uidx[j] = n;
                umap[n++] = j;
            } else {
                uidx[j] = -1;
            }
        }
    /* assemble lower(H) column by column: the diagonal, then every neighbour numbered later */
    long nnz = 0;
    for (long u = 0; u < n; ++u) {
        long j = umap[u];
        long x = j % nx, y = (j / nx) % ny, z = j / nxy;
        long nb[6] = {x > 0 ? j - 1 : -1, x + 1 < nx ? j + 1 : -1, y > 0 ? j - nx : -1,
                      y + 1 < ny ? j + nx : -1, z > 0 ? j - nxy : -1, z + 1 < nz ? j + nxy : -1};
        int cnt = 0;
        for (int q = 0; q < 6; ++q) if (nb[q] >= 0 && uidx[nb[q]] >= 0) ++cnt;
        colptr[u] = nnz;
        rowidx[nnz] = u; val[nnz] = d[j] + beta * cnt; ++nnz;
        long later[6];
        int nl = 0;
        for (int q = 0; q < 6; ++q)
            if (nb[q] >= 0 && uidx[nb[q]] > u) later[nl++] = uidx[nb[q]];
        for (int a = 1; a < nl; ++a) /* ascending row order */
            for (int b = a; b > 0 && later[b - 1] > later[b]; --b) {
                long t = later[b]; later[b] = later[b - 1]; later[b - 1] = t;
            }
        for (int q = 0; q < nl; ++q) { rowidx[nnz] = later[q]; val[nnz] = -beta; ++nnz; }
    }
    colptr[n] = nnz;
    free(uidx);
    /* right-looking IC(0), updates restricted to the pattern */
    for (long k = 0; k < n; ++k) {
        double akk = val[colptr[k]];
        if (!(akk > 0.0)) return ORC_ERR_NOT_PD;
        double lkk = sqrt(akk);
        val[colptr[k]] = lkk;
        for (long p = colptr[k] + 1; p < colptr[k + 1]; ++p) val[p] /= lkk;
        for (long p = colptr[k] + 1; p < colptr[k + 1]; ++p) {
            long i = rowidx[p];
            for (long q = colptr[k] + 1; q <= p; ++q) {
                long jj = rowidx[q];
                for (long r = colptr[jj]; r < colptr[jj + 1]; ++r)
                    if (rowidx[r] == i) { val[r] -= val[p] * val[q]; break; }
            }
        }
    }
    *n_out = n;
    *nnz_out = nnz;
    return ORC_OK;
}

int orc_ic0(int nx, int ny, int nz, const unsigned char *mask, const double *d, double beta,
            long *colptr, long *rowidx, double *val, long *umap, long *n_out, long *nnz_out) {
    return orc_ic0_ordered(nx, ny, nz, mask, d, beta, 0, colptr, rowidx, val, umap, n_out, nnz_out);
}

/* x = (L L')^{-1} b with the compressed-column factor of orc_ic0 */
void orc_ic0_solve(long n, const long *colptr, const long *rowidx, const double *val, const double *b,
                   double *x) {
    double *v = (double *)malloc(sizeof(double) * (n ? n : 1));
    for (long k = 0; k < n; ++k) v[k] = b[k];
    for (long k = 0; k < n; ++k) { /* forward: L v = b */
        v[k] /= val[colptr[k]];
        for (long p = colptr[k] + 1; p < colptr[k + 1]; ++p) v[rowidx[p]] -= val[p] * v[k];
    }
    for (long k = n - 1; k >= 0; --k) { /* back: L' x = v */
        double s = v[k];
        for (long p = colptr[k] + 1; p < colptr[k + 1]; ++p) s -= val[p] * x[rowidx[p]];
        x[k] = s / val[colptr[k]];
    }
    free(v);
}

/* p = (L L')^{-1} g for the IC(0) factor of H(w) = diag(d(w)) + beta C'C in the given
 * unknown order (0 natural, 1 red-black); voxel-indexed arrays */
int orc_precondition_ordered(const orc_t *h, const double *d, const double *g, double *p, int order) {
    long nv = h->nv;
    long *colptr = (long *)malloc(sizeof(long) * (nv + 1));
    long *rowidx = (long *)malloc(sizeof(long) * 4 * nv);
    double *val = (double *)malloc(sizeof(double) * 4 * nv);
    long *umap = (long *)malloc(sizeof(long) * nv);
    double *gb = (double *)malloc(sizeof(double) * nv), *pb = (double *)malloc(sizeof(double) * nv);
    int st = ORC_ERR_OOM;
    if (colptr && rowidx && val && umap && gb && pb) {
        long n, nnz;
        st = orc_ic0_ordered(h->nx, h->ny, h->nz, h->mask, d, h->beta, order, colptr, rowidx, val, umap, &n, &nnz);
        if (st == ORC_OK) {
            for (long u = 0; u < n; ++u) gb[u] = g[umap[u]];
            orc_ic0_solve(n, colptr, rowidx, val, gb, pb);
            for (long j = 0; j < nv; ++j) p[j] = 0.0;
            for (long u = 0; u < n; ++u) p[umap[u]] = pb[u];
        }
    }
    free(colptr); free(rowidx); free(val); free(umap); free(gb); free(pb);
    return st;
}

int orc_precondition(const orc_t *h, const double *d, const double *g, double *p) {
    return orc_precondition_ordered(h, d, g, p, 0);
}

/* ---------------------------------------------------------------------------------
 * IC with a drop tolerance (Sec. III-B: the paper's L_t and its NCG-MLS-IC).  Incomplete
 * Cholesky of H = diag(d) + beta C'C over the mask voxels in natural order, computed
 * column by column (left-looking): column j of L is H(j:, j) minus L(j:, k) L_jk summed
 * over the earlier columns k with L_jk != 0, divided by L_jj = sqrt of its diagonal
 * entry.  Every off-diagonal entry -- an entry of H or fill-in -- whose magnitude is
 * below tau is set to zero as soon as it is computed, so later columns use the dropped
 * factor; the diagonal is never dropped.  tau = 0 gives the complete Cholesky factor.
 * On success *colptr, *rowidx, *val (L in compressed-column form, diagonal first, rows
 * ascending) and *umap (voxel of each unknown) are malloc'ed: release them with orc_free.
 * ------------------------------------------------------------------------------- */
void orc_free(void *p) { free(p); }

static int cmp_long(const void *a, const void *b) {
    long x = *(const long *)a, y = *(const long *)b;
    return (x > y) - (x < y);
}

int orc_ict(int nx, int ny, int nz, const unsigned char *mask, const double *d, double beta, double tau,
            long **colptr_out, long **rowidx_out, double **val_out, long **umap_out, long *n_out,
            long *nnz_out) {
    long nv = (long)nx * ny * nz, nxy = (long)nx * ny;
    long *uidx = (long *)malloc(sizeof(long) * nv), *umap = (long *)malloc(sizeof(long) * nv);
    long n = 0;
    if (!uidx || !umap) { free(uidx); free(umap); return ORC_ERR_OOM; }
    for (long j = 0; j < nv; ++j) {
        if (mask == NULL || mask[j]) { uidx[j] = n; umap[n++] = j; } else { uidx[j] = -1; }
    }
    long cap = 8 * n + 16, nnz = 0;
    long *colptr = (long *)malloc(sizeof(long) * (n + 1));
    long *rowidx = (long *)malloc(sizeof(long) * cap);
    double *val = (double *)malloc(sizeof(double) * cap);
    /* row lists: for every row i, its entries L_ik (k < i) in increasing k, threaded
       through the positions p of the column storage (nextp[p]; colof[p] = k) */
    long *nextp = (long *)malloc(sizeof(long) * cap), *colof = (long *)malloc(sizeof(long) * cap);
    long *rhead = (long *)malloc(sizeof(long) * (n ? n : 1)), *rtail = (long *)malloc(sizeof(long) * (n ? n : 1));
    double *w = (double *)calloc(n ? n : 1, sizeof(double));
    unsigned char *mark = (unsigned char *)calloc(n ? n : 1, 1);
    long *pat = (long *)malloc(sizeof(long) * (n ? n : 1));
    int st = ORC_OK;
    if (!colptr || !rowidx || !val || !nextp || !colof || !rhead || !rtail || !w || !mark || !pat) {
        st = ORC_ERR_OOM;
        goto fail;
    }
    for (long i = 0; i < n; ++i) rhead[i] = rtail[i] = -1;
    for (long j = 0; j < n; ++j) {
        long vj = umap[j];
        colptr[j] = nnz; /* also closes column j - 1, whose rows the loop below scans */
        long x = vj % nx, y = (vj / nx) % ny, z = vj / nxy;
        long nb[6] = {x > 0 ? vj - 1 : -1, x + 1 < nx ? vj + 1 : -1, y > 0 ? vj - nx : -1,
                      y + 1 < ny ? vj + nx : -1, z > 0 ? vj - nxy : -1, z + 1 < nz ? vj + nxy : -1};
        int cnt = 0;
        long np = 0;
        for (int q = 0; q < 6; ++q) if (nb[q] >= 0 && uidx[nb[q]] >= 0) ++cnt;
        /* scatter H(j:, j) */
        w[j] = d[vj] + beta * cnt;
        mark[j] = 1;
        pat[np++] = j;
        for (int q = 0; q < 6; ++q) {
            long u = nb[q] >= 0 ? uidx[nb[q]] : -1;
            if (u > j) { w[u] = -beta; mark[u] = 1; pat[np++] = u; }
        }
        /* subtract L(j:, k) L_jk for every earlier column k with L_jk kept */
        for (long pj = rhead[j]; pj >= 0; pj = nextp[pj]) {
            long k = colof[pj];
            double ljk = val[pj];
            for (long p = pj; p < colptr[k + 1]; ++p) { /* rows >= j of column k */
                long i = rowidx[p];
                if (!mark[i]) { mark[i] = 1; w[i] = 0.0; pat[np++] = i; }
                w[i] -= val[p] * ljk;
            }
        }
        if (!(w[j] > 0.0)) { st = ORC_ERR_NOT_PD; goto fail; }
        double ljj = sqrt(w[j]);
        if (np > 2) qsort(pat + 1, (size_t)(np - 1), sizeof(long), cmp_long);
        if (nnz + np > cap) {
            long nc = 2 * cap + np;
            long *r2 = (long *)realloc(rowidx, sizeof(long) * nc);
            if (r2) rowidx = r2;
            double *v2 = (double *)realloc(val, sizeof(double) * nc);
            if (v2) val = v2;
            long *n2 = (long *)realloc(nextp, sizeof(long) * nc);
            if (n2) nextp = n2;
            long *c2 = (long *)realloc(colof, sizeof(long) * nc);
            if (c2) colof = c2;
            if (!r2 || !v2 || !n2 || !c2) { st = ORC_ERR_OOM; goto fail; }
            cap = nc;
        }
        rowidx[nnz] = j;
        val[nnz] = ljj;
        ++nnz;
        for (long q = 1; q < np; ++q) {
            long i = pat[q];
            double c = w[i] / ljj;
            if (fabs(c) >= tau) { /* kept: append to row i's list */
                rowidx[nnz] = i;
                val[nnz] = c;
                colof[nnz] = j;
                nextp[nnz] = -1;
                if (rtail[i] >= 0) nextp[rtail[i]] = nnz; else rhead[i] = nnz;
                rtail[i] = nnz;
                ++nnz;
            }
        }
        for (long q = 0; q < np; ++q) { mark[pat[q]] = 0; w[pat[q]] = 0.0; }
    }
    colptr[n] = nnz;
    free(uidx); free(nextp); free(colof); free(rhead); free(rtail); free(w); free(mark); free(pat);
    *colptr_out = colptr; *rowidx_out = rowidx; *val_out = val; *umap_out = umap;
    *n_out = n; *nnz_out = nnz;
    return ORC_OK;
fail:
    free(uidx); free(umap); free(colptr); free(rowidx); free(val); free(nextp); free(colof);
    free(rhead); free(rtail); free(w); free(mark); free(pat);
    return st;
}

/* H_max of Sec. III-B: the largest |H_jk| of H = diag(d) + beta C'C over the mask voxels */
double orc_hmax(const orc_t *h, const double *d) {
    double m = 0.0;
    for (long j = 0; j < h->nv; ++j) {
        if (!h->mask[j]) continue;
        int cnt = 0;
        for (int ax = 0; ax < 3; ++ax) cnt += (fwd_nbr(h, j, ax) >= 0) + (bwd_nbr(h, j, ax) >= 0);
        double hjj = fabs(d[j] + h->beta * cnt);
        if (hjj > m) m = hjj;
        if (cnt > 0 && fabs(h->beta) > m) m = fabs(h->beta);
    }
    return m;
}

void orc_set_droptol(orc_t *h, double droptol) { h->droptol = droptol; }

/* p = (L L')^{-1} g with the drop-tolerance factor of H(w) = diag(d) + beta C'C, absolute
 * tolerance tau; voxel-indexed arrays */
int orc_precondition_ict(const orc_t *h, const double *d, const double *g, double *p, double tau) {
    long *colptr = NULL, *rowidx = NULL, *umap = NULL, n = 0, nnz = 0;
    double *val = NULL;
    int st = orc_ict(h->nx, h->ny, h->nz, h->mask, d, h->beta, tau, &colptr, &rowidx, &val, &umap, &n, &nnz);
    if (st != ORC_OK) return st;
    double *gb = (double *)malloc(sizeof(double) * (n ? n : 1)), *pb = (double *)malloc(sizeof(double) * (n ? n : 1));
    if (!gb || !pb) {
        st = ORC_ERR_OOM;
    } else {
        for (long u = 0; u < n; ++u) gb[u] = g[umap[u]];
        orc_ic0_solve(n, colptr, rowidx, val, gb, pb);
        for (long j = 0; j < h->nv; ++j) p[j] = 0.0;
        for (long u = 0; u < n; ++u) p[umap[u]] = pb[u];
    }
    free(gb); free(pb); free(colptr); free(rowidx); free(val); free(umap);
    return st;
}

/* ---------------------------------------------------------------------------------
 * Preconditioned NCG with the monotonic line search (Algorithm box, Eq. 13-16).
 * w: [nv] in/out (read as the start point unless init != 0, which applies Eq. 6).
 * cost_hist [niter+1], alpha_hist [niter], mu_hist [niter], inner_cost [niter*nls]
 * (Psi after each inner step) may be NULL.  precond: 0 = IC(0), 1 = diagonal of H,
 * 2 = none, 3 = red-black IC(0), 4 = IC with the drop tolerance droptol * H_max.
 * ------------------------------------------------------------------------------- */
int orc_solve(const orc_t *h, double *w, int init, int niter, int nls, int precond, double *cost_hist,
              double *alpha_hist, double *mu_hist, double *inner_cost) {
    long nv = h->nv;
    double *g = (double *)calloc(nv, sizeof(double)), *gprev = (double *)calloc(nv, sizeof(double));
    double *d = (double *)calloc(nv, sizeof(double)), *p = (double *)calloc(nv, sizeof(double));
    double *z = (double *)calloc(nv, sizeof(double)), *wk = (double *)calloc(nv, sizeof(double));
    double *gk = (double *)calloc(nv, sizeof(double));
    int st = ORC_OK;
    if (!g || !gprev || !d || !p || !z || !wk || !gk) { st = ORC_ERR_OOM; goto done; }
    if (init) orc_init(h, w);
    for (long j = 0; j < nv; ++j) if (!h->mask[j]) w[j] = 0.0;
    if (cost_hist) cost_hist[0] = orc_cost(h, w);
    double gp_prev = 0.0;
    for (int i = 0; i < niter; ++i) {
        orc_grad(h, w, g);
        orc_curv(h, w, d);
        if (precond == 0 || precond == 3) {
            st = orc_precondition_ordered(h, d, g, p, precond == 3 ? 1 : 0);
            if (st != ORC_OK) goto done;
        } else if (precond == 4) { /* tolerance H_max^i * droptol, this iteration's H */
            st = orc_precondition_ict(h, d, g, p, h->droptol * orc_hmax(h, d));
            if (st != ORC_OK) goto done;
        } else {
            for (long j = 0; j < nv; ++j) {
                if (!h->mask[j]) { p[j] = 0.0; continue; }
                if (precond == 2) { p[j] = g[j]; continue; }
                int cnt = 0;
                for (int ax = 0; ax < 3; ++ax) cnt += (fwd_nbr(h, j, ax) >= 0) + (bwd_nbr(h, j, ax) >= 0);
                double hjj = d[j] + h->beta * cnt;
                if (!(hjj > 0.0)) { st = ORC_ERR_NOT_PD; goto done; }
                p[j] = g[j] / hjj;
            }
        }
        double gp = dot(nv, g, p), gprevp = dot(nv, gprev, p);
        double mu = 0.0;
        if (i > 0 && gp_prev != 0.0) mu = (gp - gprevp) / gp_prev;
        for (long j = 0; j < nv; ++j) z[j] = -p[j] + mu * z[j];
        double cz2 = edge_dot(h, z, z), a = edge_dot(h, z, w);
        double alpha = 0.0;
        for (int k = 0; k < nls; ++k) {
            for (long j = 0; j < nv; ++j) wk[j] = w[j] + alpha * z[j];
            orc_grad_phi(h, wk, gk);
            orc_curv(h, wk, d);
            for (long j = 0; j < nv; ++j) wk[j] = z[j] * z[j] * d[j];
            double fp = dot(nv, z, gk), D = sum(nv, wk);
            fp += h->beta * (a + alpha * cz2);
            double den = D + h->beta * cz2;
            if (den == 0.0) { alpha = 0.0; break; }
            alpha = alpha - fp / den;
            if (inner_cost) {
                for (long j = 0; j < nv; ++j) wk[j] = w[j] + alpha * z[j];
                inner_cost[(long)i * nls + k] = orc_cost(h, wk);
            }
        }
        for (long j = 0; j < nv; ++j) w[j] += alpha * z[j];
        for (long j = 0; j < nv; ++j) gprev[j] = g[j];
        gp_prev = gp;
        if (alpha_hist) alpha_hist[i] = alpha;
        if (mu_hist) mu_hist[i] = mu;
        if (cost_hist) cost_hist[i + 1] = orc_cost(h, w);
    }
done:
    free(g); free(gprev); free(d); free(p); free(z); free(wk); free(gk);
    return st;
}

/* One voxel's data-term pieces straight from its raw data (for sampled checks on
 * volumes too large for the grid functions).  y_vox: [L][nc] complex, s_vox: [nc]
 * complex or NULL.  out = {phi_j, dphi_j, d_j}. */
int orc_voxel(int nc, int L, const double *te, const double *y_vox, const double *s_vox, double w,
              double *out) {
    if (nc < 1 || L < 2 || L > ORC_MAXL) return ORC_ERR_ARG;
    long T = (long)nc * nc * L * L;
    double *ra = (double *)malloc(sizeof(double) * T), *rg = (double *)malloc(sizeof(double) * T);
    double *dt = (double *)malloc(sizeof(double) * T);
    if (!ra || !rg || !dt) { free(ra); free(rg); free(dt); return ORC_ERR_OOM; }
    pair_weights(nc, L, y_vox, 2, s_vox, 2, NULL, ra, rg);
    tuple_dt(nc, L, te, dt);
    voxel_terms(T, ra, rg, dt, w, out, out + 1, out + 2);
    free(ra); free(rg); free(dt);
    return ORC_OK;
}

/* Curvature d_j of Eq. 10 at w for every voxel of a volume straight from its raw data,
 * voxel by voxel (r of Eq. 3 formed per voxel, nothing kept): for volumes whose precomputed
 * r (orc_create) would not fit in host memory.  y: [L][nc][nv] complex, s: [nc][nv] complex
 * or NULL, mask: [nv] or NULL; out: [nv], 0 outside the mask. */
int orc_curv_raw(int nx, int ny, int nz, int nc, int L, const double *y, const double *s, const double *te,
                 const unsigned char *mask, const double *w, double *out) {
    if (nx < 1 || ny < 1 || nz < 1 || nc < 1 || L < 2 || L > ORC_MAXL || !y || !te || !w || !out) return ORC_ERR_ARG;
    if (!s && nc != 1) return ORC_ERR_ARG;
    long nv = (long)nx * ny * nz, T = (long)nc * nc * L * L;
    double *dt = (double *)malloc(sizeof(double) * T);
    if (!dt) return ORC_ERR_OOM;
    tuple_dt(nc, L, te, dt);
    int st = ORC_OK;
#pragma omp parallel if (g_threads > 1) num_threads(g_threads)
    {
        double *ra = (double *)malloc(sizeof(double) * T), *rg = (double *)malloc(sizeof(double) * T);
        if (!ra || !rg) {
#pragma omp atomic write
            st = ORC_ERR_OOM;
        }
#pragma omp for schedule(dynamic, 256)
        for (long j = 0; j < nv; ++j) {
            if ((mask && !mask[j]) || !ra || !rg) { out[j] = 0.0; continue; }
            pair_weights(nc, L, y + 2 * j, 2 * nv, s ? s + 2 * j : NULL, 2 * nv, NULL, ra, rg);
            voxel_terms(T, ra, rg, dt, w[j], NULL, NULL, out + j);
        }
        free(ra);
        free(rg);
    }
    free(dt);
    return st;
}

/* raw r_cdmnj of Eq. 3 for one voxel (modulus, angle), T = nc*nc*L*L, order c,d,m,n */
int orc_voxel_r(int nc, int L, const double *y_vox, const double *s_vox, double *rabs, double *rang) {
    if (nc < 1 || L < 2 || L > ORC_MAXL) return ORC_ERR_ARG;
    pair_weights(nc, L, y_vox, 2, s_vox, 2, NULL, rabs, rang);
    return ORC_OK;
}
