/*
 * FP64 CPU oracle for the complex-valued holographic Gaussian renderer.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  It shares no code,
 * header, table or helper with the CUDA path.
 *
 * Everything is plain double precision, written step by step from the paper
 * (arXiv 2506.08350):
 *   - activation and projection: Eq. gaussian_density, Eq. gaussian_decompose,
 *     Eq. gaussian_projection and Eq. gaussian_projection_2d (Sec. 3), the
 *     exponent term of Supp. D.3;
 *   - plane assignment by argmax: Eq. hard_assignment (Sec. 4.1);
 *   - complex per-plane compositing: the per-plane field equation of Sec. 4.1
 *     and Algorithm 2 (effective alpha, complex scale, transmittance update,
 *     early termination after the add);
 *   - adjoints: Supp. D.4, re-derived here in reverse mode from the forward
 *     definition (the paper's chain is used as a cross-check, not as code).
 *
 * Readings of the paper taken here (the same list is kept in the design notes):
 *   R1 default order front-to-back (nearest first), order=1 back-to-front;
 *   R2 only same-plane Gaussians attenuate;  R3 G counted once in alpha;
 *   R4 support of Gaussian n = {p : o_n G_n(p) >= alpha_min}, independent of
 *      any tiling, alpha = min(alpha_max, o G), stop when T < T_eps after the add;
 *   R5 scale = exp(log_scale), opacity = sigmoid(logit);
 *   R6 argmax ties -> lowest plane index; STE backward is the elementwise
 *      product with softmax(rho'/tau);
 *   R7 only the assigned plane's rho receives gradient;
 *   R8 2D covariance dilation, J clamp, near-plane cull as options;
 *   R14 sort key = camera-space z of the mean, ties by index.
 *
 * The search for candidate Gaussians of a pixel uses a uniform grid of 8x8
 * pixel cells built from each Gaussian's support bounding box.  It only
 * narrows the candidates: every candidate is still tested per pixel with the
 * exact support rule, so the result is the per-pixel definition.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define CELL 8

/* opt[] layout (all doubles):
 *   0 alpha_min, 1 alpha_max, 2 T_eps, 3 dilation (px^2), 4 near_z (m),
 *   5 clip factor (<= 0: J is not clamped), 6 order (0 front-to-back, 1 back-to-front),
 *   7 ste tau */
enum { O_AMIN = 0, O_AMAX, O_TEPS, O_DIL, O_NEAR, O_CLIP, O_ORDER, O_TAU };

/* ---------- small dense helpers (row-major) ---------- */
static void quat_to_rot(const double q[4], double R[9]) {
    /* unit quaternion (w, x, y, z) -> rotation matrix */
    double w = q[0], x = q[1], y = q[2], z = q[3];
    R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
    R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
    R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
}

/* Everything the projection of one Gaussian produces, plus the intermediates
 * its adjoint needs. */
typedef struct {
    int valid;
    double qn[4], qnorm, R[9], s[3], Sigma[9];
    double t[3], tcx, tcy;   /* camera-space mean; clamped x, y used in J */
    int clx, cly;            /* which of x, y were clamped: 0 no, +1 / -1 side */
    double J[6], T[6];       /* J (2x3), T = J W3 (2x3) */
    double cov[3];           /* Sigma' (a, b, c) after dilation */
    double det, conic[3], mu[2], depth, opac;
} proj_t;

static void project_one(int H, int W, const double* mean, const double* log_s, const double* quat, double logit,
                        const double* Vm, const double* intr, const double* opt, proj_t* P) {
    memset(P, 0, sizeof(*P));
    double fx = intr[0], fy = intr[1], cx = intr[2], cy = intr[3];
    /* world -> camera: t = W3 x + tvec (Vm is 4x4 row-major) */
    for (int i = 0; i < 3; i++)
        P->t[i] = Vm[4 * i + 0] * mean[0] + Vm[4 * i + 1] * mean[1] + Vm[4 * i + 2] * mean[2] + Vm[4 * i + 3];
    P->depth = P->t[2];
    if (!(P->t[2] >= opt[O_NEAR])) { P->valid = 0; return; }
    /* activations */
    double qn2 = quat[0] * quat[0] + quat[1] * quat[1] + quat[2] * quat[2] + quat[3] * quat[3];
    P->qnorm = sqrt(qn2);
    for (int i = 0; i < 4; i++) P->qn[i] = quat[i] / P->qnorm;
    quat_to_rot(P->qn, P->R);
    for (int i = 0; i < 3; i++) P->s[i] = exp(log_s[i]);
    P->opac = 1.0 / (1.0 + exp(-logit));
    /* Sigma = R S S^T R^T */
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            double acc = 0;
            for (int k = 0; k < 3; k++) acc += P->R[3 * i + k] * P->s[k] * P->s[k] * P->R[3 * j + k];
            P->Sigma[3 * i + j] = acc;
        }
    /* Jacobian of the perspective projection at the (optionally clamped) mean */
    double tz = P->t[2];
    P->tcx = P->t[0]; P->tcy = P->t[1];
    if (opt[O_CLIP] > 0) {
        double limx = opt[O_CLIP] * (0.5 * W) / fx; /* clip * tan(half field of view) */
        double limy = opt[O_CLIP] * (0.5 * H) / fy;
        double rx = P->t[0] / tz, ry = P->t[1] / tz;
        if (rx > limx) { P->tcx = limx * tz; P->clx = 1; }
        else if (rx < -limx) { P->tcx = -limx * tz; P->clx = -1; }
        if (ry > limy) { P->tcy = limy * tz; P->cly = 1; }
        else if (ry < -limy) { P->tcy = -limy * tz; P->cly = -1; }
    }
    P->J[0] = fx / tz; P->J[1] = 0;       P->J[2] = -fx * P->tcx / (tz * tz);
    P->J[3] = 0;       P->J[4] = fy / tz; P->J[5] = -fy * P->tcy / (tz * tz);
    for (int i = 0; i < 2; i++)
        for (int j = 0; j < 3; j++) {
            double acc = 0;
            for (int k = 0; k < 3; k++) acc += P->J[3 * i + k] * Vm[4 * k + j];
            P->T[3 * i + j] = acc;
        }
    /* Sigma' = T Sigma T^T + dilation I */
    double TS[6];
    for (int i = 0; i < 2; i++)
        for (int j = 0; j < 3; j++) {
            double acc = 0;
            for (int k = 0; k < 3; k++) acc += P->T[3 * i + k] * P->Sigma[3 * k + j];
            TS[3 * i + j] = acc;
        }
    double c2[4];
    for (int i = 0; i < 2; i++)
        for (int j = 0; j < 2; j++) {
            double acc = 0;
            for (int k = 0; k < 3; k++) acc += TS[3 * i + k] * P->T[3 * j + k];
            c2[2 * i + j] = acc;
        }
    P->cov[0] = c2[0] + opt[O_DIL];
    P->cov[1] = 0.5 * (c2[1] + c2[2]);
    P->cov[2] = c2[3] + opt[O_DIL];
    P->det = P->cov[0] * P->cov[2] - P->cov[1] * P->cov[1];
    if (!(P->det > 0)) { P->valid = 0; return; }
    P->conic[0] = P->cov[2] / P->det;
    P->conic[1] = -P->cov[1] / P->det;
    P->conic[2] = P->cov[0] / P->det;
    P->mu[0] = fx * P->t[0] / tz + cx;
    P->mu[1] = fy * P->t[1] / tz + cy;
    P->valid = 1;
}

static int argmax_plane(const double* logits, int L) {
    int best = 0;
    for (int l = 1; l < L; l++)
        if (logits[l] > logits[best]) best = l; /* ties keep the lowest index */
    return best;
}

/*
 * Project N Gaussians for one view.
 * Outputs per Gaussian: mu[2], conic[3], cov[3], opac, depth, plane, w[C][2]
 * (w = c e^{j phi}), bbox[4] (support box x0, x1, y0, y1 in pixels), valid.
 */
void oracle_project(int N, int L, int C, int H, int W,
                    const double* means, const double* log_scales, const double* quats,
                    const double* opacity_logits, const double* amplitude, const double* phase,
                    const double* plane_logits, const double* viewmat, const double* intr,
                    const double* opt,
                    double* mu, double* conic, double* cov, double* opac, double* depth,
                    int* plane, double* w, double* bbox, int* valid) {
#pragma omp parallel for schedule(static)
    for (int n = 0; n < N; n++) {
        proj_t P;
        project_one(H, W, means + 3 * n, log_scales + 3 * n, quats + 4 * n, opacity_logits[n], viewmat, intr, opt, &P);
        valid[n] = P.valid;
        depth[n] = P.depth;
        plane[n] = argmax_plane(plane_logits + (size_t)L * n, L);
        for (int c = 0; c < C; c++) {
            w[2 * (C * n + c) + 0] = amplitude[C * n + c] * cos(phase[C * n + c]);
            w[2 * (C * n + c) + 1] = amplitude[C * n + c] * sin(phase[C * n + c]);
        }
        mu[2 * n] = P.mu[0]; mu[2 * n + 1] = P.mu[1];
        for (int k = 0; k < 3; k++) { conic[3 * n + k] = P.conic[k]; cov[3 * n + k] = P.cov[k]; }
        opac[n] = P.opac;
        /* bounding box of the support ellipse {d : d^T conic d <= 2 ln(o / alpha_min)} */
        if (!P.valid) { bbox[4 * n] = 1; bbox[4 * n + 1] = 0; bbox[4 * n + 2] = 1; bbox[4 * n + 3] = 0; continue; }
        if (opt[O_AMIN] > 0) {
            if (P.opac < opt[O_AMIN]) { bbox[4 * n] = 1; bbox[4 * n + 1] = 0; bbox[4 * n + 2] = 1; bbox[4 * n + 3] = 0; continue; }
            double k = 2.0 * log(P.opac / opt[O_AMIN]);
            double rx = sqrt(k * P.cov[0]) + 1e-9, ry = sqrt(k * P.cov[2]) + 1e-9;
            bbox[4 * n] = P.mu[0] - rx; bbox[4 * n + 1] = P.mu[0] + rx;
            bbox[4 * n + 2] = P.mu[1] - ry; bbox[4 * n + 3] = P.mu[1] + ry;
        } else {
            bbox[4 * n] = -INFINITY; bbox[4 * n + 1] = INFINITY; bbox[4 * n + 2] = -INFINITY; bbox[4 * n + 3] = INFINITY;
        }
    }
}

/* ---------- depth order ---------- */
/* The visiting order compares depth keys: the camera-space depth rounded
 * once to FP32 (the precision in which the order is decided; Gaussians whose
 * keys are equal are visited by index). */
static const double* g_sort_depth;
static int cmp_front(const void* a, const void* b) {
    int i = *(const int*)a, j = *(const int*)b;
    const float di = (float)g_sort_depth[i], dj = (float)g_sort_depth[j];
    if (di < dj) return -1;
    if (di > dj) return 1;
    return (i > j) - (i < j);
}

/* Writes the visiting order: ascending (depth key, index) for front-to-back,
 * the exact reverse for back-to-front.  Only valid Gaussians are listed. */
int oracle_sort(int N, const double* depth, const int* valid, int order, int* out) {
    int m = 0;
    for (int n = 0; n < N; n++)
        if (valid[n]) out[m++] = n;
    g_sort_depth = depth;
    qsort(out, m, sizeof(int), cmp_front);
    if (order == 1)
        for (int i = 0; i < m / 2; i++) { int t = out[i]; out[i] = out[m - 1 - i]; out[m - 1 - i] = t; }
    return m;
}

/* ---------- candidate grid (search acceleration only) ---------- */
typedef struct {
    int gx, gy, L;
    int64_t* off;   /* [L][gy][gx] + 1 */
    int* idx;       /* Gaussian ids in visiting order */
} grid_t;

static void cell_range(const double* bb, int row0, int row1, int W, int* x0, int* x1, int* y0, int* y1) {
    double bx0 = bb[0], bx1 = bb[1], by0 = bb[2], by1 = bb[3];
    if (bx0 < 0) bx0 = 0;
    if (by0 < row0) by0 = row0;
    if (bx1 > W - 1) bx1 = W - 1;
    if (by1 > row1 - 1) by1 = row1 - 1;
    if (bx0 > bx1 || by0 > by1) { *x0 = 1; *x1 = 0; *y0 = 1; *y1 = 0; return; }
    *x0 = (int)floor(bx0) / CELL; *x1 = (int)floor(bx1) / CELL;
    *y0 = (int)floor(by0) / CELL; *y1 = (int)floor(by1) / CELL;
}

static void grid_build(grid_t* g, int L, int H, int W, int row0, int row1, int m, const int* ord,
                       const int* plane, const double* bbox) {
    g->gx = (W + CELL - 1) / CELL; g->gy = (H + CELL - 1) / CELL; g->L = L;
    size_t ncell = (size_t)L * g->gx * g->gy;
    g->off = (int64_t*)calloc(ncell + 1, sizeof(int64_t));
    for (int s = 0; s < m; s++) {
        int n = ord[s], x0, x1, y0, y1;
        cell_range(bbox + 4 * n, row0, row1, W, &x0, &x1, &y0, &y1);
        for (int y = y0; y <= y1; y++)
            for (int x = x0; x <= x1; x++) g->off[((size_t)plane[n] * g->gy + y) * g->gx + x + 1]++;
    }
    for (size_t i = 0; i < ncell; i++) g->off[i + 1] += g->off[i];
    g->idx = (int*)malloc(sizeof(int) * (g->off[ncell] > 0 ? g->off[ncell] : 1));
    int64_t* cur = (int64_t*)malloc(sizeof(int64_t) * (ncell > 0 ? ncell : 1));
    memcpy(cur, g->off, sizeof(int64_t) * ncell);
    for (int s = 0; s < m; s++) {
        int n = ord[s], x0, x1, y0, y1;
        cell_range(bbox + 4 * n, row0, row1, W, &x0, &x1, &y0, &y1);
        for (int y = y0; y <= y1; y++)
            for (int x = x0; x <= x1; x++) g->idx[cur[((size_t)plane[n] * g->gy + y) * g->gx + x]++] = n;
    }
    free(cur);
}

static void grid_free(grid_t* g) { free(g->off); free(g->idx); }

/* alpha of Gaussian n at pixel centre (x = j, y = i), per Algorithm 2 /
 * Supp. D.3: power = 1/2 d^T conic d, alpha = min(alpha_max, o exp(-power)). */
static inline double eval_alpha(const double* mu, const double* conic, double o, double x, double y,
                                double amax, double* G_out, double* dx_out, double* dy_out, int* clamped) {
    double dx = x - mu[0], dy = y - mu[1];
    double power = 0.5 * (conic[0] * dx * dx + 2.0 * conic[1] * dx * dy + conic[2] * dy * dy);
    double G = exp(-power);
    double a = o * G;
    *clamped = 0;
    if (a > amax) { a = amax; *clamped = 1; }
    *G_out = G; *dx_out = dx; *dy_out = dy;
    return a;
}

/*
 * Composite all planes of one view, for image rows row0 <= i < row1 (the
 * full image is row0 = 0, row1 = H; a band of rows is used to time a bounded
 * sample).  U[L][C][H][W][2], T_final[L][H][W], n_contrib[L][H][W] (number of Gaussians
 * that added to the pixel).  Per pixel and plane, in visiting order, Gaussians
 * of that plane whose alpha >= alpha_min add w alpha T; T <- T (1 - alpha);
 * the walk stops once T < T_eps (after the add).
 */
void oracle_composite(int N, int L, int C, int H, int W,
                      const double* mu, const double* conic, const double* opac,
                      const double* depth, const int* plane, const double* w,
                      const double* bbox, const int* valid, const double* opt,
                      int row0, int row1,
                      double* U, double* T_final, int* n_contrib) {
    int* ord = (int*)malloc(sizeof(int) * (N > 0 ? N : 1));
    int m = oracle_sort(N, depth, valid, (int)opt[O_ORDER], ord);
    grid_t g;
    grid_build(&g, L, H, W, row0, row1, m, ord, plane, bbox);
    const double amin = opt[O_AMIN], amax = opt[O_AMAX], teps = opt[O_TEPS];
#pragma omp parallel for collapse(2) schedule(dynamic, 4)
    for (int l = 0; l < L; l++)
        for (int i = row0; i < row1; i++) {
            double acc[2 * 16];
            for (int j = 0; j < W; j++) {
                size_t cell = ((size_t)l * g.gy + i / CELL) * g.gx + j / CELL;
                double T = 1.0;
                int cnt = 0;
                for (int c = 0; c < 2 * C; c++) acc[c] = 0;
                for (int64_t e = g.off[cell]; e < g.off[cell + 1]; e++) {
                    int n = g.idx[e];
                    double G, dx, dy; int cl;
                    double a = eval_alpha(mu + 2 * n, conic + 3 * n, opac[n], (double)j, (double)i, amax, &G, &dx, &dy, &cl);
                    if (a < amin) continue;
                    for (int c = 0; c < C; c++) {
                        acc[2 * c] += w[2 * (C * n + c)] * a * T;
                        acc[2 * c + 1] += w[2 * (C * n + c) + 1] * a * T;
                    }
                    T *= (1.0 - a);
                    cnt++;
                    if (T < teps) break;
                }
                for (int c = 0; c < C; c++) {
                    size_t o = ((((size_t)l * C + c) * H + i) * W + j) * 2;
                    U[o] = acc[2 * c]; U[o + 1] = acc[2 * c + 1];
                }
                T_final[((size_t)l * H + i) * W + j] = T;
                n_contrib[((size_t)l * H + i) * W + j] = cnt;
            }
        }
    grid_free(&g);
    free(ord);
}

/*
 * Adjoint of oracle_composite for one view.
 * gU[L][C][H][W][2] holds g = dL/dRe U + j dL/dIm U.  Accumulates (+=):
 *   g_mu[N][2], g_conic[N][3] (d/dA, d/dB, d/dC of conic (A, B; B, C), B counted once),
 *   g_opac[N] (w.r.t. the activated opacity o), g_w[N][C][2] (dL/dRe w, dL/dIm w).
 * For each pixel the contributors n_1..n_K (same walk as the forward) give
 *   dU/dalpha_k = w_k T_k - S_k / (1 - alpha_k),  S_k = sum_{m>k} w_m alpha_m T_m,
 *   dU/dw_k = alpha_k T_k;
 * a clamped alpha (= alpha_max) passes no gradient to o G.
 */
void oracle_composite_backward(int N, int L, int C, int H, int W,
                               const double* mu, const double* conic, const double* opac,
                               const double* depth, const int* plane, const double* w,
                               const double* bbox, const int* valid, const double* opt,
                               int row0, int row1,
                               const double* gU,
                               double* g_mu, double* g_conic, double* g_opac, double* g_w) {
    int* ord = (int*)malloc(sizeof(int) * (N > 0 ? N : 1));
    int m = oracle_sort(N, depth, valid, (int)opt[O_ORDER], ord);
    grid_t g;
    grid_build(&g, L, H, W, row0, row1, m, ord, plane, bbox);
    const double amin = opt[O_AMIN], amax = opt[O_AMAX], teps = opt[O_TEPS];
#pragma omp parallel
    {
        int cap = 1024;
        int* kn = (int*)malloc(sizeof(int) * cap);
        double* ka = (double*)malloc(sizeof(double) * cap);
        double* kT = (double*)malloc(sizeof(double) * cap);
        double* kG = (double*)malloc(sizeof(double) * cap);
        double* kdx = (double*)malloc(sizeof(double) * cap);
        double* kdy = (double*)malloc(sizeof(double) * cap);
        int* kcl = (int*)malloc(sizeof(int) * cap);
#pragma omp for collapse(2) schedule(dynamic, 4)
        for (int l = 0; l < L; l++)
            for (int i = row0; i < row1; i++)
                for (int j = 0; j < W; j++) {
                    size_t cell = ((size_t)l * g.gy + i / CELL) * g.gx + j / CELL;
                    double T = 1.0;
                    int K = 0;
                    for (int64_t e = g.off[cell]; e < g.off[cell + 1]; e++) {
                        int n = g.idx[e];
                        double G, dx, dy; int cl;
                        double a = eval_alpha(mu + 2 * n, conic + 3 * n, opac[n], (double)j, (double)i, amax, &G, &dx, &dy, &cl);
                        if (a < amin) continue;
                        if (K == cap) {
                            cap *= 2;
                            kn = (int*)realloc(kn, sizeof(int) * cap); ka = (double*)realloc(ka, sizeof(double) * cap);
                            kT = (double*)realloc(kT, sizeof(double) * cap); kG = (double*)realloc(kG, sizeof(double) * cap);
                            kdx = (double*)realloc(kdx, sizeof(double) * cap); kdy = (double*)realloc(kdy, sizeof(double) * cap);
                            kcl = (int*)realloc(kcl, sizeof(int) * cap);
                        }
                        kn[K] = n; ka[K] = a; kT[K] = T; kG[K] = G; kdx[K] = dx; kdy[K] = dy; kcl[K] = cl;
                        K++;
                        T *= (1.0 - a);
                        if (T < teps) break;
                    }
                    double gre[16], gim[16], S[2 * 16];
                    for (int c = 0; c < C; c++) {
                        size_t o = ((((size_t)l * C + c) * H + i) * W + j) * 2;
                        gre[c] = gU[o]; gim[c] = gU[o + 1];
                        S[2 * c] = 0; S[2 * c + 1] = 0;
                    }
                    for (int k = K - 1; k >= 0; k--) {
                        int n = kn[k];
                        double a = ka[k], Tk = kT[k];
                        double dLda = 0;
                        for (int c = 0; c < C; c++) {
                            double wr = w[2 * (C * n + c)], wi = w[2 * (C * n + c) + 1];
                            double dUr = wr * Tk - S[2 * c] / (1.0 - a);
                            double dUi = wi * Tk - S[2 * c + 1] / (1.0 - a);
                            dLda += gre[c] * dUr + gim[c] * dUi;
#pragma omp atomic
                            g_w[2 * (C * n + c)] += gre[c] * a * Tk;
#pragma omp atomic
                            g_w[2 * (C * n + c) + 1] += gim[c] * a * Tk;
                            S[2 * c] += wr * a * Tk;
                            S[2 * c + 1] += wi * a * Tk;
                        }
                        if (kcl[k]) continue; /* alpha = alpha_max: flat in o G */
                        double G = kG[k], o = opac[n];
                        double dLdo = dLda * G;
                        double dLdpower = -dLda * o * G;
                        double dx = kdx[k], dy = kdy[k];
                        const double* K3 = conic + 3 * n;
                        /* power = 1/2 (A dx^2 + 2 B dx dy + C dy^2), d = p - mu */
                        double gmx = -dLdpower * (K3[0] * dx + K3[1] * dy);
                        double gmy = -dLdpower * (K3[1] * dx + K3[2] * dy);
#pragma omp atomic
                        g_opac[n] += dLdo;
#pragma omp atomic
                        g_mu[2 * n] += gmx;
#pragma omp atomic
                        g_mu[2 * n + 1] += gmy;
#pragma omp atomic
                        g_conic[3 * n] += 0.5 * dx * dx * dLdpower;
#pragma omp atomic
                        g_conic[3 * n + 1] += dx * dy * dLdpower;
#pragma omp atomic
                        g_conic[3 * n + 2] += 0.5 * dy * dy * dLdpower;
                    }
                }
        free(kn); free(ka); free(kT); free(kG); free(kdx); free(kdy); free(kcl);
    }
    grid_free(&g);
    free(ord);
}

/*
 * Compositing with continuous plane weights rho[N][L] (the smooth extension of
 * the per-plane field used to define a dense plane-weight gradient): per
 * pixel and plane l, every visible Gaussian in visiting order, whatever its
 * assigned plane, with alpha = min(alpha_max, o G) >= alpha_min adds
 * w alpha rho_l T and T <- T (1 - alpha rho_l); the walk stops once
 * T < T_eps (after the add).  With one-hot rho this is oracle_composite.
 */
void oracle_composite_soft(int N, int L, int C, int H, int W,
                           const double* mu, const double* conic, const double* opac,
                           const double* depth, const double* rho, const double* w,
                           const double* bbox, const int* valid, const double* opt,
                           double* U, double* T_final) {
    int* ord = (int*)malloc(sizeof(int) * (N > 0 ? N : 1));
    int* zero = (int*)calloc(N > 0 ? N : 1, sizeof(int));
    int m = oracle_sort(N, depth, valid, (int)opt[O_ORDER], ord);
    grid_t g;
    grid_build(&g, 1, H, W, 0, H, m, ord, zero, bbox);
    const double amin = opt[O_AMIN], amax = opt[O_AMAX], teps = opt[O_TEPS];
#pragma omp parallel for collapse(2) schedule(dynamic, 4)
    for (int l = 0; l < L; l++)
        for (int i = 0; i < H; i++) {
            double acc[2 * 16];
            for (int j = 0; j < W; j++) {
                size_t cell = (size_t)(i / CELL) * g.gx + j / CELL;
                double T = 1.0;
                for (int c = 0; c < 2 * C; c++) acc[c] = 0;
                for (int64_t e = g.off[cell]; e < g.off[cell + 1]; e++) {
                    int n = g.idx[e];
                    double G, dx, dy; int cl;
                    double a = eval_alpha(mu + 2 * n, conic + 3 * n, opac[n], (double)j, (double)i, amax, &G, &dx, &dy, &cl);
                    if (a < amin) continue;
                    double ae = a * rho[(size_t)n * L + l];
                    if (ae == 0.0) continue;
                    for (int c = 0; c < C; c++) {
                        acc[2 * c] += w[2 * (C * n + c)] * ae * T;
                        acc[2 * c + 1] += w[2 * (C * n + c) + 1] * ae * T;
                    }
                    T *= (1.0 - ae);
                    if (T < teps) break;
                }
                for (int c = 0; c < C; c++) {
                    size_t o = ((((size_t)l * C + c) * H + i) * W + j) * 2;
                    U[o] = acc[2 * c]; U[o + 1] = acc[2 * c + 1];
                }
                T_final[((size_t)l * H + i) * W + j] = T;
            }
        }
    grid_free(&g);
    free(zero);
    free(ord);
}

/*
 * Dense plane-weight gradient of the hard-assignment compositing for one view:
 * drho[N][L] (+=) is dL/drho_{n,l} of oracle_composite_soft at the one-hot rho
 * of the argmax planes, for the planes l a Gaussian is NOT assigned to (the
 * assigned plane's value comes from oracle_composite_backward as o dL/do).
 * At rho_{n,l} = 0 Gaussian n adds nothing and attenuates nothing on plane l,
 * so for every pixel the plane-l walk reaches it at (alpha = min(alpha_max,
 * o G) >= alpha_min, the walk not yet stopped):
 *   dU_l/drho_{n,l} = o G (w_n T_l - S_l),
 * with T_l the plane's transmittance at n's place in the visiting order and
 * S_l the sum of the plane's contributions behind it (d alpha_eff / d rho =
 * o G: the alpha_max clamp is inactive at rho = 0).
 */
void oracle_composite_rho_dense(int N, int L, int C, int H, int W,
                                const double* mu, const double* conic, const double* opac,
                                const double* depth, const int* plane, const double* w,
                                const double* bbox, const int* valid, const double* opt,
                                const double* gU, double* drho) {
    int* ord = (int*)malloc(sizeof(int) * (N > 0 ? N : 1));
    int* zero = (int*)calloc(N > 0 ? N : 1, sizeof(int));
    int m = oracle_sort(N, depth, valid, (int)opt[O_ORDER], ord);
    grid_t g;
    grid_build(&g, 1, H, W, 0, H, m, ord, zero, bbox);
    const double amin = opt[O_AMIN], amax = opt[O_AMAX], teps = opt[O_TEPS];
#pragma omp parallel
    {
        int cap = 1024;
        int* vn = (int*)malloc(sizeof(int) * cap);       /* virtual entries: Gaussian,  */
        double* vg = (double*)malloc(sizeof(double) * cap); /* o G, T at its place,      */
        double* vT = (double*)malloc(sizeof(double) * cap);
        double* vP = (double*)malloc(sizeof(double) * 2 * 16 * cap); /* prefix of the plane's field */
#pragma omp for collapse(2) schedule(dynamic, 4)
        for (int l = 0; l < L; l++)
            for (int i = 0; i < H; i++)
                for (int j = 0; j < W; j++) {
                    size_t cell = (size_t)(i / CELL) * g.gx + j / CELL;
                    double T = 1.0, pre[2 * 16];
                    for (int c = 0; c < 2 * C; c++) pre[c] = 0;
                    int K = 0;
                    for (int64_t e = g.off[cell]; e < g.off[cell + 1]; e++) {
                        int n = g.idx[e];
                        double G, dx, dy; int cl;
                        double a = eval_alpha(mu + 2 * n, conic + 3 * n, opac[n], (double)j, (double)i, amax, &G, &dx, &dy, &cl);
                        if (a < amin) continue;
                        if (plane[n] == l) {
                            for (int c = 0; c < C; c++) {
                                pre[2 * c] += w[2 * (C * n + c)] * a * T;
                                pre[2 * c + 1] += w[2 * (C * n + c) + 1] * a * T;
                            }
                            T *= (1.0 - a);
                            if (T < teps) break;
                        } else {
                            if (K == cap) {
                                cap *= 2;
                                vn = (int*)realloc(vn, sizeof(int) * cap);
                                vg = (double*)realloc(vg, sizeof(double) * cap);
                                vT = (double*)realloc(vT, sizeof(double) * cap);
                                vP = (double*)realloc(vP, sizeof(double) * 2 * 16 * cap);
                            }
                            vn[K] = n; vg[K] = opac[n] * G; vT[K] = T;
                            for (int c = 0; c < 2 * C; c++) vP[(size_t)K * 32 + c] = pre[c];
                            K++;
                        }
                    }
                    /* the plane's whole field; S = field - prefix at each virtual entry */
                    for (int k = 0; k < K; k++) {
                        int n = vn[k];
                        double d = 0;
                        for (int c = 0; c < C; c++) {
                            size_t o = ((((size_t)l * C + c) * H + i) * W + j) * 2;
                            double Sr = pre[2 * c] - vP[(size_t)k * 32 + 2 * c];
                            double Si = pre[2 * c + 1] - vP[(size_t)k * 32 + 2 * c + 1];
                            double dUr = w[2 * (C * n + c)] * vT[k] - Sr;
                            double dUi = w[2 * (C * n + c) + 1] * vT[k] - Si;
                            d += gU[o] * dUr + gU[o + 1] * dUi;
                        }
#pragma omp atomic
                        drho[(size_t)n * L + l] += vg[k] * d;
                    }
                }
        free(vn); free(vg); free(vT); free(vP);
    }
    grid_free(&g);
    free(zero);
    free(ord);
}

/*
 * Adjoint of oracle_project for one view, accumulating (+=) into the
 * parameter gradients.  Inputs are the per-Gaussian 2D gradients of
 * oracle_composite_backward.  The plane-logit gradient follows the
 * straight-through estimator of Eq. ste: dL/drho'_n = dL/drho_n (elementwise)
 * softmax(rho'_n / tau), with dL/drho_{n,l} = o dL/do at the assigned plane
 * (alpha = o G rho, rho = 1 there) and 0 elsewhere.
 */
void oracle_project_backward(int N, int L, int C, int H, int W,
                             const double* means, const double* log_scales, const double* quats,
                             const double* opacity_logits, const double* amplitude, const double* phase,
                             const double* plane_logits, const double* viewmat, const double* intr,
                             const double* opt,
                             const double* g_mu, const double* g_conic, const double* g_opac, const double* g_w,
                             double* gm, double* gls, double* gq, double* gol, double* gamp, double* gph, double* gpl) {
    const double* Vm = viewmat;
    double fx = intr[0], fy = intr[1];
#pragma omp parallel for schedule(static)
    for (int n = 0; n < N; n++) {
        proj_t P;
        project_one(H, W, means + 3 * n, log_scales + 3 * n, quats + 4 * n, opacity_logits[n], Vm, intr, opt, &P);
        /* appearance: w_c = a_c (cos phi_c, sin phi_c) */
        for (int c = 0; c < C; c++) {
            double ph = phase[C * n + c], am = amplitude[C * n + c];
            double gr = g_w[2 * (C * n + c)], gi = g_w[2 * (C * n + c) + 1];
            gamp[C * n + c] += gr * cos(ph) + gi * sin(ph);
            gph[C * n + c] += am * (-gr * sin(ph) + gi * cos(ph));
        }
        if (!P.valid) continue;
        /* opacity: o = sigmoid(logit) */
        double o = P.opac;
        gol[n] += g_opac[n] * o * (1.0 - o);
        /* plane logits (STE) */
        {
            int a = argmax_plane(plane_logits + (size_t)L * n, L);
            double drho = o * g_opac[n];
            double tau = opt[O_TAU];
            const double* r = plane_logits + (size_t)L * n;
            double mx = r[0];
            for (int l = 1; l < L; l++) if (r[l] > mx) mx = r[l];
            double Z = 0;
            for (int l = 0; l < L; l++) Z += exp((r[l] - mx) / tau);
            gpl[(size_t)L * n + a] += drho * exp((r[a] - mx) / tau) / Z;
        }
        /* conic -> Sigma' : dL/dSigma' = -K G_K K, G_K symmetric with off-diagonal dB/2 */
        double Kc[4] = {P.conic[0], P.conic[1], P.conic[1], P.conic[2]};
        double GK[4] = {g_conic[3 * n], 0.5 * g_conic[3 * n + 1], 0.5 * g_conic[3 * n + 1], g_conic[3 * n + 2]};
        double tmp[4], GS2[4];
        for (int i = 0; i < 2; i++)
            for (int j = 0; j < 2; j++) tmp[2 * i + j] = Kc[2 * i] * GK[j] + Kc[2 * i + 1] * GK[2 + j];
        for (int i = 0; i < 2; i++)
            for (int j = 0; j < 2; j++) GS2[2 * i + j] = -(tmp[2 * i] * Kc[j] + tmp[2 * i + 1] * Kc[2 + j]);
        /* Sigma' = T Sigma T^T (+ const): dL/dSigma = T^T G T, dL/dT = 2 G T Sigma */
        double GSig[9], GT[6];
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) {
                double acc = 0;
                for (int a = 0; a < 2; a++)
                    for (int b = 0; b < 2; b++) acc += P.T[3 * a + i] * GS2[2 * a + b] * P.T[3 * b + j];
                GSig[3 * i + j] = acc;
            }
        for (int a = 0; a < 2; a++)
            for (int j = 0; j < 3; j++) {
                double acc = 0;
                for (int b = 0; b < 2; b++)
                    for (int k = 0; k < 3; k++) acc += 2.0 * GS2[2 * a + b] * P.T[3 * b + k] * P.Sigma[3 * k + j];
                GT[3 * a + j] = acc;
            }
        /* T = J W3: dL/dJ = dL/dT W3^T */
        double GJ[6];
        for (int a = 0; a < 2; a++)
            for (int k = 0; k < 3; k++) {
                double acc = 0;
                for (int j = 0; j < 3; j++) acc += GT[3 * a + j] * Vm[4 * k + j];
                GJ[3 * a + k] = acc;
            }
        /* J and mu as functions of t */
        double tx = P.t[0], ty = P.t[1], tz = P.t[2];
        double gt[3] = {0, 0, 0};
        /* mu = (fx tx/tz + cx, fy ty/tz + cy) */
        gt[0] += g_mu[2 * n] * fx / tz;
        gt[1] += g_mu[2 * n + 1] * fy / tz;
        gt[2] += -g_mu[2 * n] * fx * tx / (tz * tz) - g_mu[2 * n + 1] * fy * ty / (tz * tz);
        /* J00 = fx/tz, J11 = fy/tz */
        gt[2] += -GJ[0] * fx / (tz * tz) - GJ[4] * fy / (tz * tz);
        /* J02 = -fx tcx / tz^2 with tcx = tx, or +-limx tz when clamped */
        if (P.clx == 0) { gt[0] += -GJ[2] * fx / (tz * tz); gt[2] += GJ[2] * 2.0 * fx * tx / (tz * tz * tz); }
        else            { gt[2] += GJ[2] * fx * P.tcx / (tz * tz * tz); } /* J02 = -fx (s lim)/tz */
        if (P.cly == 0) { gt[1] += -GJ[5] * fy / (tz * tz); gt[2] += GJ[5] * 2.0 * fy * ty / (tz * tz * tz); }
        else            { gt[2] += GJ[5] * fy * P.tcy / (tz * tz * tz); }
        /* t = W3 x + tvec */
        for (int k = 0; k < 3; k++) gm[3 * n + k] += Vm[k] * gt[0] + Vm[4 + k] * gt[1] + Vm[8 + k] * gt[2];
        /* Sigma = M M^T, M = R diag(s): dL/dM = 2 GSig M */
        double M[9], GM[9];
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) M[3 * i + j] = P.R[3 * i + j] * P.s[j];
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) {
                double acc = 0;
                for (int k = 0; k < 3; k++) acc += 2.0 * GSig[3 * i + k] * M[3 * k + j];
                GM[3 * i + j] = acc;
            }
        double GR[9];
        for (int j = 0; j < 3; j++) {
            double gs = 0;
            for (int i = 0; i < 3; i++) { GR[3 * i + j] = GM[3 * i + j] * P.s[j]; gs += GM[3 * i + j] * P.R[3 * i + j]; }
            gls[3 * n + j] += gs * P.s[j]; /* s = exp(log_s) */
        }
        /* R(qn) -> qn */
        double w = P.qn[0], x = P.qn[1], y = P.qn[2], z = P.qn[3];
        double gqn[4];
        gqn[0] = 2 * (-z * GR[1] + y * GR[2] + z * GR[3] - x * GR[5] - y * GR[6] + x * GR[7]);
        gqn[1] = 2 * (y * GR[1] + z * GR[2] + y * GR[3] - 2 * x * GR[4] - w * GR[5] + z * GR[6] + w * GR[7] - 2 * x * GR[8]);
        gqn[2] = 2 * (-2 * y * GR[0] + x * GR[1] + w * GR[2] + x * GR[3] + z * GR[5] - w * GR[6] + z * GR[7] - 2 * y * GR[8]);
        gqn[3] = 2 * (-2 * z * GR[0] - w * GR[1] + x * GR[2] + w * GR[3] - 2 * z * GR[4] + y * GR[5] + x * GR[6] + y * GR[7]);
        /* qn = q / |q| */
        double dot = 0;
        for (int k = 0; k < 4; k++) dot += P.qn[k] * gqn[k];
        for (int k = 0; k < 4; k++) gq[4 * n + k] += (gqn[k] - P.qn[k] * dot) / P.qnorm;
    }
}
