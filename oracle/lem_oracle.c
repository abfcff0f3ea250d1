/*
 * FP64 CPU oracle for local-expansion-move stereo (Taniai et al., "Continuous 3D
 * Label Stereo Matching using Local Expansion Moves", arXiv 1603.08328).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow reference that the
 * CUDA path is checked against.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg load it; the product library never does.  It
 * shares no code, header or table with the CUDA path.
 *
 * Everything is double precision, written for a reader to check against the
 * paper by eye:
 *   - preprocessing: gray-value x-gradient with the [-0.5 0 0.5] kernel
 *     (Sec. 3.2, data term), guide I/255 and its window mean / covariance
 *     (Eq. gf), contrast weights w_pq (smoothness term);
 *   - raw matching cost rho(s|f) with the warp s' = s - (a s_u + b s_v + c, 0)
 *     and linear interpolation of the right view (Eqs. warp / photofunc);
 *   - the data term phi_p(f) by definition (guided-filter aggregation, Eq. gf,
 *     count-normalised at the image border), and the paper's region scheme that
 *     computes phi_p(alpha) for all p in an expansion region at once through the
 *     filtering region M (Sec. 3.5);
 *   - the curvature smoothness term psi (Eqs. smooth_phi, smweight, smooth);
 *   - the binary expansion-move graph (footnote to Lemma 2: neighbours outside
 *     the region fold into unaries) with every term quantised as rne(S*x);
 *   - min-cut by Dinic's algorithm, an independent Edmonds-Karp, and exhaustive
 *     enumeration for tiny graphs, all returning the canonical cut (the nodes
 *     that can still reach the sink in the residual graph: the unique minimal
 *     switching set);
 *   - Algorithm 2 (iterative alpha_ij-expansion: propagation then randomised
 *     perturbation) and Algorithm 1 (grids x 16 disjoint groups, Eq. groupindex),
 *     with SplitMix64 (Steele, Lea, Flood 2014) random draws.
 *
 * Compile with -ffp-contract=off so no multiply-add is fused: the random
 * candidate labels must be bit-identical to the GPU's.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#else
static int omp_get_max_threads(void) { return 1; }
#endif

/* ------------------------------------------------------------------------- */
/* parameters and context                                                    */
/* ------------------------------------------------------------------------- */

typedef struct {
    int gf_radius;        /* r': local regression window W'_k is (2r'+1)^2       */
    double gf_eps;        /* e: (Sigma_k + e U)                                   */
    double tau_col;       /* truncation of the colour term                        */
    double tau_grad;      /* truncation of the gradient term                      */
    double alpha_grad;    /* alpha: weight of the gradient term                   */
    double lambda;        /* smoothness weight                                    */
    double tau_dis;       /* truncation of psi-bar                                */
    double eps_w;         /* lower bound of the contrast weight                   */
    double gamma;         /* contrast weight scale                                */
    double disp_min, disp_max;
    int n_levels;
    int cell[3];
    int k_prop[3];
    int k_rand[3];
    double quant_scale;   /* S in rne(S*x)                                        */
    uint64_t seed;
    int n_threads;        /* 0: OpenMP default                                    */
    int reverse_order;    /* visit the regions of a group in reverse order        */
    int visit;            /* candidates drawn per region visit (1: Algorithm 2)   */
    int k_cnn[3];         /* candidates per visit cell taken from the proposal map */
    int k_rans[3];        /* RANSAC plane candidates per visit (Algorithm 2, RANSAC proposal) */
    int data_term;        /* 0: guided filter (LE-GF), 1: bilateral weights (LE-BF)  */
    double bf_gamma;      /* LE-BF weight scale on 0..255 colours                    */
} lo_params;

typedef struct {
    int H, W;
    lo_params p;
    double *Lc;   /* H*W*4: R, G, B (0..255), x-gradient of gray (left)  */
    double *Rc;   /* same, right view                                   */
    double *mu;   /* H*W*3: window mean of the guide                    */
    double *A;    /* H*W*9: (Sigma_k + e U)^-1                          */
    double *wq;   /* H*W*4: max(w_pq, eps) for the 4 forward neighbours */
    float *lab;   /* H*W*3: current plane labels (a, b, c)              */
    double *cost; /* H*W: phi_p(f_p) for the current labels             */
    float *prop;  /* H*W*3: proposal map (a, b, c) or NULL              */
} lo_ctx;

/* forward neighbours: right, down-left, down, down-right (each unordered pair of
 * the 8-neighbourhood appears exactly once) */
static const int FDX[4] = {1, -1, 0, 1};
static const int FDY[4] = {0, 1, 1, 1};

static inline int imin(int a, int b) { return a < b ? a : b; }
static inline int imax(int a, int b) { return a > b ? a : b; }

/* ------------------------------------------------------------------------- */
/* preprocessing                                                             */
/* ------------------------------------------------------------------------- */

/* 3x3 inverse by Gauss-Jordan elimination with partial pivoting. */
static void inv3(const double *m, double *out) {
    double a[3][6];
    for (int i = 0; i < 3; i++) {
        for (int j = 0; j < 3; j++) {
            a[i][j] = m[3 * i + j];
            a[i][3 + j] = (i == j) ? 1.0 : 0.0;
        }
    }
    for (int c = 0; c < 3; c++) {
        int piv = c;
        for (int r = c + 1; r < 3; r++)
            if (fabs(a[r][c]) > fabs(a[piv][c])) piv = r;
        if (piv != c)
            for (int j = 0; j < 6; j++) {
                double t = a[c][j];
                a[c][j] = a[piv][j];
                a[piv][j] = t;
            }
        double d = a[c][c];
        for (int j = 0; j < 6; j++) a[c][j] /= d;
        for (int r = 0; r < 3; r++) {
            if (r == c) continue;
            double f = a[r][c];
            for (int j = 0; j < 6; j++) a[r][j] -= f * a[c][j];
        }
    }
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) out[3 * i + j] = a[i][3 + j];
}

/* gray value (BT.601 weights, not rounded) and its x-gradient with the
 * [-0.5 0 0.5] kernel; the border replicates the edge pixel */
static void pack_view(const double *rgb, int H, int W, double *out) {
    double *g = (double *)malloc(sizeof(double) * (size_t)W);
    for (int y = 0; y < H; y++) {
        for (int x = 0; x < W; x++) {
            const double *c = rgb + ((size_t)y * W + x) * 3;
            g[x] = 0.299 * c[0] + 0.587 * c[1] + 0.114 * c[2];
        }
        for (int x = 0; x < W; x++) {
            const double *c = rgb + ((size_t)y * W + x) * 3;
            double *o = out + ((size_t)y * W + x) * 4;
            int xm = imax(x - 1, 0), xp = imin(x + 1, W - 1);
            o[0] = c[0];
            o[1] = c[1];
            o[2] = c[2];
            o[3] = 0.5 * (g[xp] - g[xm]);
        }
    }
    free(g);
}

static void guide_stats(lo_ctx *c) {
    const int H = c->H, W = c->W, r = c->p.gf_radius;
    for (int ky = 0; ky < H; ky++) {
        for (int kx = 0; kx < W; kx++) {
            int x0 = imax(kx - r, 0), x1 = imin(kx + r, W - 1);
            int y0 = imax(ky - r, 0), y1 = imin(ky + r, H - 1);
            double n = 0, m[3] = {0, 0, 0};
            for (int y = y0; y <= y1; y++)
                for (int x = x0; x <= x1; x++) {
                    const double *l = c->Lc + ((size_t)y * W + x) * 4;
                    for (int ch = 0; ch < 3; ch++) m[ch] += l[ch] / 255.0;
                    n += 1;
                }
            for (int ch = 0; ch < 3; ch++) m[ch] /= n;
            /* population covariance, second pass around the mean */
            double S[9] = {0};
            for (int y = y0; y <= y1; y++)
                for (int x = x0; x <= x1; x++) {
                    const double *l = c->Lc + ((size_t)y * W + x) * 4;
                    double d[3];
                    for (int ch = 0; ch < 3; ch++) d[ch] = l[ch] / 255.0 - m[ch];
                    for (int i = 0; i < 3; i++)
                        for (int j = 0; j < 3; j++) S[3 * i + j] += d[i] * d[j];
                }
            for (int i = 0; i < 9; i++) S[i] /= n;
            for (int i = 0; i < 3; i++) S[4 * i] += c->p.gf_eps;
            size_t k = (size_t)ky * W + kx;
            for (int ch = 0; ch < 3; ch++) c->mu[k * 3 + ch] = m[ch];
            inv3(S, c->A + k * 9);
        }
    }
}

static void contrast_weights(lo_ctx *c) {
    const int H = c->H, W = c->W;
    for (int y = 0; y < H; y++)
        for (int x = 0; x < W; x++)
            for (int d = 0; d < 4; d++) {
                int qx = x + FDX[d], qy = y + FDY[d];
                double w = 0.0;
                if (qx >= 0 && qx < W && qy >= 0 && qy < H) {
                    const double *lp = c->Lc + ((size_t)y * W + x) * 4;
                    const double *lq = c->Lc + ((size_t)qy * W + qx) * 4;
                    double l1 = fabs(lp[0] - lq[0]) + fabs(lp[1] - lq[1]) + fabs(lp[2] - lq[2]);
                    w = exp(-l1 / c->p.gamma);
                    if (w < c->p.eps_w) w = c->p.eps_w;
                }
                c->wq[((size_t)y * W + x) * 4 + d] = w;
            }
}

static lo_ctx *create_common(const double *left, const double *right, int H, int W,
                             const lo_params *p) {
    lo_ctx *c = (lo_ctx *)calloc(1, sizeof(lo_ctx));
    c->H = H;
    c->W = W;
    c->p = *p;
    size_t n = (size_t)H * W;
    c->Lc = (double *)malloc(sizeof(double) * n * 4);
    c->Rc = (double *)malloc(sizeof(double) * n * 4);
    c->mu = (double *)malloc(sizeof(double) * n * 3);
    c->A = (double *)malloc(sizeof(double) * n * 9);
    c->wq = (double *)malloc(sizeof(double) * n * 4);
    c->lab = (float *)calloc(n * 3, sizeof(float));
    c->cost = (double *)calloc(n, sizeof(double));
    pack_view(left, H, W, c->Lc);
    pack_view(right, H, W, c->Rc);
    guide_stats(c);
    contrast_weights(c);
    return c;
}

/* Context from uint8 RGB images (H x W x 3, interleaved). */
lo_ctx *lo_create(const uint8_t *left, const uint8_t *right, int H, int W, const lo_params *p) {
    size_t n = (size_t)H * W * 3;
    double *l = (double *)malloc(sizeof(double) * n);
    double *r = (double *)malloc(sizeof(double) * n);
    for (size_t i = 0; i < n; i++) {
        l[i] = left[i];
        r[i] = right[i];
    }
    lo_ctx *c = create_common(l, r, H, W, p);
    free(l);
    free(r);
    return c;
}

/* Context from real-valued RGB images (0..255 scale), for closed-form checks. */
lo_ctx *lo_create_f64(const double *left, const double *right, int H, int W, const lo_params *p) {
    return create_common(left, right, H, W, p);
}

void lo_destroy(lo_ctx *c) {
    if (!c) return;
    free(c->Lc);
    free(c->Rc);
    free(c->mu);
    free(c->A);
    free(c->wq);
    free(c->lab);
    free(c->cost);
    free(c->prop);
    free(c);
}

/* Proposal map of the learned proposer: H*W*3 plane labels (a, b, c), copied;
 * NULL clears it.  The k_cnn[level] map candidates of a visit need it. */
void lo_set_proposals(lo_ctx *c, const float *abc) {
    size_t n = (size_t)c->H * c->W * 3;
    if (!abc) {
        free(c->prop);
        c->prop = NULL;
        return;
    }
    if (!c->prop) c->prop = (float *)malloc(sizeof(float) * n);
    memcpy(c->prop, abc, sizeof(float) * n);
}

/* Read-only views of the preprocessed planes, for the tests. */
void lo_get_planes(const lo_ctx *c, double *Lc, double *Rc, double *mu, double *A, double *wq) {
    size_t n = (size_t)c->H * c->W;
    if (Lc) memcpy(Lc, c->Lc, sizeof(double) * n * 4);
    if (Rc) memcpy(Rc, c->Rc, sizeof(double) * n * 4);
    if (mu) memcpy(mu, c->mu, sizeof(double) * n * 3);
    if (A) memcpy(A, c->A, sizeof(double) * n * 9);
    if (wq) memcpy(wq, c->wq, sizeof(double) * n * 4);
}

/* ------------------------------------------------------------------------- */
/* data term                                                                 */
/* ------------------------------------------------------------------------- */

/* rho(s|f): warp s' = s - (a s_u + b s_v + c, 0); the right view is sampled by
 * linear interpolation along u (rows are rectified, v stays integer), with u'
 * clamped to [0, W-1]; the colour L1 distance and gradient difference are
 * truncated and mixed with weight alpha (Eq. photofunc). */
double lo_rho(const lo_ctx *c, double a, double b, double cc, int su, int sv) {
    const int W = c->W;
    double d = a * su + b * sv + cc;
    double up = su - d;
    if (up < 0.0) up = 0.0;
    if (up > W - 1) up = W - 1;
    int i0 = (int)floor(up);
    if (i0 > W - 1) i0 = W - 1;
    int i1 = imin(i0 + 1, W - 1);
    double t = up - i0;
    const double *l = c->Lc + ((size_t)sv * W + su) * 4;
    const double *r0 = c->Rc + ((size_t)sv * W + i0) * 4;
    const double *r1 = c->Rc + ((size_t)sv * W + i1) * 4;
    double col = 0.0;
    for (int ch = 0; ch < 3; ch++) {
        double rv = (1.0 - t) * r0[ch] + t * r1[ch];
        col += fabs(l[ch] - rv);
    }
    double gr = (1.0 - t) * r0[3] + t * r1[3];
    double gd = fabs(l[3] - gr);
    double pa = c->p.alpha_grad;
    return (1.0 - pa) * fmin(col, c->p.tau_col) + pa * fmin(gd, c->p.tau_grad);
}

/* Guided-filter coefficients of window k for the raw cost of label f:
 * a_k = (Sigma_k + eU)^-1 (mean(I rho) - mu_k mean(rho)),  b_k = mean(rho) - a_k . mu_k
 * out = {a_k[0..2], b_k}. */
void lo_gf_coeffs(const lo_ctx *c, double a, double b, double cc, int kx, int ky, double *out) {
    const int H = c->H, W = c->W, r = c->p.gf_radius;
    int x0 = imax(kx - r, 0), x1 = imin(kx + r, W - 1);
    int y0 = imax(ky - r, 0), y1 = imin(ky + r, H - 1);
    double n = 0, mr = 0, mi[3] = {0, 0, 0};
    for (int y = y0; y <= y1; y++)
        for (int x = x0; x <= x1; x++) {
            double rho = lo_rho(c, a, b, cc, x, y);
            const double *l = c->Lc + ((size_t)y * W + x) * 4;
            mr += rho;
            for (int ch = 0; ch < 3; ch++) mi[ch] += (l[ch] / 255.0) * rho;
            n += 1;
        }
    mr /= n;
    size_t k = (size_t)ky * W + kx;
    const double *mu = c->mu + k * 3;
    const double *A = c->A + k * 9;
    double cov[3];
    for (int ch = 0; ch < 3; ch++) cov[ch] = mi[ch] / n - mu[ch] * mr;
    double bk = mr;
    for (int i = 0; i < 3; i++) {
        double ai = 0;
        for (int j = 0; j < 3; j++) ai += A[3 * i + j] * cov[j];
        out[i] = ai;
        bk -= ai * mu[i];
    }
    out[3] = bk;
}

/* phi_p(f) by definition: the guided-filter output at p of the raw-cost image
 * rho_f, i.e. the mean over the windows W'_k containing p (clipped to the
 * image) of a_k . I_p + b_k.  In the interior this equals sum_s omega_ps rho(s|f)
 * with omega from Eq. gf. */
double lo_phi_def(const lo_ctx *c, double a, double b, double cc, int pu, int pv) {
    const int H = c->H, W = c->W, r = c->p.gf_radius;
    /* raw costs over the matching window W_p = union of the W'_k */
    int mx0 = imax(pu - 2 * r, 0), mx1 = imin(pu + 2 * r, W - 1);
    int my0 = imax(pv - 2 * r, 0), my1 = imin(pv + 2 * r, H - 1);
    int mw = mx1 - mx0 + 1, mh = my1 - my0 + 1;
    double *rho = (double *)malloc(sizeof(double) * (size_t)mw * mh);
    for (int y = my0; y <= my1; y++)
        for (int x = mx0; x <= mx1; x++) rho[(size_t)(y - my0) * mw + (x - mx0)] = lo_rho(c, a, b, cc, x, y);
    const double *lp = c->Lc + ((size_t)pv * W + pu) * 4;
    double Ip[3] = {lp[0] / 255.0, lp[1] / 255.0, lp[2] / 255.0};
    double acc = 0, nk = 0;
    for (int ky = imax(pv - r, 0); ky <= imin(pv + r, H - 1); ky++)
        for (int kx = imax(pu - r, 0); kx <= imin(pu + r, W - 1); kx++) {
            int x0 = imax(kx - r, 0), x1 = imin(kx + r, W - 1);
            int y0 = imax(ky - r, 0), y1 = imin(ky + r, H - 1);
            double n = 0, mr = 0, mi[3] = {0, 0, 0};
            for (int y = y0; y <= y1; y++)
                for (int x = x0; x <= x1; x++) {
                    double v = rho[(size_t)(y - my0) * mw + (x - mx0)];
                    const double *l = c->Lc + ((size_t)y * W + x) * 4;
                    mr += v;
                    for (int ch = 0; ch < 3; ch++) mi[ch] += (l[ch] / 255.0) * v;
                    n += 1;
                }
            mr /= n;
            size_t k = (size_t)ky * W + kx;
            const double *mu = c->mu + k * 3;
            const double *A = c->A + k * 9;
            double cov[3];
            for (int ch = 0; ch < 3; ch++) cov[ch] = mi[ch] / n - mu[ch] * mr;
            double q = mr;
            for (int i = 0; i < 3; i++) {
                double ai = 0;
                for (int j = 0; j < 3; j++) ai += A[3 * i + j] * cov[j];
                q += ai * (Ip[i] - mu[i]);
            }
            acc += q;
            nk += 1;
        }
    free(rho);
    return acc / nk;
}

/* The explicit weights omega_ps of Eq. gf for s in the matching window of p:
 * (1/|W'|^2) sum_{k: p,s in W'_k} (1 + (I_p - mu_k)^T (Sigma_k + eU)^-1 (I_s - mu_k)).
 * out is (4r'+1)^2, row-major, centred on p; entries outside the image are 0.
 * Only meaningful away from the border (no clipped window). */
void lo_phi_weights(const lo_ctx *c, int pu, int pv, double *out) {
    const int H = c->H, W = c->W, r = c->p.gf_radius;
    const int side = 4 * r + 1;
    const double nw = (double)(2 * r + 1) * (2 * r + 1);
    memset(out, 0, sizeof(double) * side * side);
    const double *lp = c->Lc + ((size_t)pv * W + pu) * 4;
    double Ip[3] = {lp[0] / 255.0, lp[1] / 255.0, lp[2] / 255.0};
    for (int ky = pv - r; ky <= pv + r; ky++)
        for (int kx = pu - r; kx <= pu + r; kx++) {
            if (kx < 0 || ky < 0 || kx >= W || ky >= H) continue;
            size_t k = (size_t)ky * W + kx;
            const double *mu = c->mu + k * 3;
            const double *A = c->A + k * 9;
            double g[3];
            for (int i = 0; i < 3; i++) {
                g[i] = 0;
                for (int j = 0; j < 3; j++) g[i] += (Ip[j] - mu[j]) * A[3 * j + i];
            }
            for (int sy = ky - r; sy <= ky + r; sy++)
                for (int sx = kx - r; sx <= kx + r; sx++) {
                    if (sx < 0 || sy < 0 || sx >= W || sy >= H) continue;
                    const double *ls = c->Lc + ((size_t)sy * W + sx) * 4;
                    double q = 1.0;
                    for (int i = 0; i < 3; i++) q += g[i] * (ls[i] / 255.0 - mu[i]);
                    out[(sy - pv + 2 * r) * side + (sx - pu + 2 * r)] += q / (nw * nw);
                }
        }
}

/* phi_p(alpha) for every p of the expansion region R = [x0,x0+w) x [y0,y0+h) at
 * once, as in Sec. 3.5: raw costs over the filtering region M (R grown by the
 * matching-window radius 2r', clipped), guided-filter coefficients for every
 * window centre k in R grown by r', then their window means at p in R.  Box
 * sums are plain separable sums over the clipped windows.  out is w*h,
 * row-major. */
/* LE-BF data term (Sec. 4, "LE-BF"): the weights of Eq. unary are bilateral,
 * w_ps = exp(-|I_p - I_s|_1 / gamma) on the 0..255 left colours, "defined
 * similarly to Eq. smweight" (readings: gamma = bf_gamma, default 10 like the
 * smoothness weight; the window is the LE-GF matching window, (4r'+1)^2 clipped
 * to the image; the weights are not normalised, as in Eq. smweight), so
 * phi_p(f) = sum_{s in W_p} w_ps rho(s|f), O(|W|) per pixel. */
double lo_phi_bf(const lo_ctx *c, double a, double b, double cc, int pu, int pv) {
    const int H = c->H, W = c->W, R = 2 * c->p.gf_radius;
    const double *lp = c->Lc + ((size_t)pv * W + pu) * 4;
    double sum = 0.0;
    for (int sv = imax(0, pv - R); sv <= imin(H - 1, pv + R); sv++)
        for (int su = imax(0, pu - R); su <= imin(W - 1, pu + R); su++) {
            const double *ls = c->Lc + ((size_t)sv * W + su) * 4;
            const double l1 = fabs(lp[0] - ls[0]) + fabs(lp[1] - ls[1]) + fabs(lp[2] - ls[2]);
            sum += exp(-l1 / c->p.bf_gamma) * lo_rho(c, a, b, cc, su, sv);
        }
    return sum;
}

void lo_region_cost(const lo_ctx *c, int x0, int y0, int w, int h, const float *abc, double *out) {
    const int H = c->H, W = c->W, r = c->p.gf_radius;
    if (c->p.data_term == 1) {
        for (int y = 0; y < h; y++)
            for (int x = 0; x < w; x++) out[y * w + x] = lo_phi_bf(c, abc[0], abc[1], abc[2], x0 + x, y0 + y);
        return;
    }
    const double a = abc[0], b = abc[1], cc = abc[2];
    int Mx0 = imax(x0 - 2 * r, 0), Mx1 = imin(x0 + w + 2 * r, W);
    int My0 = imax(y0 - 2 * r, 0), My1 = imin(y0 + h + 2 * r, H);
    int Kx0 = imax(x0 - r, 0), Kx1 = imin(x0 + w + r, W);
    int Ky0 = imax(y0 - r, 0), Ky1 = imin(y0 + h + r, H);
    int Mw = Mx1 - Mx0, Mh = My1 - My0, Kw = Kx1 - Kx0, Kh = Ky1 - Ky0;
    /* 4 channels over M: rho, I_r rho, I_g rho, I_b rho */
    double *X = (double *)malloc(sizeof(double) * (size_t)Mw * Mh * 4);
    for (int y = My0; y < My1; y++)
        for (int x = Mx0; x < Mx1; x++) {
            double rho = lo_rho(c, a, b, cc, x, y);
            const double *l = c->Lc + ((size_t)y * W + x) * 4;
            double *o = X + ((size_t)(y - My0) * Mw + (x - Mx0)) * 4;
            o[0] = rho;
            for (int ch = 0; ch < 3; ch++) o[1 + ch] = (l[ch] / 255.0) * rho;
        }
    /* horizontal window sums at K columns, for every M row */
    double *Hs = (double *)malloc(sizeof(double) * (size_t)Kw * Mh * 4);
    for (int y = 0; y < Mh; y++)
        for (int kx = Kx0; kx < Kx1; kx++) {
            int sx0 = imax(kx - r, 0), sx1 = imin(kx + r, W - 1);
            double s[4] = {0, 0, 0, 0};
            for (int x = sx0; x <= sx1; x++)
                for (int ch = 0; ch < 4; ch++) s[ch] += X[((size_t)y * Mw + (x - Mx0)) * 4 + ch];
            for (int ch = 0; ch < 4; ch++) Hs[((size_t)y * Kw + (kx - Kx0)) * 4 + ch] = s[ch];
        }
    /* vertical sums -> window means -> a_k, b_k over K */
    double *AB = (double *)malloc(sizeof(double) * (size_t)Kw * Kh * 4);
    for (int ky = Ky0; ky < Ky1; ky++)
        for (int kx = Kx0; kx < Kx1; kx++) {
            int sy0 = imax(ky - r, 0), sy1 = imin(ky + r, H - 1);
            int sx0 = imax(kx - r, 0), sx1 = imin(kx + r, W - 1);
            double n = (double)(sx1 - sx0 + 1) * (sy1 - sy0 + 1);
            double s[4] = {0, 0, 0, 0};
            for (int y = sy0; y <= sy1; y++)
                for (int ch = 0; ch < 4; ch++) s[ch] += Hs[((size_t)(y - My0) * Kw + (kx - Kx0)) * 4 + ch];
            double mr = s[0] / n;
            size_t k = (size_t)ky * W + kx;
            const double *mu = c->mu + k * 3;
            const double *A = c->A + k * 9;
            double cov[3];
            for (int ch = 0; ch < 3; ch++) cov[ch] = s[1 + ch] / n - mu[ch] * mr;
            double *o = AB + ((size_t)(ky - Ky0) * Kw + (kx - Kx0)) * 4;
            double bk = mr;
            for (int i = 0; i < 3; i++) {
                double ai = 0;
                for (int j = 0; j < 3; j++) ai += A[3 * i + j] * cov[j];
                o[i] = ai;
                bk -= ai * mu[i];
            }
            o[3] = bk;
        }
    /* window means of a_k, b_k at p in R:  phi_p = abar . I_p + bbar */
    double *H2 = (double *)malloc(sizeof(double) * (size_t)w * Kh * 4);
    for (int ky = 0; ky < Kh; ky++)
        for (int px = x0; px < x0 + w; px++) {
            int kx0 = imax(px - r, 0), kx1 = imin(px + r, W - 1);
            double s[4] = {0, 0, 0, 0};
            for (int kx = kx0; kx <= kx1; kx++)
                for (int ch = 0; ch < 4; ch++) s[ch] += AB[((size_t)ky * Kw + (kx - Kx0)) * 4 + ch];
            for (int ch = 0; ch < 4; ch++) H2[((size_t)ky * w + (px - x0)) * 4 + ch] = s[ch];
        }
    for (int py = y0; py < y0 + h; py++)
        for (int px = x0; px < x0 + w; px++) {
            int ky0 = imax(py - r, 0), ky1 = imin(py + r, H - 1);
            int kx0 = imax(px - r, 0), kx1 = imin(px + r, W - 1);
            double n = (double)(kx1 - kx0 + 1) * (ky1 - ky0 + 1);
            double s[4] = {0, 0, 0, 0};
            for (int ky = ky0; ky <= ky1; ky++)
                for (int ch = 0; ch < 4; ch++) s[ch] += H2[((size_t)(ky - Ky0) * w + (px - x0)) * 4 + ch];
            const double *l = c->Lc + ((size_t)py * W + px) * 4;
            double phi = s[3] / n;
            for (int ch = 0; ch < 3; ch++) phi += (s[ch] / n) * (l[ch] / 255.0);
            out[(size_t)(py - y0) * w + (px - x0)] = phi;
        }
    free(X);
    free(Hs);
    free(AB);
    free(H2);
}

/* ------------------------------------------------------------------------- */
/* smoothness term                                                           */
/* ------------------------------------------------------------------------- */

static inline double disp_at(const float *f, int u, int v) {
    return (double)f[0] * u + (double)f[1] * v + (double)f[2];
}

/* psi-bar_pq(f_p, f_q) = |d_p(f_p) - d_p(f_q)| + |d_q(f_q) - d_q(f_p)|  (Eq. smooth) */
double lo_psibar(int pu, int pv, int qu, int qv, const float *fp, const float *fq) {
    return fabs(disp_at(fp, pu, pv) - disp_at(fq, pu, pv)) + fabs(disp_at(fq, qu, qv) - disp_at(fp, qu, qv));
}

/* psi_pq = max(w_pq, eps) min(psi-bar, tau_dis), for q the forward neighbour
 * dir of p (Eq. smooth_phi); no lambda. */
double lo_psi(const lo_ctx *c, int pu, int pv, int dir, const float *fp, const float *fq) {
    int qu = pu + FDX[dir], qv = pv + FDY[dir];
    double wv = c->wq[((size_t)pv * c->W + pu) * 4 + dir];
    return wv * fmin(lo_psibar(pu, pv, qu, qv, fp, fq), c->p.tau_dis);
}

static inline int64_t quant(double S, double x) { return (int64_t)nearbyint(S * x); }

/* E(f) = sum_p phi_p(f_p) + lambda sum_{(p,q) in N8} psi_pq(f_p, f_q) (Eq. mrf),
 * each unordered neighbour pair counted once; the unary part is taken from
 * `cost`.  Also returns the quantised energy sum Q(phi_p) + sum Q(lambda psi). */
void lo_energy_of(const lo_ctx *c, const float *lab, const double *cost, double *E, int64_t *Eq) {
    const int H = c->H, W = c->W;
    const double S = c->p.quant_scale, lam = c->p.lambda;
    double e = 0;
    int64_t q = 0;
    for (int y = 0; y < H; y++)
        for (int x = 0; x < W; x++) {
            size_t p = (size_t)y * W + x;
            e += cost[p];
            q += quant(S, cost[p]);
            for (int d = 0; d < 4; d++) {
                int qx = x + FDX[d], qy = y + FDY[d];
                if (qx < 0 || qx >= W || qy >= H) continue;
                double ps = lam * lo_psi(c, x, y, d, lab + p * 3, lab + ((size_t)qy * W + qx) * 3);
                e += ps;
                q += quant(S, ps);
            }
        }
    *E = e;
    *Eq = q;
}

void lo_energy(const lo_ctx *c, double *E, int64_t *Eq) { lo_energy_of(c, c->lab, c->cost, E, Eq); }

/* ------------------------------------------------------------------------- */
/* binary expansion-move graph                                               */
/* ------------------------------------------------------------------------- */

/* Builds the s-t graph of the expansion move "each p in R keeps f_p (x_p = 0)
 * or takes alpha (x_p = 1)".  A node with x_p = 1 lies on the sink side, so the
 * s->p edge carries U_p(1) and p->t carries U_p(0).  Neighbours q outside R are
 * fixed: their pairwise terms fold into p's unaries (footnote to Lemma 2).  For
 * a pair inside R with A = psi(f_p,f_q), B = psi(f_p,alpha), C = psi(alpha,f_q),
 * D = psi(alpha,alpha) = 0 (all times lambda, quantised), the decomposition
 * A + (C-A) x_p + (D-C) x_q + (B+C-A-D)(1-x_p) x_q gives the edge p->q with
 * capacity B+C-A >= 0 (Lemma 1); a quantised A above B+C (rounding only) is
 * lowered to B+C.  Unaries are then shifted so min(U(0), U(1)) = 0.
 *
 * lab/cost: the current labels and cached phi_p(f_p) of the whole image;
 * phi_alpha: phi_p(alpha) for p in R (w*h, row-major).
 * tcap: w*h*2 {s->p, p->t}; ncap: w*h*4 forward directions (0 outside R).
 * Returns the constant term; *nclamp counts lowered pairs.  If clamp_mask is
 * given, bit d of clamp_mask[p] is set when pair (p, p+dir d) was lowered. */
int64_t lo_build_graph(const lo_ctx *c, int x0, int y0, int w, int h, const float *alpha,
                       const float *lab, const double *cost, const double *phi_alpha,
                       int32_t *tcap, int32_t *ncap, int *nclamp, uint8_t *clamp_mask) {
    const int H = c->H, W = c->W;
    const double S = c->p.quant_scale, lam = c->p.lambda;
    const int n = w * h;
    int64_t *U0 = (int64_t *)calloc((size_t)n, sizeof(int64_t));
    int64_t *U1 = (int64_t *)calloc((size_t)n, sizeof(int64_t));
    int64_t cst = 0;
    int ncl = 0;
    for (int iy = 0; iy < h; iy++)
        for (int ix = 0; ix < w; ix++) {
            int i = iy * w + ix;
            U0[i] += quant(S, cost[(size_t)(y0 + iy) * W + x0 + ix]);
            U1[i] += quant(S, phi_alpha[i]);
            if (clamp_mask) clamp_mask[i] = 0;
        }
    for (int iy = 0; iy < h; iy++)
        for (int ix = 0; ix < w; ix++) {
            int i = iy * w + ix;
            int pu = x0 + ix, pv = y0 + iy;
            const float *fp = lab + ((size_t)pv * W + pu) * 3;
            for (int d = 0; d < 4; d++) ncap[i * 4 + d] = 0;
            /* all 8 neighbours; a pair inside R is handled once, from its
             * first node in the forward direction */
            for (int d8 = 0; d8 < 8; d8++) {
                int fwd = d8 < 4;
                int d = d8 & 3;
                int dx = fwd ? FDX[d] : -FDX[d];
                int dy = fwd ? FDY[d] : -FDY[d];
                int qu = pu + dx, qv = pv + dy;
                if (qu < 0 || qu >= W || qv < 0 || qv >= H) continue;
                const float *fq = lab + ((size_t)qv * W + qu) * 3;
                int qin = qu >= x0 && qu < x0 + w && qv >= y0 && qv < y0 + h;
                /* psi with the pair's weight: stored at the forward node */
                int bu = fwd ? pu : qu, bv = fwd ? pv : qv;
                double wv = c->wq[((size_t)bv * W + bu) * 4 + d];
                if (!qin) {
                    double pk = lam * wv * fmin(lo_psibar(pu, pv, qu, qv, fp, fq), c->p.tau_dis);
                    double pa = lam * wv * fmin(lo_psibar(pu, pv, qu, qv, alpha, fq), c->p.tau_dis);
                    U0[i] += quant(S, pk);
                    U1[i] += quant(S, pa);
                } else if (fwd) {
                    int j = (qv - y0) * w + (qu - x0);
                    int64_t A = quant(S, lam * wv * fmin(lo_psibar(pu, pv, qu, qv, fp, fq), c->p.tau_dis));
                    int64_t B = quant(S, lam * wv * fmin(lo_psibar(pu, pv, qu, qv, fp, alpha), c->p.tau_dis));
                    int64_t C = quant(S, lam * wv * fmin(lo_psibar(pu, pv, qu, qv, alpha, fq), c->p.tau_dis));
                    if (A > B + C) {
                        A = B + C;
                        ncl++;
                        if (clamp_mask) clamp_mask[i] |= (uint8_t)(1u << d);
                    }
                    cst += A;
                    U1[i] += C - A;
                    U1[j] += -C;
                    ncap[i * 4 + d] = (int32_t)(B + C - A);
                }
            }
        }
    for (int i = 0; i < n; i++) {
        int64_t m = U0[i] < U1[i] ? U0[i] : U1[i];
        cst += m;
        tcap[2 * i] = (int32_t)(U1[i] - m);
        tcap[2 * i + 1] = (int32_t)(U0[i] - m);
    }
    free(U0);
    free(U1);
    if (nclamp) *nclamp = ncl;
    return cst;
}

/* ------------------------------------------------------------------------- */
/* min-cut solvers on the region grid graph                                  */
/* ------------------------------------------------------------------------- */

typedef struct {
    int n, m;          /* nodes incl. s = n-2, t = n-1; edges (paired) */
    int *head, *nxt, *to;
    int64_t *cap;      /* residual capacity */
} flow_graph;

static void fg_init(flow_graph *g, int n, int maxe) {
    g->n = n;
    g->m = 0;
    g->head = (int *)malloc(sizeof(int) * n);
    for (int i = 0; i < n; i++) g->head[i] = -1;
    g->nxt = (int *)malloc(sizeof(int) * maxe);
    g->to = (int *)malloc(sizeof(int) * maxe);
    g->cap = (int64_t *)malloc(sizeof(int64_t) * maxe);
}

static void fg_free(flow_graph *g) {
    free(g->head);
    free(g->nxt);
    free(g->to);
    free(g->cap);
}

static void fg_add(flow_graph *g, int u, int v, int64_t c) {
    g->to[g->m] = v;
    g->cap[g->m] = c;
    g->nxt[g->m] = g->head[u];
    g->head[u] = g->m++;
    g->to[g->m] = u;
    g->cap[g->m] = 0;
    g->nxt[g->m] = g->head[v];
    g->head[v] = g->m++;
}

static void fg_from_grid(flow_graph *g, int w, int h, const int32_t *tcap, const int32_t *ncap) {
    int n = w * h;
    fg_init(g, n + 2, 2 * (2 * n + 4 * n));
    int s = n, t = n + 1;
    for (int i = 0; i < n; i++) {
        if (tcap[2 * i] > 0) fg_add(g, s, i, tcap[2 * i]);
        if (tcap[2 * i + 1] > 0) fg_add(g, i, t, tcap[2 * i + 1]);
    }
    for (int iy = 0; iy < h; iy++)
        for (int ix = 0; ix < w; ix++) {
            int i = iy * w + ix;
            for (int d = 0; d < 4; d++) {
                int jx = ix + FDX[d], jy = iy + FDY[d];
                if (jx < 0 || jx >= w || jy >= h) continue;
                if (ncap[i * 4 + d] > 0) fg_add(g, i, jy * w + jx, ncap[i * 4 + d]);
            }
        }
}

/* cut[i] = 1 iff node i reaches t through edges with residual capacity */
static void fg_sink_side(const flow_graph *g, uint8_t *cut, int nnodes) {
    int n = g->n, t = n - 1;
    uint8_t *seen = (uint8_t *)calloc((size_t)n, 1);
    int *q = (int *)malloc(sizeof(int) * n);
    int qh = 0, qt = 0;
    seen[t] = 1;
    q[qt++] = t;
    while (qh < qt) {
        int v = q[qh++];
        for (int e = g->head[v]; e >= 0; e = g->nxt[e]) {
            int u = g->to[e];
            /* edge e is v->u; its partner e^1 is u->v */
            if (!seen[u] && g->cap[e ^ 1] > 0) {
                seen[u] = 1;
                q[qt++] = u;
            }
        }
    }
    for (int i = 0; i < nnodes; i++) cut[i] = seen[i];
    free(seen);
    free(q);
}

/* Dinic: BFS level graph from s, blocking flow by iterative DFS with
 * current-arc pointers.  Returns the max-flow value. */
int64_t lo_maxflow_dinic(int w, int h, const int32_t *tcap, const int32_t *ncap, uint8_t *cut) {
    flow_graph g;
    fg_from_grid(&g, w, h, tcap, ncap);
    const int n = g.n, s = n - 2, t = n - 1;
    int *level = (int *)malloc(sizeof(int) * n);
    int *it = (int *)malloc(sizeof(int) * n);
    int *q = (int *)malloc(sizeof(int) * n);
    int *stack_e = (int *)malloc(sizeof(int) * n);
    int64_t flow = 0;
    for (;;) {
        for (int i = 0; i < n; i++) level[i] = -1;
        int qh = 0, qt = 0;
        level[s] = 0;
        q[qt++] = s;
        while (qh < qt) {
            int v = q[qh++];
            for (int e = g.head[v]; e >= 0; e = g.nxt[e])
                if (g.cap[e] > 0 && level[g.to[e]] < 0) {
                    level[g.to[e]] = level[v] + 1;
                    q[qt++] = g.to[e];
                }
        }
        if (level[t] < 0) break;
        for (int i = 0; i < n; i++) it[i] = g.head[i];
        /* repeated DFS from s along level-increasing edges */
        for (;;) {
            int depth = 0, v = s;
            int found = 0;
            while (1) {
                if (v == t) {
                    found = 1;
                    break;
                }
                int e = it[v];
                while (e >= 0 && !(g.cap[e] > 0 && level[g.to[e]] == level[v] + 1)) e = g.nxt[e];
                it[v] = e;
                if (e < 0) {
                    /* dead end: retreat */
                    level[v] = -1;
                    if (depth == 0) break;
                    depth--;
                    v = g.to[stack_e[depth] ^ 1];
                    it[v] = g.nxt[it[v]];
                    continue;
                }
                stack_e[depth++] = e;
                v = g.to[e];
            }
            if (!found) break;
            int64_t b = INT64_MAX;
            for (int k = 0; k < depth; k++)
                if (g.cap[stack_e[k]] < b) b = g.cap[stack_e[k]];
            for (int k = 0; k < depth; k++) {
                g.cap[stack_e[k]] -= b;
                g.cap[stack_e[k] ^ 1] += b;
            }
            flow += b;
        }
    }
    if (cut) fg_sink_side(&g, cut, w * h);
    free(level);
    free(it);
    free(q);
    free(stack_e);
    fg_free(&g);
    return flow;
}

/* Edmonds-Karp, written independently of the Dinic path: explicit residual
 * arrays per node (s/t edges and the 8 grid directions), shortest augmenting
 * paths by BFS with parent pointers. */
int64_t lo_maxflow_ek(int w, int h, const int32_t *tcap, const int32_t *ncap, uint8_t *cut) {
    const int n = w * h;
    /* res_s[i]: s->i, res_t[i]: i->t, rs_back[i]: i->s, rt_back[i]: t->i,
     * res8[i*8+k]: i -> neighbour k (k<4 forward dirs, k>=4 the reverse dirs) */
    int64_t *res_s = (int64_t *)calloc((size_t)n, sizeof(int64_t));
    int64_t *res_t = (int64_t *)calloc((size_t)n, sizeof(int64_t));
    int64_t *rs_back = (int64_t *)calloc((size_t)n, sizeof(int64_t));
    int64_t *rt_back = (int64_t *)calloc((size_t)n, sizeof(int64_t));
    int64_t *res8 = (int64_t *)calloc((size_t)n * 8, sizeof(int64_t));
    for (int i = 0; i < n; i++) {
        res_s[i] = tcap[2 * i];
        res_t[i] = tcap[2 * i + 1];
    }
    for (int iy = 0; iy < h; iy++)
        for (int ix = 0; ix < w; ix++) {
            int i = iy * w + ix;
            for (int d = 0; d < 4; d++) {
                int jx = ix + FDX[d], jy = iy + FDY[d];
                if (jx < 0 || jx >= w || jy >= h) continue;
                res8[(size_t)i * 8 + d] = ncap[i * 4 + d];
            }
        }
    /* node ids: 0..n-1 pixels, n = s, n+1 = t.  parent[v] encodes the edge used
     * to reach v: (u, k) with k in 0..7 grid, 8 = from s, 9 = to t. */
    int *par_u = (int *)malloc(sizeof(int) * (n + 2));
    int *par_k = (int *)malloc(sizeof(int) * (n + 2));
    int *queue = (int *)malloc(sizeof(int) * (n + 2));
    int64_t flow = 0;
    const int S = n, T = n + 1;
    for (;;) {
        for (int i = 0; i < n + 2; i++) par_u[i] = -2;
        par_u[S] = -1;
        int qh = 0, qt = 0;
        queue[qt++] = S;
        int reached = 0;
        while (qh < qt && !reached) {
            int u = queue[qh++];
            if (u == S) {
                for (int i = 0; i < n; i++)
                    if (res_s[i] > 0 && par_u[i] == -2) {
                        par_u[i] = S;
                        par_k[i] = 8;
                        queue[qt++] = i;
                    }
                continue;
            }
            /* u is a pixel */
            if (res_t[u] > 0 && par_u[T] == -2) {
                par_u[T] = u;
                par_k[T] = 9;
                reached = 1;
                break;
            }
            if (rs_back[u] > 0) { /* back to s: never useful for a shortest path */
            }
            int ux = u % w, uy = u / w;
            for (int k = 0; k < 8; k++) {
                int d = k & 3;
                int vx = k < 4 ? ux + FDX[d] : ux - FDX[d];
                int vy = k < 4 ? uy + FDY[d] : uy - FDY[d];
                if (vx < 0 || vx >= w || vy < 0 || vy >= h) continue;
                int v = vy * w + vx;
                if (res8[(size_t)u * 8 + k] > 0 && par_u[v] == -2) {
                    par_u[v] = u;
                    par_k[v] = k;
                    queue[qt++] = v;
                }
            }
        }
        if (!reached) break;
        /* bottleneck */
        int64_t b = INT64_MAX;
        for (int v = T; v != S;) {
            int u = par_u[v], k = par_k[v];
            int64_t r = (k == 8) ? res_s[v] : (k == 9) ? res_t[u] : res8[(size_t)u * 8 + k];
            if (r < b) b = r;
            v = u;
        }
        for (int v = T; v != S;) {
            int u = par_u[v], k = par_k[v];
            if (k == 8) {
                res_s[v] -= b;
                rs_back[v] += b;
            } else if (k == 9) {
                res_t[u] -= b;
                rt_back[u] += b;
            } else {
                res8[(size_t)u * 8 + k] -= b;
                int kr = k < 4 ? k + 4 : k - 4;
                res8[(size_t)v * 8 + kr] += b;
            }
            v = u;
        }
        flow += b;
    }
    if (cut) {
        /* sink side: nodes with a residual path to t; search backwards from t */
        uint8_t *seen = (uint8_t *)calloc((size_t)n, 1);
        int qh = 0, qt = 0;
        for (int i = 0; i < n; i++)
            if (res_t[i] > 0) {
                seen[i] = 1;
                queue[qt++] = i;
            }
        while (qh < qt) {
            int v = queue[qh++];
            int vx = v % w, vy = v / w;
            /* u -> v residual, u a neighbour of v */
            for (int k = 0; k < 8; k++) {
                int d = k & 3;
                int ux = k < 4 ? vx - FDX[d] : vx + FDX[d];
                int uy = k < 4 ? vy - FDY[d] : vy + FDY[d];
                if (ux < 0 || ux >= w || uy < 0 || uy >= h) continue;
                int u = uy * w + ux;
                if (!seen[u] && res8[(size_t)u * 8 + k] > 0) {
                    seen[u] = 1;
                    queue[qt++] = u;
                }
            }
        }
        for (int i = 0; i < n; i++) cut[i] = seen[i];
        free(seen);
    }
    free(res_s);
    free(res_t);
    free(rs_back);
    free(rt_back);
    free(res8);
    free(par_u);
    free(par_k);
    free(queue);
    return flow;
}

/* Exhaustive enumeration (w*h <= 20): the minimum of the cut function over all
 * 2^n labellings, and the intersection of all minimisers (the minimal
 * minimiser, unique because cut functions are submodular).  Returns the
 * minimum cut value. */
int64_t lo_mincut_enum(int w, int h, const int32_t *tcap, const int32_t *ncap, uint8_t *cut) {
    const int n = w * h;
    if (n > 20) return -1;
    int64_t best = INT64_MAX;
    uint32_t inter = 0;
    for (uint32_t x = 0; x < (1u << n); x++) {
        int64_t v = 0;
        for (int i = 0; i < n; i++) v += ((x >> i) & 1u) ? tcap[2 * i] : tcap[2 * i + 1];
        for (int iy = 0; iy < h; iy++)
            for (int ix = 0; ix < w; ix++) {
                int i = iy * w + ix;
                for (int d = 0; d < 4; d++) {
                    int jx = ix + FDX[d], jy = iy + FDY[d];
                    if (jx < 0 || jx >= w || jy >= h) continue;
                    int j = jy * w + jx;
                    if (!((x >> i) & 1u) && ((x >> j) & 1u)) v += ncap[i * 4 + d];
                }
            }
        if (v < best) {
            best = v;
            inter = x;
        } else if (v == best) {
            inter &= x;
        }
    }
    if (cut)
        for (int i = 0; i < n; i++) cut[i] = (inter >> i) & 1u;
    return best;
}

/* ------------------------------------------------------------------------- */
/* random draws: SplitMix64 (Steele, Lea, Flood 2014)                         */
/* ------------------------------------------------------------------------- */

static inline uint64_t sm_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static inline uint64_t sm_next(uint64_t *state) {
    *state += 0x9E3779B97F4A7C15ull;
    return sm_mix(*state);
}

static inline double sm_u01(uint64_t *state) { return (double)(sm_next(state) >> 11) * 0x1.0p-53; }

uint64_t lo_splitmix64_next(uint64_t *state) { return sm_next(state); }

/* stream of one proposal of one alpha_ij-expansion */
uint64_t lo_proposal_stream(uint64_t seed, int iter, int level, int ci, int cj, int proposal) {
    uint64_t s = sm_mix(seed);
    s = sm_mix(s ^ (uint64_t)iter);
    s = sm_mix(s ^ (uint64_t)level);
    s = sm_mix(s ^ (((uint64_t)(uint32_t)cj << 32) | (uint64_t)(uint32_t)ci));
    s = sm_mix(s ^ (uint64_t)proposal);
    return s;
}

uint64_t lo_init_stream(uint64_t seed, int64_t pixel) {
    return sm_mix(sm_mix(seed ^ 0x5851F42D4C957F2Dull) ^ (uint64_t)pixel);
}

/* random unit vector by rejection from the cube [-1,1]^3: triples that land
 * outside the unit ball (or at 0) are drawn again, at most 1000 times (the
 * acceptance rate is pi/6), after which (0,0,1) is returned. */
static void unit_vector(uint64_t *st, double v[3]) {
    for (int t = 0; t < 1000; t++) {
        double x = 2.0 * sm_u01(st) - 1.0;
        double y = 2.0 * sm_u01(st) - 1.0;
        double z = 2.0 * sm_u01(st) - 1.0;
        double s = (x * x + y * y) + z * z;
        if (s > 1.0 || s == 0.0) continue;
        double l = sqrt(s);
        v[0] = x / l;
        v[1] = y / l;
        v[2] = z / l;
        return;
    }
    v[0] = 0.0;
    v[1] = 0.0;
    v[2] = 1.0;
}

/* Random initial label of pixel (u, v) (Sec. 3.4, after Bleyer et al.): a random
 * disparity z0 in [dmin, dmax] and a random unit normal n (redrawn while
 * |n_z| < 1e-3, at most 64 tries, else n = (0,0,1)); the plane through
 * (u, v, z0) with normal n is a = -n_x/n_z, b = -n_y/n_z,
 * c = (n_x u + n_y v + n_z z0)/n_z. */
void lo_init_label(uint64_t seed, int W, int u, int v, double dmin, double dmax, float *out) {
    uint64_t st = lo_init_stream(seed, (int64_t)v * W + u);
    double z0 = dmin + (dmax - dmin) * sm_u01(&st);
    double n[3] = {0.0, 0.0, 1.0};
    for (int t = 0; t < 64; t++) {
        double c[3];
        unit_vector(&st, c);
        if (fabs(c[2]) < 1e-3) continue;
        n[0] = c[0];
        n[1] = c[1];
        n[2] = c[2];
        break;
    }
    double a = -n[0] / n[2];
    double b = -n[1] / n[2];
    double cc = ((n[0] * u + n[1] * v) + n[2] * z0) / n[2];
    out[0] = (float)a;
    out[1] = (float)b;
    out[2] = (float)cc;
}

/* pick r uniformly in the (clipped) centre cell */
static void pick_pixel(uint64_t *st, int cx0, int cy0, int cw, int ch, int *ru, int *rv) {
    int n = cw * ch;
    int k = (int)(sm_u01(st) * n);
    if (k >= n) k = n - 1;
    *ru = cx0 + k % cw;
    *rv = cy0 + k / cw;
}

/* Candidate of one map proposal: alpha = m_r, the proposal map's label at a
 * pixel r drawn uniformly from the centre cell (as the propagation proposal
 * draws f_r). */
void lo_propose_map(const float *map, int W, uint64_t stream, int cx0, int cy0, int cw, int ch, float *alpha) {
    uint64_t st = stream;
    int ru, rv;
    pick_pixel(&st, cx0, cy0, cw, ch, &ru, &rv);
    const float *m = map + ((size_t)rv * W + ru) * 3;
    alpha[0] = m[0];
    alpha[1] = m[1];
    alpha[2] = m[2];
}

/* RANSAC proposer (Algorithm 2, RANSAC proposal): a plane fitted to the current
 * disparities of the centre cell C_ij by LO-RANSAC (Chum et al. 2003).  The paper
 * gives no settings; the readings: the points are the pixels r of C_ij with their
 * disparities d_r = (a u + b v) + c in FP64, taken on the 2^-20 grid (round half to
 * even) so that every sum below is an exact integer; 32 hypotheses, each the plane
 * through three pixels drawn uniformly from the proposal's stream (a repeated pixel
 * or three collinear pixels make a hypothesis void); inliers are the points within
 * 1 px of the plane; the hypothesis with the most inliers (the first on ties) is
 * refined twice by a least-squares fit to its inliers (skipped with fewer than 3
 * inliers or a singular system).  Coordinates are taken relative to the cell's
 * corner.  With no valid hypothesis the candidate is the label of the first drawn
 * pixel.  Every floating-point step below is one correctly rounded operation in the
 * order written. */
#define RANSAC_HYP 32
#define RANSAC_LO 2
#define RANSAC_Q 1048576.0 /* 2^20 */

static int64_t ransac_dq(const float *f, int u, int v) {
    const double d = ((double)f[0] * (double)u + (double)f[1] * (double)v) + (double)f[2];
    return (int64_t)nearbyint(d * RANSAC_Q);
}

static int ransac_inliers(const int64_t *dq, int n, int cw, double a, double b, double c, unsigned char *in) {
    int cnt = 0;
    for (int k = 0; k < n; k++) {
        const int x = k % cw, y = k / cw;
        const double r = (double)dq[k] / RANSAC_Q - ((a * (double)x + b * (double)y) + c);
        const int ok = fabs(r) <= 1.0;
        if (in) in[k] = (unsigned char)ok;
        cnt += ok;
    }
    return cnt;
}

void lo_propose_ransac(const float *lab, int W, uint64_t stream, int cx0, int cy0, int cw, int ch, float *alpha) {
    uint64_t st = stream;
    const int n = cw * ch;
    int64_t *dq = (int64_t *)malloc(sizeof(int64_t) * n);
    unsigned char *in = (unsigned char *)malloc(n);
    for (int k = 0; k < n; k++) {
        const int u = cx0 + k % cw, v = cy0 + k / cw;
        dq[k] = ransac_dq(lab + ((size_t)v * W + u) * 3, u, v);
    }
    int best = -1, best_cnt = -1, first = -1;
    double ba = 0, bb = 0, bc = 0;
    for (int hyp = 0; hyp < RANSAC_HYP; hyp++) {
        int id[3];
        for (int j = 0; j < 3; j++) {
            int k = (int)(sm_u01(&st) * n);
            if (k >= n) k = n - 1;
            id[j] = k;
        }
        if (first < 0) first = id[0];
        if (id[0] == id[1] || id[0] == id[2] || id[1] == id[2]) continue;
        const int64_t x0 = id[0] % cw, y0 = id[0] / cw, x1 = id[1] % cw, y1 = id[1] / cw;
        const int64_t x2 = id[2] % cw, y2 = id[2] / cw;
        const int64_t du1 = x1 - x0, dv1 = y1 - y0, du2 = x2 - x0, dv2 = y2 - y0;
        const int64_t det = du1 * dv2 - du2 * dv1;
        if (det == 0) continue;
        const int64_t dd1 = dq[id[1]] - dq[id[0]], dd2 = dq[id[2]] - dq[id[0]];
        const int64_t na = dd1 * dv2 - dd2 * dv1, nb = du1 * dd2 - du2 * dd1;
        const double den = (double)det * RANSAC_Q;
        const double a = (double)na / den, b = (double)nb / den;
        const double c = ((double)dq[id[0]] / RANSAC_Q - a * (double)x0) - b * (double)y0;
        const int cnt = ransac_inliers(dq, n, cw, a, b, c, NULL);
        if (cnt > best_cnt) {
            best_cnt = cnt;
            best = hyp;
            ba = a;
            bb = b;
            bc = c;
        }
    }
    if (best < 0) {
        const int k = first < 0 ? 0 : first;
        const float *f = lab + ((size_t)(cy0 + k / cw) * W + cx0 + k % cw) * 3;
        alpha[0] = f[0];
        alpha[1] = f[1];
        alpha[2] = f[2];
        free(dq);
        free(in);
        return;
    }
    for (int it = 0; it < RANSAC_LO; it++) {
        const int cnt = ransac_inliers(dq, n, cw, ba, bb, bc, in);
        if (cnt < 3) break;
        int64_t Suu = 0, Suv = 0, Su = 0, Svv = 0, Sv = 0, Sn = 0, Sud = 0, Svd = 0, Sd = 0;
        for (int k = 0; k < n; k++) {
            if (!in[k]) continue;
            const int64_t x = k % cw, y = k / cw;
            Suu += x * x;
            Suv += x * y;
            Su += x;
            Svv += y * y;
            Sv += y;
            Sn += 1;
            Sud += x * dq[k];
            Svd += y * dq[k];
            Sd += dq[k];
        }
        const double m00 = (double)Suu, m01 = (double)Suv, m02 = (double)Su, m11 = (double)Svv, m12 = (double)Sv;
        const double m22 = (double)Sn, r0 = (double)Sud, r1 = (double)Svd, r2 = (double)Sd;
        /* Cramer's rule on the symmetric system [m00 m01 m02; m01 m11 m12; m02 m12 m22] */
        const double c00 = m11 * m22 - m12 * m12, c01 = m01 * m22 - m12 * m02, c02 = m01 * m12 - m11 * m02;
        const double det = (m00 * c00 - m01 * c01) + m02 * c02;
        if (det == 0.0) break;
        const double da = (r0 * c00 - m01 * (r1 * m22 - m12 * r2)) + m02 * (r1 * m12 - m11 * r2);
        const double db = (m00 * (r1 * m22 - m12 * r2) - r0 * c01) + m02 * (m01 * r2 - r1 * m02);
        const double dc = (m00 * (m11 * r2 - r1 * m12) - m01 * (m01 * r2 - r1 * m02)) + r0 * c02;
        const double den = det * RANSAC_Q;
        ba = da / den;
        bb = db / den;
        bc = dc / den;
    }
    /* back to image coordinates */
    const double c_img = (bc - ba * (double)cx0) - bb * (double)cy0;
    alpha[0] = (float)ba;
    alpha[1] = (float)bb;
    alpha[2] = (float)c_img;
    free(dq);
    free(in);
}

/* Candidate alpha of one proposal (Algorithm 2).  perturb = 0: propagation,
 * alpha = f_r.  perturb = 1: the label f_r is turned into a disparity d and unit
 * normal n at r, d' = d + U[-rd, rd] (clamped to [dmin, dmax]), n' = n + rn * v
 * for a random unit vector v, redrawn while |n'_z/|n'|| < 1e-3 (at most 64
 * tries, else n' = n), and (d', n'/|n'|) is turned back into a plane. */
void lo_propose(const float *lab, int W, uint64_t stream, int cx0, int cy0, int cw, int ch,
                int perturb, double rd, double rn, double dmin, double dmax, float *alpha) {
    uint64_t st = stream;
    int ru, rv;
    pick_pixel(&st, cx0, cy0, cw, ch, &ru, &rv);
    const float *f = lab + ((size_t)rv * W + ru) * 3;
    if (!perturb) {
        alpha[0] = f[0];
        alpha[1] = f[1];
        alpha[2] = f[2];
        return;
    }
    double a = f[0], b = f[1], c = f[2];
    double d = (a * ru + b * rv) + c;
    double len = sqrt((a * a + b * b) + 1.0);
    double n[3] = {-a / len, -b / len, 1.0 / len};
    double dp = d + rd * (2.0 * sm_u01(&st) - 1.0);
    if (dp < dmin) dp = dmin;
    if (dp > dmax) dp = dmax;
    double m[3] = {n[0], n[1], n[2]};
    for (int t = 0; t < 64; t++) {
        double v[3];
        unit_vector(&st, v);
        double q[3] = {n[0] + rn * v[0], n[1] + rn * v[1], n[2] + rn * v[2]};
        double ql = sqrt((q[0] * q[0] + q[1] * q[1]) + q[2] * q[2]);
        if (ql == 0.0) continue;
        q[0] /= ql;
        q[1] /= ql;
        q[2] /= ql;
        if (fabs(q[2]) < 1e-3) continue;
        m[0] = q[0];
        m[1] = q[1];
        m[2] = q[2];
        break;
    }
    alpha[0] = (float)(-m[0] / m[2]);
    alpha[1] = (float)(-m[1] / m[2]);
    alpha[2] = (float)(((m[0] * ru + m[1] * rv) + m[2] * dp) / m[2]);
}

/* ------------------------------------------------------------------------- */
/* the method: Algorithms 1 and 2                                            */
/* ------------------------------------------------------------------------- */

/* state: random initial labels and their costs */
void lo_init_state(lo_ctx *c) {
    const int H = c->H, W = c->W;
    for (int v = 0; v < H; v++)
        for (int u = 0; u < W; u++)
            lo_init_label(c->p.seed, W, u, v, c->p.disp_min, c->p.disp_max, c->lab + ((size_t)v * W + u) * 3);
    int nt = c->p.n_threads;
#pragma omp parallel for schedule(dynamic, 16) num_threads(nt > 0 ? nt : omp_get_max_threads())
    for (int p = 0; p < H * W; p++) {
        double phi;
        lo_region_cost(c, p % W, p / W, 1, 1, c->lab + (size_t)p * 3, &phi);
        c->cost[p] = phi;
    }
}

/* replace the labels; the costs of changed pixels are recomputed */
void lo_set_labels(lo_ctx *c, const float *lab) {
    const int H = c->H, W = c->W;
    int nt = c->p.n_threads;
#pragma omp parallel for schedule(dynamic, 16) num_threads(nt > 0 ? nt : omp_get_max_threads())
    for (int p = 0; p < H * W; p++) {
        const float *f = lab + (size_t)p * 3;
        float *g = c->lab + (size_t)p * 3;
        if (f[0] == g[0] && f[1] == g[1] && f[2] == g[2] && !(c->cost[p] != c->cost[p])) continue;
        g[0] = f[0];
        g[1] = f[1];
        g[2] = f[2];
        double phi;
        lo_region_cost(c, p % W, p / W, 1, 1, g, &phi);
        c->cost[p] = phi;
    }
}

void lo_get_state(const lo_ctx *c, float *lab, double *cost) {
    size_t n = (size_t)c->H * c->W;
    if (lab) memcpy(lab, c->lab, sizeof(float) * n * 3);
    if (cost) memcpy(cost, c->cost, sizeof(double) * n);
}

void lo_put_state(lo_ctx *c, const float *lab, const double *cost) {
    size_t n = (size_t)c->H * c->W;
    memcpy(c->lab, lab, sizeof(float) * n * 3);
    memcpy(c->cost, cost, sizeof(double) * n);
}

/* One expansion move with candidate alpha on R; returns the number of
 * switched pixels, and the flow / constant through the pointers. */
static int expand_move(lo_ctx *c, int x0, int y0, int w, int h, const float *alpha, int64_t *flow_out) {
    const int W = c->W;
    int n = w * h;
    double *phiA = (double *)malloc(sizeof(double) * n);
    int32_t *tcap = (int32_t *)malloc(sizeof(int32_t) * n * 2);
    int32_t *ncap = (int32_t *)malloc(sizeof(int32_t) * n * 4);
    uint8_t *cut = (uint8_t *)malloc((size_t)n);
    lo_region_cost(c, x0, y0, w, h, alpha, phiA);
    lo_build_graph(c, x0, y0, w, h, alpha, c->lab, c->cost, phiA, tcap, ncap, NULL, NULL);
    int64_t f = lo_maxflow_dinic(w, h, tcap, ncap, cut);
    if (flow_out) *flow_out = f;
    int sw = 0;
    for (int iy = 0; iy < h; iy++)
        for (int ix = 0; ix < w; ix++) {
            int i = iy * w + ix;
            if (!cut[i]) continue;
            size_t p = (size_t)(y0 + iy) * W + x0 + ix;
            c->lab[p * 3 + 0] = alpha[0];
            c->lab[p * 3 + 1] = alpha[1];
            c->lab[p * 3 + 2] = alpha[2];
            c->cost[p] = phiA[i];
            sw++;
        }
    free(phiA);
    free(tcap);
    free(ncap);
    free(cut);
    return sw;
}

/* expansion region R_ij (3x3 cells around cell (i,j), clipped) and centre cell */
void lo_region_of(int H, int W, int s, int ci, int cj, int *R, int *C) {
    int x0 = imax(0, (ci - 1) * s), x1 = imin(W, (ci + 2) * s);
    int y0 = imax(0, (cj - 1) * s), y1 = imin(H, (cj + 2) * s);
    R[0] = x0;
    R[1] = y0;
    R[2] = x1 - x0;
    R[3] = y1 - y0;
    int cx0 = ci * s, cx1 = imin(W, (ci + 1) * s);
    int cy0 = cj * s, cy1 = imin(H, (cj + 1) * s);
    C[0] = cx0;
    C[1] = cy0;
    C[2] = cx1 - cx0;
    C[3] = cy1 - cy0;
}

/* Algorithm 2 at cell (i, j): K_prop propagation proposals, K_RANS RANSAC
 * proposals, then K_rand perturbation proposals with the perturbation size
 * halved after each.  The perturbation sizes are this call's own copies of the
 * outer ones.  With a proposal map, k_cnn map proposals follow the RANSAC ones
 * (proposal indices K_prop + K_RANS .. K_prop + K_RANS + k_cnn - 1); k_cnn = 0 is
 * the method as published.
 * With visit = K > 1 (the batched schedule variant) the candidates of each run
 * of K consecutive proposals are all drawn from the labels at the start of
 * that run; their moves are then made one after the other, each against the
 * labels left by the previous one.  visit = 1 is Algorithm 2 as printed. */
static int visit_proposals(const lo_ctx *c, int level) {
    const int kc = c->prop ? c->p.k_cnn[level] : 0;
    return c->p.k_prop[level] + c->p.k_rans[level] + kc + c->p.k_rand[level];
}

/* Candidates t0 .. t1-1 of the visit of cell (i, j) at `level`, drawn from the
 * labels `lab` (Algorithm 2, in proposal order: propagation, RANSAC, map,
 * perturbation) at pixels of the centre cell C_ij.  *rd and *rn are the visit's
 * own perturbation sizes, halved after each perturbation proposal. */
static void draw_candidates(const lo_ctx *c, const float *lab, int iter, int level, int ci, int cj, int t0, int t1,
                            double *rd, double *rn, float (*alpha)[3]) {
    const int W = c->W;
    int R[4], C[4];
    lo_region_of(c->H, W, c->p.cell[level], ci, cj, R, C);
    const int kp = c->p.k_prop[level], kr = c->p.k_rans[level], kc = c->prop ? c->p.k_cnn[level] : 0;
    for (int t = t0; t < t1; t++) {
        const uint64_t stream = lo_proposal_stream(c->p.seed, iter, level, ci, cj, t);
        if (t >= kp && t < kp + kr) {
            lo_propose_ransac(lab, W, stream, C[0], C[1], C[2], C[3], alpha[t - t0]);
            continue;
        }
        if (t >= kp + kr && t < kp + kr + kc) {
            lo_propose_map(c->prop, W, stream, C[0], C[1], C[2], C[3], alpha[t - t0]);
            continue;
        }
        const int perturb = t >= kp + kr + kc;
        lo_propose(lab, W, stream, C[0], C[1], C[2], C[3], perturb, perturb ? *rd : 0.0, perturb ? *rn : 0.0,
                   c->p.disp_min, c->p.disp_max, alpha[t - t0]);
        if (perturb) {
            *rd *= 0.5;
            *rn *= 0.5;
        }
    }
}

static void iterative_expansion(lo_ctx *c, int iter, int level, int ci, int cj, double rd, double rn,
                                long long *accepted, long long *evals) {
    const int H = c->H, W = c->W, s = c->p.cell[level];
    int R[4], C[4];
    lo_region_of(H, W, s, ci, cj, R, C);
    const int nprop = visit_proposals(c, level);
    const int K = c->p.visit < 1 ? 1 : (c->p.visit > 64 ? 64 : c->p.visit);
    float alpha[64][3];
    for (int t0 = 0; t0 < nprop; t0 += K) {
        const int t1 = t0 + K < nprop ? t0 + K : nprop;
        draw_candidates(c, c->lab, iter, level, ci, cj, t0, t1, &rd, &rn, alpha);
        for (int t = t0; t < t1; t++) {
            *accepted += expand_move(c, R[0], R[1], R[2], R[3], alpha[t - t0], NULL);
            *evals += (long long)R[2] * R[3];
        }
    }
}

/* outer perturbation sizes of iteration `iter`: r_d = (dmax-dmin)/2, r_n = 1,
 * both halved after every iteration (Algorithm 1) */
static void outer_delta(const lo_ctx *c, int iter, double *rd, double *rn) {
    double f = ldexp(1.0, -iter);
    *rd = 0.5 * (c->p.disp_max - c->p.disp_min) * f;
    *rn = 1.0 * f;
}

/* All alpha_ij-expansions of group k = 4 (j mod 4) + (i mod 4) (Eq. groupindex)
 * at grid level `level`, in parallel over the cells (they are independent,
 * Lemma 3).  Returns the number of switched pixels; *evals gets the number of
 * pixel-label cost evaluations. */
long long lo_expand_group(lo_ctx *c, int iter, int level, int group, long long *evals) {
    const int H = c->H, W = c->W, s = c->p.cell[level];
    const int nx = (W + s - 1) / s, ny = (H + s - 1) / s;
    const int gi = group % 4, gj = group / 4;
    const int cx = gi < nx ? (nx - gi + 3) / 4 : 0;
    const int cy = gj < ny ? (ny - gj + 3) / 4 : 0;
    const int ncell = cx * cy;
    double rd, rn;
    outer_delta(c, iter, &rd, &rn);
    long long acc = 0, ev = 0;
    int nt = c->p.n_threads;
    int rev = c->p.reverse_order;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : acc, ev) num_threads(nt > 0 ? nt : omp_get_max_threads())
    for (int k = 0; k < ncell; k++) {
        int kk = rev ? ncell - 1 - k : k;
        int ci = gi + 4 * (kk % cx), cj = gj + 4 * (kk / cx);
        long long a = 0, e = 0;
        iterative_expansion(c, iter, level, ci, cj, rd, rn, &a, &e);
        acc += a;
        ev += e;
    }
    if (evals) *evals = ev;
    return acc;
}

/* The alpha_ij-expansions of an explicit list of cells (i, j) = (cells[2k],
 * cells[2k+1]) of one group, as lo_expand_group runs them: used by the
 * stripe-decomposed driver, where each domain runs the cells whose centre
 * cell lies in its stripe.  Returns the number of switched pixels. */
long long lo_expand_cells(lo_ctx *c, int iter, int level, const int *cells, int ncell, long long *evals) {
    double rd, rn;
    outer_delta(c, iter, &rd, &rn);
    long long acc = 0, ev = 0;
    int nt = c->p.n_threads;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : acc, ev) num_threads(nt > 0 ? nt : omp_get_max_threads())
    for (int k = 0; k < ncell; k++) {
        long long a = 0, e = 0;
        iterative_expansion(c, iter, level, cells[2 * k], cells[2 * k + 1], rd, rn, &a, &e);
        acc += a;
        ev += e;
    }
    if (evals) *evals = ev;
    return acc;
}

/* Every candidate of the visit of cell (i, j) at `level` in outer iteration
 * `iter`, drawn from the labels `lab` (H x W x 3) as the visit draws them when
 * no move happens in between (Algorithm 2 with the outer perturbation sizes of
 * Algorithm 1).  out: room for the visit's proposal count x 3 floats, or NULL.
 * Returns that count. */
int lo_visit_candidates(const lo_ctx *c, const float *lab, int iter, int level, int ci, int cj, float *out) {
    const int nprop = visit_proposals(c, level);
    if (!out) return nprop;
    double rd, rn;
    outer_delta(c, iter, &rd, &rn);
    draw_candidates(c, lab, iter, level, ci, cj, 0, nprop, &rd, &rn, (float(*)[3])out);
    return nprop;
}

/* One outer iteration of Algorithm 1: every grid level, every group. */
long long lo_iterate(lo_ctx *c, int iter, long long *evals) {
    long long acc = 0, ev = 0;
    for (int l = 0; l < c->p.n_levels; l++)
        for (int g = 0; g < 16; g++) {
            long long e = 0;
            acc += lo_expand_group(c, iter, l, g, &e);
            ev += e;
        }
    if (evals) *evals = ev;
    return acc;
}

/* Cells (i, j) of group k at grid size s, in the order lo_expand_group
 * visits them; returns the count (out may be NULL). */
int lo_group_cells(int H, int W, int s, int group, int *out) {
    const int nx = (W + s - 1) / s, ny = (H + s - 1) / s;
    const int gi = group % 4, gj = group / 4;
    const int cx = gi < nx ? (nx - gi + 3) / 4 : 0;
    const int cy = gj < ny ? (ny - gj + 3) / 4 : 0;
    if (out)
        for (int k = 0; k < cx * cy; k++) {
            out[2 * k] = gi + 4 * (k % cx);
            out[2 * k + 1] = gj + 4 * (k / cx);
        }
    return cx * cy;
}

int lo_openmp_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
