/*
 * lem.h -- C ABI of the GB300 (sm_103a) local-expansion-move stereo library.
 *
 * Method: Taniai, Matsushita, Sato, Naemura, "Continuous 3D Label Stereo
 * Matching using Local Expansion Moves" (arXiv 1603.08328).  Every pixel p of
 * the left image carries a disparity plane f_p = (a, b, c), d_p = a u + b v + c
 * (Sec. 3.2), and the energy E(f) = sum_p phi_p(f_p) + lambda sum_pq psi_pq
 * (Eq. mrf) is lowered by local alpha-expansions on 3x3-cell regions
 * (Sec. 3.3, Algorithms 1-2).
 *
 * Conventions for every entry point:
 *  - All functions return an int status (LEM_OK = 0, negative on error) and
 *    never throw, trap or abort.  lem_last_error() gives the text of the last
 *    failure on a handle.
 *  - Work is ordered on the CUDA stream given in lem_params.stream (NULL: the
 *    legacy default stream).  Outputs written to device memory are valid once
 *    that stream has been synchronised; the library does not synchronise unless
 *    a function says so.
 *  - Pointers documented as "device" must be device (or managed) memory owned
 *    by the caller; "host" pointers are read before the call returns.  The
 *    handle owns all memory it allocates and frees it in lem_destroy().
 *  - Images are 8-bit RGB, rows of `width` interleaved R,G,B triples.
 *  - Labels are float32 triples (a, b, c); pixel coordinates are 0-based pixel
 *    centres, u = column, v = row; a left pixel u matches right pixel u - d.
 */
#ifndef LEM_H
#define LEM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define LEM_OK 0
#define LEM_ERR_ARG (-1)           /* bad argument (null pointer, value out of range) */
#define LEM_ERR_SHAPE (-2)         /* image or region shape mismatch / too large        */
#define LEM_ERR_CUDA (-3)          /* a CUDA call failed (text in lem_last_error)        */
#define LEM_ERR_MAXFLOW_LIMIT (-4) /* a min-cut hit its round limit (labels kept)        */
#define LEM_ERR_OOM (-5)           /* device allocation failed                           */

/* internal storage of the packed images */
#define LEM_DATA_GF 0
#define LEM_DATA_BF 1
#define LEM_STORE_F32 0
#define LEM_STORE_F16 1
#define LEM_STORE_BF16 2

/* largest expansion region (nodes) a single CTA min-cut holds in shared memory:
 * 75 x 75, i.e. 3x3 cells of 25 px.  Levels with larger regions (or whose data
 * term and cut need more shared memory than a CTA has) run each region on
 * several co-resident CTAs of a cooperative launch, with the graph in global
 * memory; the result is the same canonical cut. */
#define LEM_MAX_REGION_NODES 5625
/* largest cell size (pixels) of a grid level */
#define LEM_MAX_CELL 1024

/* element types of a lem_image */
#define LEM_IMG_U8 0   /* uint8 colours 0..255                                      */
#define LEM_IMG_F16 1  /* IEEE half, colours on the 0..255 scale                    */
#define LEM_IMG_BF16 2 /* bfloat16, colours on the 0..255 scale                     */
#define LEM_IMG_F32 3  /* float, colours on the 0..255 scale                        */

/* An image of H x W pixels, each `channels` values of type `dtype` of which the
 * first three are R, G, B (further channels, e.g. alpha, are ignored).  The
 * method's colour terms are those of 8-bit images (Sec. 3.2: colour L1 distance
 * truncated at tau_col on the 0..255 scale, BT.601 gray for the gradient, the
 * guide scaled to [0, 1]), so a float colour is rounded to the nearest integer
 * and clamped to [0, 255] when the handle is created; a uint8 image is taken as
 * it is.  A zero in channels, stride_px or dtype selects the default, so an
 * image initialised with the first five fields only is packed 8-bit RGB.
 * Ownership: read during lem_create* only (host images are copied). */
typedef struct {
    const void *data;    /* pixel (0, 0)                                                    */
    int height, width;
    int64_t stride_row;  /* bytes between rows (>= (width-1)*stride_px + channels*size)     */
    int on_device;       /* 1: `data` is device memory, 0: host memory                      */
    int channels;        /* values per pixel, 3..16 (0: 3)                                  */
    int64_t stride_px;   /* bytes between pixels, >= channels*size (0: channels*size)       */
    int dtype;           /* LEM_IMG_U8 (0), LEM_IMG_F16, LEM_IMG_BF16 or LEM_IMG_F32; the
                            data pointer and both strides are multiples of the element size */
} lem_image;

/* Parameters.  lem_default_params() fills the values of the paper's
 * experiments (Sec. 4, settings): e = 0.01^2, tau_col = 10, tau_grad = 2,
 * alpha = 0.9, 41x41 matching windows (r' = 10), lambda = 1, tau_dis = 1,
 * eps = 0.01, gamma = 10, 8-neighbourhood, cells 5/15/25 px with
 * {K_prop, K_rand} = {1,7}, {2,0}, {2,0}. */
typedef struct {
    int gf_radius;        /* r': regression window (2r'+1)^2, matching window (4r'+1)^2 */
    double gf_eps;        /* e in (Sigma_k + e U)^-1 (guide scaled to [0,1])            */
    double tau_col;       /* truncation of the colour L1 term (0..255 scale)            */
    double tau_grad;      /* truncation of the gradient term                            */
    double alpha_grad;    /* alpha: weight of the gradient term                         */
    double lambda;        /* smoothness weight                                          */
    double tau_dis;       /* truncation of psi-bar                                      */
    double eps_w;         /* lower bound of the contrast weight w_pq                    */
    double gamma;         /* contrast weight scale                                      */
    double disp_min;      /* disparity range of the random init / perturbation          */
    double disp_max;
    int n_levels;         /* number of grid levels (<= 3)                               */
    int cell[3];          /* cell size in pixels per level, 1..LEM_MAX_CELL; a level whose
                             3x3-cell regions exceed LEM_MAX_REGION_NODES uses the multi-CTA
                             path: lem_expand_iteration then launches directly (no CUDA graph)
                             and lem_autotune leaves that level as it is                  */
    int k_prop[3];        /* propagation proposals per region visit, per level          */
    int k_rand[3];        /* perturbation proposals per region visit, per level         */
    double quant_scale;   /* S: every energy term is quantised as rne(S x)              */
    int store_dtype;      /* LEM_STORE_F32 (default), _F16, _BF16                        */
    double cond_fp64;     /* 3x3 inverses with a larger condition estimate use FP64     */
    uint64_t seed;        /* seed of all random draws                                   */
    void *stream;         /* cudaStream_t                                               */
    int max_rounds;       /* push-relabel round limit per cut                           */
    int gr_interval;      /* push-relabel rounds between global relabels                */
    int strip_rows;       /* rows per strip of the cost-aggregation pipeline            */
    int threads;          /* threads per CTA of the batch data-term/graph kernels       */
    int use_graph;        /* 1: lem_expand_iteration replays outer iterations as a CUDA graph */
    int candidates_per_visit; /* 1 (default): Algorithm 2 as printed, each proposal drawn from the
                                 labels left by the previous move.  K in 2..8: batched schedule, the
                                 candidates of each run of K proposals are drawn from the labels at
                                 the start of the run (perturbation size still halved per
                                 candidate), then cut in order, each against the updated labels. */
    int k_cnn[3];         /* map proposals per region visit, per level (default 0: the method as
                             published).  Proposal indices K_prop .. K_prop + k_cnn - 1 of a visit
                             take alpha = m_r, the proposal map's label at a pixel r drawn
                             uniformly from the centre cell (as propagation draws f_r); the
                             perturbations follow.  Needs a map (lem_set_proposals or
                             lem_cnn_propose) before the first expansion. */
    /* Launch configuration of the expansion kernel per grid level (0 = the default).
     * None of them changes a result: each cost is summed in a fixed order by one
     * thread and the cut is the unique minimal one.  lem_autotune picks them. */
    int level_threads[3];     /* threads per CTA: 128, 256, 512 or 1024; default by region size
                                 (<= 400 nodes: 256, <= 2500: 512, else 1024)               */
    int level_gr_interval[3]; /* push-relabel rounds between global relabels; default gr_interval
                                 (CTA path) or max(gr_interval, 64) (multi-CTA path)          */
    int level_strip_rows[3];  /* rows per strip of the cost pipeline; default strip_rows         */
    int k_rans[3];        /* RANSAC proposals per region visit, per level (Algorithm 2, RANSAC proposal;
                             default 0, the paper's setting outside its V3 experiments, where it
                             uses 1).  Proposal indices K_prop .. K_prop + k_rans - 1 take the plane
                             LO-RANSAC fits to the current disparities of the centre cell: 32
                             three-pixel hypotheses drawn from the proposal's stream, 1 px inliers,
                             the best refined twice by least squares. */
    int data_term;        /* LEM_DATA_GF (default): guided-filter weights (Eq. gf, LE-GF);
                             LEM_DATA_BF: bilateral weights exp(-|I_p - I_s|_1 / bf_gamma) over the
                             (4r'+1)^2 window, not normalised, O(|W|) per pixel (Sec. 4, LE-BF; the
                             paper uses lambda = 20 with it) */
    double bf_gamma;      /* LE-BF weight scale on 0..255 colours (default 10)                     */
    int cluster_visits;   /* 1 (default): a level whose visit is two propagation candidates (K_prop = 2,
                             no other proposal) runs two CTAs per region as a cluster when its regions
                             leave SMs idle (two CTAs per region fit in one wave): the second CTA
                             computes the data term of the second candidate as drawn before the first
                             move while the first CTA makes that move; the first move can only turn
                             f_r into alpha_1, so the second move then takes its data term from one of
                             the two planes.  Same labels as 0 (one CTA), bit for bit. */
    int split_visits;     /* batched visits (candidates_per_visit >= 2) on the guided-filter data term,
                             without RANSAC proposals, at levels whose regions are at most
                             LEM_MAX_REGION_NODES nodes and whose filtering regions are at most 128 px
                             wide: 1 runs each visit as two launches, the data terms of all its
                             candidates (one warp per region and candidate, exact fixed-point window
                             sums) and then its moves (one CTA per region; level_threads is that CTA's
                             size, 32 .. 1024); 0 (default) runs the visit in one kernel.  The moves
                             are the same; the data terms differ only in FP32 rounding. */
    int work_queue;       /* 1: one-kernel expansion launches run as many CTAs as fit on the GPU at
                             once, each taking regions from a work queue (largest first) until none
                             is left; 0 (default): one CTA per region.  The regions of a group are
                             independent, so the results are the same. */
    int dataflow;         /* 1: lem_expand_iteration runs each level as one launch instead of 16: the
                             regions of all 16 groups drain one work queue in group order, and a region
                             starts once every region of an earlier group within three cells of it (the
                             regions whose moves read or write its labels or the one-pixel ring around
                             them) is done.  Regions that touch each other still move in group order
                             and the others commute, so the labels are those of the 16 group launches,
                             bit for bit; a slow region holds up only its neighbours.  Levels with
                             split_visits or the multi-CTA cut keep their group launches; the two-CTA
                             cluster visit is not used.  0 (default): one launch per group. */
} lem_params;

/* An expansion region R (clipped to the image): columns [x0, x0+w), rows
 * [y0, y0+h) of pair `img` of the handle (0 for a single-pair handle).  The
 * centre cell C of a 3x3-cell region (Sec. 3.3: the region is C grown by one
 * cell; its propagation candidate is the label of a pixel of C) may be given in
 * cx0, cy0, cw, ch; it must then lie inside R.  The batch calls do not read it
 * (their candidates are passed in); cw = ch = 0 leaves it unset. */
typedef struct {
    int x0, y0, w, h;
    int img;                /* pair index, 0 .. lem_pair_count(h) - 1 */
    int cx0, cy0, cw, ch;   /* centre cell (optional)                  */
} lem_region;

/* Counters (evals, accepted, maxflow_limit) cover the work done since the
 * previous call on the same handle that returned stats (or since lem_create). */
typedef struct {
    int64_t energy_q;      /* sum_p Q(phi_p) + sum_pq Q(lambda psi_pq), Q(x) = rne(S x) */
    double energy;         /* energy_q / S                                             */
    int64_t evals;         /* pixel-label cost evaluations done                        */
    int64_t accepted;      /* pixels that switched to a candidate label                */
    int64_t maxflow_limit; /* cuts that hit the round limit                            */
    int32_t fp64_inverses; /* guide-covariance inverses taken in FP64 (lem_create)     */
    int32_t iterations;    /* outer iterations done so far on this handle              */
    int64_t pr_rounds;     /* push-relabel rounds (all cuts)                           */
    int64_t pr_global_relabels; /* global relabels (all cuts)                          */
    int64_t pr_bfs_levels; /* BFS frontiers processed by the global relabels           */
    int64_t accepted_by_kind[4]; /* switched pixels by proposal kind: propagation, RANSAC,
                                    map (learned proposer), perturbation                   */
    int64_t dep_waits_given_up; /* dataflow launches: regions that stopped waiting for a
                                   neighbour after the wait limit (about 2 s) and moved anyway;
                                   nonzero means the labels are not valid (reported by
                                   lem_expand_iteration as LEM_ERR_CUDA when stats are read) */
    double ms;             /* lem_expand_iteration: GPU time of the iterations of this call (CUDA
                              events on the handle's stream around them); 0 from other calls  */
} lem_stats;

typedef struct lem_handle lem_handle;

/* Fills `p` with the paper's parameter values (Sec. 4, settings of the
 * experiments: cells 5 / 15 / 25, {K_prop, K_rand} = {1, 7}, {2, 0}, {2, 0}, the
 * data-term and smoothness constants; see lem_params).  disp_max is set to 60;
 * callers set it to their range. */
void lem_default_params(lem_params *p);

/* The paper's settings for the Middlebury V3 benchmark (Sec. 4): the three cell
 * sizes become 1, 3 and 9 % of the image width (rounded to the nearest pixel,
 * at least 1 px), lambda = 0.5 and one RANSAC proposal per visit at every level
 * (K_RANS = 1); every other field of `p` is kept.  The paper's MC-CNN matching
 * cost is not part of this library: the data term stays the one `p` selects.
 * Errors: LEM_ERR_ARG (p NULL, width < 1). */
int lem_v3_params(lem_params *p, int width);

/* Creates a handle for one rectified pair.  Copies both images to the device,
 * packs (R, G, B, x-gradient of gray) per pixel (Sec. 3.2, data term: gradient
 * kernel [-0.5 0 0.5], BT.601 gray, edge pixels replicated), computes the
 * guide statistics mu_k and (Sigma_k + eU)^-1 over every clipped window W'_k
 * (Eq. gf), the contrast weights lambda*max(w_pq, eps) of the 4 forward
 * neighbours (Eq. smweight), draws the random initial labels (Sec. 3.4:
 * random disparity in [disp_min, disp_max] and random unit normal) and fills
 * the cost cache phi_p(f_p).  left/right: same height and width, each at
 * least one regression window (2 gf_radius + 1 pixels), any layout and element
 * type lem_image describes (converted to packed 8-bit RGB on the device first).
 * Errors: LEM_ERR_ARG (null pointers, bad parameters, an unknown dtype, fewer
 * than 3 or more than 16 channels, a pointer or stride that is not a multiple
 * of the element size), LEM_ERR_SHAPE (sizes, strides), LEM_ERR_OOM,
 * LEM_ERR_CUDA.  On error *out is NULL. */
int lem_create(const lem_image *left, const lem_image *right, const lem_params *p, lem_handle **out);

/* A handle for n_pairs independent pairs (sizes may differ), each prepared as by
 * lem_create (Sec. 3.2) and solved together:
 * each (level, group) launch of lem_expand_group / lem_expand_iteration runs
 * the regions of every pair (pairs are independent, so their regions never
 * interact).  Pair b draws its random numbers from seed + b * 0x9E3779B97F4A7C15,
 * so pair 0 of a batch reproduces lem_create with the same parameters.  The
 * label, cost and plane arrays of lem_get_labels, lem_set_labels and
 * lem_get_planes hold the pairs in order, each row-major (see lem_pair_info);
 * lem_energy sums over the pairs.  The batch entry points (lem_unary_batch,
 * lem_pairwise_batch, lem_mincut_batch) take each region's pair from its img.
 * Errors as lem_create; n_pairs must be in [1, 4096]. */
int lem_create_batch(const lem_image *lefts, const lem_image *rights, int n_pairs, const lem_params *p,
                     lem_handle **out);

/* lem_create_batch with a disparity range per pair: disp_ranges holds
 * (disp_min, disp_max) of pair b at [2b], [2b+1] (HOST, copied; NULL: the
 * range of `p` for every pair).  The range bounds the pair's random initial
 * labels and perturbations (Sec. 3.4) and scales its network input.
 * Errors as lem_create_batch, and LEM_ERR_ARG for a range that is not finite
 * with max >= min. */
int lem_create_batch_ranges(const lem_image *lefts, const lem_image *rights, int n_pairs,
                            const double *disp_ranges, const lem_params *p, lem_handle **out);

/* Number of pairs of a handle (-1 for NULL).  Handle bookkeeping; the paper
 * has no counterpart. */
int lem_pair_count(const lem_handle *h);

/* Height, width and first pixel index (in the concatenated per-pixel arrays)
 * of pair `pair`.  Any output may be NULL.  Errors: LEM_ERR_ARG. */
int lem_pair_info(const lem_handle *h, int pair, int *height, int *width, int64_t *pixel_offset);

/* Quantised energy of one pair (Eq. mrf; see lem_energy).  Synchronises the stream.
 * Errors: LEM_ERR_ARG, LEM_ERR_CUDA. */
int lem_energy_pair(lem_handle *h, int pair, double *energy, int64_t *energy_q);

/* Frees the handle and everything it owns.  NULL is accepted.  Handle
 * bookkeeping; the paper has no counterpart. */
int lem_destroy(lem_handle *h);

/* Text of the last error on `h` (or of the last failed lem_create when h is
 * NULL).  The pointer stays valid until the next call on the same handle. */
const char *lem_last_error(const lem_handle *h);

/* Data term phi_p(alpha) (Eq. unary_term with the guided-filter weights of
 * Eq. gf, count-normalised at the image border) for every p of each region and
 * each of its K candidate labels, computed per region through the filtering
 * region M (Sec. 3.5): raw costs rho(s|alpha) (Eqs. warp, photofunc; linear
 * interpolation along u, u' clamped to [0, W-1]) over R grown by 2r', guided-
 * filter coefficients over R grown by r', their window means over R.
 *   regions : host, n_regions entries, each inside the image of its pair img, w*h >= 1
 *   labels  : device float32, n_regions*K*3: candidate k of region i at (i*K+k)*3
 *   costs   : device float32, packed region-major: region i starts at
 *             K * sum_{j<i} w_j*h_j; within it candidate k occupies w_i*h_i
 *             values, row-major over R.
 * Errors: LEM_ERR_ARG (also img out of range), LEM_ERR_SHAPE (region outside
 * its image, centre cell outside the region), LEM_ERR_CUDA. */
int lem_unary_batch(lem_handle *h, const lem_region *regions, int n_regions, const float *labels, int K,
                    float *costs);

/* Binary expansion-move graph of each region against the handle's current
 * labels and cost cache (Sec. 3.3; footnote to Lemma 2: neighbours outside R
 * fold into the unaries; pairs inside R use the A + (C-A)x_p + (D-C)x_q +
 * (B+C-A-D)(1-x_p)x_q decomposition with D = 0, valid by Lemma 1).  Every term
 * is quantised as rne(S x); a quantised A above B + C is lowered to B + C.
 * x_p = 1 (take alpha) puts p on the sink side.
 *   regions     : host, n_regions entries (at most LEM_MAX_REGION_NODES nodes each), against
 *                 the labels of pair img
 *   alpha       : device float32, n_regions*3
 *   costs_alpha : device float32, phi_p(alpha) packed as lem_unary_batch with K = 1
 *   tcaps       : device int32, 2 per node {s->p: U_p(1)-m, p->t: U_p(0)-m}, packed like costs_alpha
 *   ncaps       : device int32, 4 per node: capacity of p->q for the forward
 *                 neighbours q = p+(1,0), p+(-1,1), p+(0,1), p+(1,1) inside R, else 0
 *   const_term  : device int64, n_regions: energy of the terms touching R minus the cut
 * Errors: LEM_ERR_ARG, LEM_ERR_SHAPE, LEM_ERR_CUDA. */
int lem_pairwise_batch(lem_handle *h, const lem_region *regions, int n_regions, const float *alpha,
                       const float *costs_alpha, int32_t *tcaps, int32_t *ncaps, int64_t *const_term);

/* Minimum s-t cut of each region graph (layout of lem_pairwise_batch): the exact
 * solution of one alpha_ij-expansion's binary problem (Eq. expansion, Sec. 3.3),
 * which is submodular by Lemma 2 and is solved by graph cuts.  Computed by
 * push-relabel with global relabelling, one CTA per region, in shared memory.
 * When some region exceeds LEM_MAX_REGION_NODES (any size up to the image is
 * accepted here) every region of the call runs on the multi-CTA path instead:
 * several co-resident CTAs per region, the graph in global memory (scratch
 * allocated by the call), same result.
 * take_alpha[p] = 1 iff p can reach the sink in the residual graph of the
 * maximum preflow: the unique minimal sink side among all minimum cuts.
 *   take_alpha : device uint8, 1 per node, packed like costs_alpha
 *   flow       : device int64, n_regions: max-flow value (= min-cut value)
 *   status     : device int32, n_regions: LEM_OK or LEM_ERR_MAXFLOW_LIMIT (LEM_ERR_CUDA on the
 *                multi-CTA path if a region barrier gave up after 1 s)
 * Errors: LEM_ERR_ARG, LEM_ERR_SHAPE, LEM_ERR_CUDA.  A region that hits the
 * round limit only sets its status; the call still returns LEM_OK. */
int lem_mincut_batch(lem_handle *h, const lem_region *regions, int n_regions, const int32_t *tcaps,
                     const int32_t *ncaps, uint8_t *take_alpha, int64_t *flow, int32_t *status);

/* All alpha_ij-expansions of one disjoint group k = 4 (j mod 4) + (i mod 4)
 * (Eq. groupindex) at grid level `level` of outer iteration `iter`, in one
 * launch (one CTA per region, Lemma 3): each region runs Algorithm 2
 * (K_prop propagation proposals, then K_rand perturbation proposals with the
 * perturbation size halved after each; outer sizes r_d = (disp_max-disp_min)/2
 * and r_n = 1 halved per iteration), each proposal evaluated, cut and committed
 * in turn.  Updates the handle's labels and cost cache.  Does not advance the
 * handle's iteration counter.  stats may be NULL (no synchronisation); when
 * given, the call synchronises the stream and fills evals/accepted/maxflow_limit
 * (energy fields are left 0).  Errors: LEM_ERR_ARG, LEM_ERR_CUDA. */
int lem_expand_group(lem_handle *h, int iter, int level, int group, lem_stats *stats);

/* n_iters outer iterations of Algorithm 1 (every level, all 16 groups),
 * continuing from the handle's iteration counter.  With params.use_graph the
 * first call runs one iteration directly and captures one iteration (48
 * group launches, or with params.dataflow 3 level launches and the memsets of
 * their done flags, and the increment of a device-side iteration index) as a
 * CUDA graph on a private stream; later iterations replay that graph on the
 * handle's stream (a handle with a level on the multi-CTA path always launches
 * directly).  stats may be NULL (no synchronisation); when given, the call
 * synchronises and fills all fields (energy after the last iteration).
 * Errors: LEM_ERR_ARG, LEM_ERR_CUDA. */
int lem_expand_iteration(lem_handle *h, int n_iters, lem_stats *stats);

/* Current labels and cost cache.  abc: float32 H*W*3, disp: float32 H*W
 * (d_p = a u + b v + c, Eq. disparity_plane), cost: phi_p(f_p) (Eq. unary_term),
 * float32 H*W; any may be NULL; `on_device` says whether the pointers are
 * device (1) or host (0) memory.  Host copies synchronise the stream.  Errors: LEM_ERR_ARG, LEM_ERR_CUDA. */
int lem_get_labels(lem_handle *h, float *abc, float *disp, float *cost, int on_device);

/* Replaces the labels (float32 H*W*3; planes of Eq. disparity_plane) and, when
 * `cost` is not NULL, the cost cache (float32 H*W, taken as phi_p(f_p) of
 * Eq. unary_term for the new labels); with cost NULL
 * the cache is recomputed by the data term.  on_device as in lem_get_labels.
 * Errors: LEM_ERR_ARG, LEM_ERR_CUDA. */
int lem_set_labels(lem_handle *h, const float *abc, const float *cost, int on_device);

/* Quantised energy of the current labels (Eq. mrf, each unordered
 * 8-neighbour pair once): *energy_q = sum_p Q(phi_p) + sum Q(lambda psi_pq),
 * *energy = *energy_q / S.  Synchronises the stream.  Either pointer may be
 * NULL.  Errors: LEM_ERR_ARG, LEM_ERR_CUDA. */
int lem_energy(lem_handle *h, double *energy, int64_t *energy_q);

/* Device views of the handle's packed planes (for tests): left/right packed
 * pixels (4 floats: R, G, B, gradient; Sec. 3.2, data term) as float32 H*W*4, guide statistics as
 * float32 H*W*9 {mu_r, mu_g, mu_b, A00, A01, A02, A11, A12, A22}, and
 * lambda*max(w, eps) for the 4 forward neighbours as float32 H*W*4.  Copies
 * into caller device buffers; any may be NULL.  Errors: LEM_ERR_ARG, LEM_ERR_CUDA. */
int lem_get_planes(lem_handle *h, float *left, float *right, float *guide, float *weights);

/* Measures the current device's FP32 fused multiply-add throughput and its
 * shared-memory load bandwidth (16-byte conflict-free loads), each the best of
 * five timed launches of a microbenchmark kernel over every SM, on `stream`
 * (cudaStream_t, NULL: the legacy default stream).  These are the roofs the data
 * term is reported against; the paper has no counterpart.  Synchronises the
 * stream.  Errors: LEM_ERR_ARG (NULL output), LEM_ERR_OOM, LEM_ERR_CUDA. */
int lem_measure_peaks(void *stream, double *fp32_tflops, double *smem_gbs);

/* Kinds of the expansion launches that lem_get_kernel_times reports. */
#define LEM_KERNEL_EXPAND 0       /* one-kernel visits (k_expand_group)                      */
#define LEM_KERNEL_VISIT_UNARY 1  /* data terms of a batched visit (k_visit_unary)           */
#define LEM_KERNEL_VISIT_CUT 2    /* moves of a batched visit (k_visit_cut)                   */
#define LEM_KERNEL_GRID 3         /* multi-CTA regions (k_expand_grid)                        */
#define LEM_KERNEL_KINDS 4
typedef struct {
    double ms[3][LEM_KERNEL_KINDS];       /* GPU time per level and kind, from CUDA events between launches */
    int64_t launches[3][LEM_KERNEL_KINDS];
} lem_kernel_times;

/* Kernel timing of lem_expand_iteration (a measurement aid; the paper has no
 * counterpart).  With on = 1 every outer iteration records a CUDA event on the
 * handle's stream before its first launch and after each expansion launch (as
 * event nodes of the CUDA graph when iterations are replayed as one); results
 * are unchanged.  Turning it on or off drops the captured graph, which the
 * next lem_expand_iteration captures again.  Errors: LEM_ERR_ARG. */
int lem_set_kernel_timing(lem_handle *h, int on);
/* Time of each launch kind at each level in the last outer iteration issued
 * on the handle
 * (events are overwritten by every iteration, so call it after each one; the
 * time between two events is the launch between them).  Synchronises the
 * stream.  All zero when timing is off.  Errors: LEM_ERR_ARG, LEM_ERR_CUDA. */
int lem_get_kernel_times(lem_handle *h, lem_kernel_times *out);

/* Largest n_regions of lem_mincut_batch_noalloc. */
#define LEM_NOALLOC_MAX_REGIONS 4096

/* The cut of lem_mincut_batch for callers that cannot allocate device memory
 * when they cut: code that runs inside a preallocated memory arena, a host
 * thread that must not call cudaMalloc/cudaFree because those synchronise the
 * device, or an embedding that forbids growing the device heap.  The paper has
 * no counterpart for the allocation-free form; the cut is the same.
 *
 * It needs no handle and allocates nothing: the scratch the batch min-cut
 * keeps per call (region descriptors, packed offsets, work counters) is a
 * fixed array of about 96 KiB in the library's device memory, which every GPU
 * that loads the library holds until the process exits.  The first call on a
 * device looks up that array's device address (once per device, with that
 * device current) and keeps it for the life of the process.  A
 * cudaDeviceReset unloads the array, so this entry point must not be called
 * after a device reset in the same process.  Every call shares the array and overwrites it (the counters are
 * cleared first), so calls whose work overlaps on the GPU race: order them on
 * one stream, or synchronise between them.
 *
 * `regions` is copied to the device with cudaMemcpyAsync on `stream`.  From
 * page-locked host memory (cudaHostAlloc / cudaHostRegister) that copy is
 * asynchronous; from pageable memory the call may return only once the copy
 * has been staged, which can wait for earlier work on the stream.  Callers
 * that must not block pass page-locked `regions`.
 *   regions     : host, n_regions <= LEM_NOALLOC_MAX_REGIONS entries, each
 *                 region at most LEM_MAX_REGION_NODES nodes; x0, y0, img and the
 *                 centre cell are ignored
 *   tcaps/ncaps : device int32, layout of lem_pairwise_batch
 *   take_alpha, flow, status : device outputs as in lem_mincut_batch
 *   max_rounds, gr_interval  : as in lem_params (>= 1)
 *   stream      : cudaStream_t (NULL: the legacy default stream)
 * Errors: LEM_ERR_ARG (NULL pointer, n_regions < 1 or above
 * LEM_NOALLOC_MAX_REGIONS, bad round parameters), LEM_ERR_SHAPE (an empty or
 * too large region), LEM_ERR_CUDA; the text is in lem_last_error(NULL). */
int lem_mincut_batch_noalloc(const lem_region *regions, int n_regions, const int32_t *tcaps, const int32_t *ncaps,
                             uint8_t *take_alpha, int64_t *flow, int32_t *status, int max_rounds, int gr_interval,
                             void *stream);

/* The candidate labels of one visit (Algorithm 2; the RANSAC and map candidates
 * included) of each listed cell of pair 0 at grid level `level` and outer
 * iteration `iter`, drawn from the current labels as lem_expand_group draws
 * them when no move happens in between: proposal t of cell k is alpha[(k *
 * nprop + t) * 3 .. + 2], nprop = k_prop + k_rans + (k_cnn if a map is set) +
 * k_rand of that level.  cells: HOST, n_cells pairs (i, j); alpha: DEVICE.
 * Synchronises the stream.  Errors: LEM_ERR_ARG, LEM_ERR_SHAPE (cell outside
 * the grid), LEM_ERR_CUDA. */
int lem_propose_batch(lem_handle *h, int iter, int level, const int *cells, int n_cells, float *alpha);

/* ------------------------------------------------------------------------- */
/* Right view and post-processing (Sec. 3.2 after Eq. photofunc, Sec. 3.4 end) */
/* ------------------------------------------------------------------------- */

/* A handle that estimates the RIGHT image's labels.  The data term of the right
 * view swaps the images and adds the disparity in the warp; that is the left-view
 * problem of the horizontally mirrored pair, so the handle is created on
 * (mirror(right), mirror(left)) and its labels, cost cache and energy live in
 * mirrored coordinates: right pixel (u, v) is label (W - 1 - u, v), and a
 * mirrored plane (a', b', c') is the right-image plane (-a', b', c' + a' (W - 1)).
 * Everything else (iterations, energy, batch calls) works as on any handle.
 * The images are read once, as by lem_create.  Errors as lem_create. */
int lem_create_right_view(const lem_image *left, const lem_image *right, const lem_params *p, lem_handle **out);

/* Post-processing parameters.  The paper applies the left-right consistency
 * check and weighted median filtering of Bleyer et al. (2011) without giving
 * their settings; the defaults are that paper's: a 1-pixel consistency
 * threshold, a 41 x 41 median window and gamma = 10 on 0..255 colours. */
typedef struct {
    float lr_threshold;   /* |d_L(p) - d_R(q)| <= lr_threshold marks p consistent            */
    int median_radius;    /* window (2 r + 1)^2, clipped to the image; 0..64                  */
    float median_gamma;   /* weight exp(-|I_p - I_q|_1 / gamma) on the left colours          */
} lem_post_params;
/* Fills `pp` with the defaults above (threshold 1, radius 20, gamma 10); a NULL
 * pointer is ignored. */
void lem_default_post_params(lem_post_params *pp);

/* Final disparity map of pair 0 of hL (left view) with hR from
 * lem_create_right_view on the same images:
 *   1. p is consistent when q = (rint(u - d_L(p)), v) lies in the image and
 *      |d_L(p) - d_R(q)| <= lr_threshold (disparities (a u + b v) + c in FP32);
 *   2. an inconsistent p takes, of the nearest consistent pixels to its left and
 *      right on its row, the plane giving the lower disparity at p (occlusions are
 *      filled from the background);
 *   3. an inconsistent p's disparity becomes the weighted median of the filled
 *      disparities in its window: the smallest window value whose cumulative
 *      weight, in ascending order of value, reaches half the total.
 * disp: DEVICE, H*W floats (final disparities); valid: DEVICE, H*W bytes (1 =
 * consistent) or NULL.  Synchronises hL's stream (and hR's when it differs).
 * Errors: LEM_ERR_ARG, LEM_ERR_SHAPE (views of different sizes), LEM_ERR_OOM,
 * LEM_ERR_CUDA. */
int lem_postprocess(lem_handle *hL, lem_handle *hR, const lem_post_params *pp, float *disp, uint8_t *valid);

/* Autotuner result: the per-level launch configuration chosen, its time per
 * (level, group) launch and that of the default configuration. */
typedef struct {
    int threads[3];
    int gr_interval[3];
    int strip_rows[3];
    float ms[3];           /* mean time of one (level, group) launch, chosen configuration */
    float ms_default[3];   /* same, default configuration                                   */
    int configs_tried;     /* candidate configurations timed (all levels)                   */
} lem_tuning;

/* Launch-shape tuning; the paper has no counterpart, and labels never depend
 * on it.  Times the expansion kernel of every level on this handle's own images and
 * labels for each candidate configuration (threads {128, 256, 512, 1024} x
 * gr_interval {8, 16, 32, 64} x strip_rows {8, 12, 16, 24, 32}; candidates whose shared
 * memory does not fit are skipped), `repeats` launches of groups 0 and 10 of
 * the level at the handle's current iteration each, and keeps the fastest per
 * level in the handle's parameters (level_threads, level_gr_interval,
 * level_strip_rows).  Labels, cost cache and statistics counters are restored
 * after every trial, so the handle's state is unchanged; a captured iteration
 * graph is rebuilt on the next lem_expand_iteration.  Synchronises the stream.
 * out may be NULL.  Errors: LEM_ERR_ARG (repeats outside 1..100),
 * LEM_ERR_MAXFLOW_LIMIT (a trial cut hit the round limit), LEM_ERR_OOM, LEM_ERR_CUDA. */
int lem_autotune(lem_handle *h, int repeats, lem_tuning *out);

/* Number of pixel-label cost evaluations in one outer iteration of Algorithm 1
 * (sum over all region visits of |R| x proposals).  Host only. */
int64_t lem_evals_per_iteration(const lem_handle *h);

/* ------------------------------------------------------------------------- */
/* Learned proposer (an extension beyond the paper: its proposals are the     */
/* random propagation and perturbation of Sec. 3.3).                          */
/* ------------------------------------------------------------------------- */

/* Proposal map of pair `pair` (H*W labels (a, b, c), row-major, 3 floats per
 * pixel, DEVICE pointer; copied, so the caller keeps ownership), read by the
 * k_cnn map proposals.  Errors: LEM_ERR_ARG (NULL, pair out of range, or
 * every k_cnn is 0: the handle keeps no map), LEM_ERR_CUDA. */
int lem_set_proposals(lem_handle *h, int pair, const float *abc_dev);
/* The proposal map of pair `pair` into a DEVICE array of H*W*3 floats.
 * Errors: LEM_ERR_ARG (also when no map was set), LEM_ERR_CUDA. */
int lem_get_proposals(lem_handle *h, int pair, float *abc_dev);

/* The proposal network: 6 layers of 3x3 convolutions (zero padding), 32
 * channels, ReLU after all but the last; input (H4, W4, 7) = left RGB, right
 * RGB (/255) and label disparity (/disp_max) at quarter resolution (4x4 block
 * means, H4 = ceil(H/4), W4 = ceil(W/4)); output (H4, W4, 3) = (d/disp_max, a,
 * b).  BF16 tensor-core convolutions with FP32 accumulation (forward and input
 * gradient on tcgen05 with a TMEM accumulator, weight gradient on mma.sync);
 * FP32 master weights trained by Adam on an L1 loss.  Runs on the stream given at creation
 * (NULL: legacy default stream). */
typedef struct lem_cnn lem_cnn;

/* He-initialised network (normal weights from a SplitMix64 stream of `seed`,
 * zero biases).  Errors: LEM_ERR_ARG, LEM_ERR_OOM, LEM_ERR_CUDA. */
int lem_cnn_create(uint64_t seed, void *stream, lem_cnn **out);
/* Frees the network and its device buffers (NULL: nothing).  Returns LEM_OK. */
int lem_cnn_destroy(lem_cnn *net);
/* Text of the last error on `net` (NULL: of the last failed lem_cnn_create);
 * owned by the library, valid until the next call on the same network. */
const char *lem_cnn_last_error(const lem_cnn *net);
/* Synchronises the network's stream and reports LEM_ERR_CUDA if a convolution
 * tile gave up waiting for its tensor-core MMAs since the last check (the
 * kernels bound that wait and leave such a tile's output unwritten);
 * lem_cnn_gradients runs this check itself.  Errors: LEM_ERR_ARG, LEM_ERR_CUDA. */
int lem_cnn_check(lem_cnn *net);
/* Number of parameters: per layer, weights (3, 3, Cin, Cout) row-major, then the
 * Cout biases; layers in order (Cin, Cout) = (7,32), (32,32) x4, (32,3). */
int64_t lem_cnn_num_params(void);
/* All parameters to / from a HOST array of lem_cnn_num_params() floats, in that
 * order; set_params also refreshes the BF16 copies the kernels read.  Errors:
 * LEM_ERR_ARG (NULL), LEM_ERR_CUDA. */
int lem_cnn_get_params(lem_cnn *net, float *host);
int lem_cnn_set_params(lem_cnn *net, const float *host);
/* Forward pass: x DEVICE (H4*W4*7 floats), y DEVICE (H4*W4*3 floats).
 * Errors: LEM_ERR_ARG (also W4 > 1597: a convolution tile stages three rows of
 * the padded grid in shared memory), LEM_ERR_OOM, LEM_ERR_CUDA. */
int lem_cnn_forward(lem_cnn *net, const float *x, int H4, int W4, float *y);
/* Loss and gradients over n_images inputs x (DEVICE, n*H4*W4*7) with targets
 * t (DEVICE, n*H4*W4*3): loss = mean over images and pixels of
 * sum_c scale_c |y_c - t_c|.  scale: HOST, 3 floats.  loss: HOST float or NULL;
 * grads: HOST array in the lem_cnn_get_params order, or NULL.  All images go
 * through each layer together (one launch per layer and pass) on one
 * zero-padded grid, so the network holds activations for about
 * n*(H4+2)*(W4+2) positions (1.25 KB each; grown on demand, cleared when the
 * shape changes, kept until lem_cnn_destroy).  Synchronises the stream.
 * Errors: LEM_ERR_ARG (also when the grid exceeds 2^31 / 32 positions or
 * W4 > 1597), LEM_ERR_OOM, LEM_ERR_CUDA. */
int lem_cnn_gradients(lem_cnn *net, const float *x, const float *t, int n_images, int H4, int W4,
                      const float *scale, float *loss, float *grads);
/* lem_cnn_gradients, then one Adam step (beta 0.9 / 0.999, eps 1e-8, rate lr). */
int lem_cnn_train_step(lem_cnn *net, const float *x, const float *t, int n_images, int H4, int W4,
                       const float *scale, float lr, float *loss);
/* Network input of pair `pair` from its images and current labels into x
 * (DEVICE, H4*W4*7).  Errors: LEM_ERR_ARG, LEM_ERR_CUDA. */
int lem_cnn_features(lem_handle *h, int pair, float *x);
/* Training target of pair `pair` from its current labels: 4x4 block means of
 * (d/disp_max, a, b), the mean slopes clamped to [-1, 1], into t (DEVICE,
 * H4*W4*3).  Errors: LEM_ERR_ARG, LEM_ERR_CUDA. */
int lem_cnn_targets(lem_handle *h, int pair, float *t);
/* Features, forward pass and bilinear upsampling of (d, a, b) to a plane per
 * pixel (c = d - a u - b v), stored as the proposal map of every pair of `h`.
 * Stream-ordered on the handle's stream (no synchronisation; the first call
 * allocates the handle's quarter-resolution buffers).  Errors: LEM_ERR_ARG
 * (also when every k_cnn is 0), LEM_ERR_OOM, LEM_ERR_CUDA. */
int lem_cnn_propose(lem_cnn *net, lem_handle *h);

#ifdef __cplusplus
}
#endif

#endif /* LEM_H */
