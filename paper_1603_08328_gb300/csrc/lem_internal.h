// Internal declarations shared by the host API (lem_api.cu) and the kernels
// (lem_kernels.cu).  Not part of the public C ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "lem.h"

namespace lem {

// Device views of one pair's packed planes.
struct DevPlanes {
    int H, W;
    const void *L;      // left:  (R, G, B, x-gradient of gray), 0..255 scale, in format fmt
    const void *R;      // right: same
    int fmt;            // LEM_STORE_F32 (float4), LEM_STORE_F16 / LEM_STORE_BF16 (4 x 16 bit)
    const float4 *gst;  // 3 float4 per pixel: {mu_r, mu_g, mu_b, A00}, {A01, A02, A11, A12}, {A22, 0, 0, 0}
    const float4 *wfw;  // lambda * max(w_pq, eps) for the forward neighbours (1,0), (-1,1), (0,1), (1,1)
};

// Scalar parameters as the kernels use them.
struct KParams {
    int r;              // guided-filter radius r'
    float tau_col, tau_grad, alpha_grad;
    float tau_dis;
    float S;            // quantisation scale
    double disp_min, disp_max;
    unsigned long long seed;
    int max_rounds;     // push-relabel round limit
    int gr_interval;    // rounds between global relabels
    int T;              // strip rows of the aggregation pipeline
    int visit;          // candidates drawn per region visit (1: Algorithm 2)
    int bf;             // data term: 0 guided filter (LE-GF), 1 bilateral weights (LE-BF)
    float bf_log2e_inv_gamma; // LE-BF: log2(e) / gamma of the colour weights
    // fixed-point scales (powers of two) of the exact window sums of the warp
    // data term: q1 for the raw-cost channels (32-bit), q2 for the guided-filter
    // coefficients (64-bit); chosen on the host so no window sum can overflow
    float q1, q2;
};

// One stereo pair inside a batch handle: its size, the pixel offset of its
// planes in the concatenated arrays, and the seed of its random draws.
struct PairDesc {
    int H, W;
    long long off;
    unsigned long long seed;
    double disp_min, disp_max;  // disparity range of the pair's random draws
};

// One grid level of Algorithm 1.
struct Level {
    int s;              // cell size
    int k_prop, k_rand;
    int k_cnn;          // map candidates (after the RANSAC candidates)
    int k_rans;         // RANSAC plane candidates (proposal indices k_prop .. k_prop + k_rans - 1)
    int threads;        // CTA size of the expansion kernel (0: by region size)
};

// Per-launch counters written by the expansion kernels.
struct Counters {
    unsigned long long accepted;
    unsigned long long limit_hits;
    unsigned long long evals;
    unsigned long long rounds;      // push-relabel rounds
    unsigned long long relabels;    // global relabels
    unsigned long long bfs_levels;  // BFS frontiers summed over global relabels
    unsigned long long accepted_kind[4];  // switched pixels by proposal kind: propagation, RANSAC,
                                          // map (learned proposer), perturbation
    unsigned long long dep_give_ups;      // dataflow waits that reached their limit
};

// Shared-memory bytes the region cost pipeline needs for regions up to
// rw x rh pixels.
size_t unary_smem_bytes(const KParams &kp, int H, int W, int rw, int rh);
// Shared-memory bytes of the CTA min-cut for a w x h region.
size_t cut_smem_bytes(int w, int h);

// CTA size of the expansion and cut kernels for regions of n nodes
inline int threads_for_nodes(int n) { return n <= 400 ? 256 : (n <= 2500 ? 512 : 1024); }

// bytes per packed image pixel in format fmt
inline size_t px_bytes(int fmt) { return fmt == LEM_STORE_F32 ? 16 : 8; }
cudaError_t launch_preprocess(const uint8_t *left, int64_t lstride, const uint8_t *right, int64_t rstride, int H,
                              int W, float lambda, float eps_w, float gamma, void *Lp, void *Rp, int fmt,
                              float4 *wfw, cudaStream_t st);
cudaError_t launch_guide_stats(const uint8_t *left, int64_t lstride, int H, int W, int r, double eps,
                               double cond_fp64, float4 *gst, int *n_fp64, cudaStream_t st);
cudaError_t launch_init_labels(int H, int W, unsigned long long seed, double dmin, double dmax, float4 *lab,
                               cudaStream_t st);
// phi_p(f_p) for every pixel with its own label (1x1 regions).
cudaError_t launch_pixel_costs(const DevPlanes &P, const KParams &kp, float4 *lab, int threads, cudaStream_t st);
// The batch test surface.  P (and lab) are the base planes (labels) of all
// pairs, P.H / P.W the largest pair's size; region i belongs to pair img[i]
// (device array) and is offset to it by pairs[img[i]].
cudaError_t launch_unary_batch(const DevPlanes &P, const KParams &kp, const PairDesc *pairs, const int *img,
                               const int4 *regions, const int64_t *offsets, int n_regions, int K, int max_w,
                               int max_h, const float *labels, float *costs, int threads, cudaStream_t st);
cudaError_t launch_pairwise_batch(const DevPlanes &P, const KParams &kp, const PairDesc *pairs, const int *img,
                                  const int4 *regions, const int64_t *offsets, int n_regions, const float4 *lab,
                                  const float *alpha, const float *costs_alpha, int32_t *tcaps, int32_t *ncaps,
                                  int64_t *cterm, int threads, cudaStream_t st);
cudaError_t launch_mincut_batch(const KParams &kp, const int4 *regions, const int64_t *offsets, int n_regions,
                                int max_nodes, size_t smem, const int32_t *tcaps, const int32_t *ncaps, uint8_t *take,
                                int64_t *flow, int32_t *status, Counters *ctr, cudaStream_t st);
// All expansions of one (level, group) over every pair of the batch: items
// lists (pair, cell i, cell j); iter < 0 reads the iteration from *iter_dev.
// prop: proposal maps of all pairs (same offsets as lab), or NULL when lv.k_cnn == 0.
// phiB: a second data-term plane (same offsets as phiA), or NULL; with it, levels
// whose visit is two propagation candidates run two CTAs per region (a cluster)
// that compute both candidates' data terms at once, with the sequential result.
// queue: NULL (one CTA per item), or two zeroed ints of a work queue that a
// grid of co-resident CTAs drains (left zeroed after the launch); not with phiB.
// done: NULL, or (with queue, without phiB) one zeroed flag per cell of the
// level of every pair: the items are then those of all 16 groups of the level
// in group order, item.w is the index of its pair's cell (0, 0) in done, and
// an item waits for the items of earlier groups within three cells before it
// starts and sets its own flag when it is done (a dataflow launch of a level).
cudaError_t launch_expand_group(const DevPlanes &P, const KParams &kp, const Level &lv, int level, int iter,
                                const int *iter_dev, const PairDesc *pairs, int max_w, int max_h, const int4 *items,
                                int n_items, float4 *lab, float *phiA, const float4 *prop, Counters *ctr, float *phiB,
                                int *queue, unsigned *done, cudaStream_t st);
cudaError_t launch_increment(int *x, cudaStream_t st);
// Batched visits on the guided-filter data term without RANSAC proposals, regions
// of at most LEM_MAX_REGION_NODES nodes and filtering regions at most 128 px
// wide: a visit is a data-term launch (one warp per region and candidate, exact
// fixed-point window sums) and a cut launch (one CTA per region, the visit's
// moves in order).  phiK holds nK data-term planes of plane_stride floats,
// alphaK n_items * nK candidate labels.  lv.threads is the cut CTA's size
// (32 .. 1024; 0: by region size).
bool visit_split(const KParams &kp, const Level &lv, int max_w, int max_h);
// lem_unary_batch with the warp data term of that path (one warp per region and
// label), for regions at most max_w wide whose filtering region fits it
bool unary_warp_fits(const KParams &kp, int W, int max_w);
cudaError_t launch_unary_batch_warp(const DevPlanes &P, const KParams &kp, const PairDesc *pairs, const int *img,
                                    const int4 *regions, const int64_t *offsets, int n_regions, int K, int max_w,
                                    const float *labels, float *costs, cudaStream_t st);
int visit_cut_threads(int nodes);
cudaError_t launch_visit_unary(const DevPlanes &P, const KParams &kp, const Level &lv, int level, int iter,
                               const int *iter_dev, const PairDesc *pairs, int max_w, int max_h, const int4 *items,
                               int n_items, int t0, int nK, const float4 *lab, float *phiK, long long plane_stride,
                               const float4 *prop, float4 *alphaK, cudaStream_t st);
// (t0: first proposal index of the visit, kc: map candidates per visit, for the
// per-kind switch counts)
cudaError_t launch_visit_cut(const DevPlanes &P, const KParams &kp, const Level &lv, const PairDesc *pairs,
                             int max_w, int max_h, const int4 *items, int n_items, int t0, int nK, int kc,
                             float4 *lab, const float *phiK, long long plane_stride, const float4 *alphaK,
                             Counters *ctr, cudaStream_t st);
// Regions above the shared-memory cut (more than LEM_MAX_REGION_NODES nodes, or
// a data term + cut that needs more than a CTA's shared memory) take the
// cooperative multi-CTA path.
bool expand_uses_grid(const KParams &kp, const Level &lv, int max_w, int max_h);
// ints of one region slot of that path at cell size s; bytes of one region's sync record
long long grid_slot_ints_host(int max_w, int max_h, int s);
size_t grid_sync_bytes();
// One (level, group) launch of the multi-CTA path; items in chunks of at most
// min(co-resident CTAs, sync_cap, slots that fit in slot_cap_ints) regions.
cudaError_t launch_expand_grid(const DevPlanes &P, const KParams &kp, const Level &lv, int level, int iter,
                               const PairDesc *pairs, int max_w, int max_h, const int4 *items, int n_items,
                               float4 *lab, float *phiA, const float4 *prop, Counters *ctr, int *slots,
                               long long slot_cap_ints, void *sync, int sync_cap, cudaStream_t st);
// lem_mincut_batch on the multi-CTA path (any region size); slots of
// grid_slot_ints(max_w, max_h) ints per region
long long grid_slot_ints_wh(int w, int h);
cudaError_t launch_mincut_grid(const KParams &kp, const int4 *regions, const int64_t *offsets, int n_regions,
                               int max_w, int max_h, const int32_t *tcaps, const int32_t *ncaps, uint8_t *take,
                               int64_t *flow, int32_t *status, Counters *ctr, int *slots, long long slot_cap_ints,
                               void *sync, int sync_cap, cudaStream_t st);
// candidates of one visit of each listed cell (see lem_propose_batch)
cudaError_t launch_propose_batch(const DevPlanes &P, const KParams &kp, const Level &lv, int level, int iter,
                                 const int2 *cells, int n_cells, const float4 *lab, const float4 *prop, float *alpha,
                                 long long *dq_scratch, cudaStream_t st);
// RANSAC cells of more pixels than this keep their quantised disparities in a
// global scratch of s * s entries per cell
constexpr int kRansacSmemCell = 25 * 25;
cudaError_t launch_energy(const DevPlanes &P, const KParams &kp, const float4 *lab, long long *partials,
                          long long *out, cudaStream_t st);
cudaError_t launch_labels_out(int H, int W, const float4 *lab, float *abc, float *disp, float *cost,
                              cudaStream_t st);
cudaError_t launch_labels_in(int H, int W, const float *abc, const float *cost, float4 *lab, cudaStream_t st);
cudaError_t launch_planes_out(int H, int W, const DevPlanes &P, float *left, float *right, float *guide,
                              float *weights, cudaStream_t st);
int energy_partials(int H, int W);
// Learned-proposer glue.  Quarter-resolution grid: H4 = ceil(H/4), W4 = ceil(W/4).
// x: H4*W4*7 (left RGB, right RGB as 4x4 block means / 255; mean label disparity / dmax)
cudaError_t launch_cnn_features(const DevPlanes &P, const float4 *lab, float dmax, float *x, cudaStream_t st);
// t: H4*W4*3 (4x4 block means of the label's disparity / dmax, a, b)
cudaError_t launch_cnn_targets(const float4 *lab, int H, int W, float dmax, float *t, cudaStream_t st);
// prop: H*W plane labels from the bilinearly upsampled quarter-resolution (d/dmax, a, b) in y (H4*W4*3)
cudaError_t launch_cnn_upsample(const float *y, int H, int W, float dmax, float4 *prop, cudaStream_t st);
// prop (float4 a, b, c, 0) from / to a caller's H*W*3 array
cudaError_t launch_props_in(int n, const float *abc, float4 *prop, cudaStream_t st);
cudaError_t launch_props_out(int n, const float4 *prop, float *abc, cudaStream_t st);
// Post-processing of one left view (planes PL, labels labL) with the labels labRm of
// the right view estimated on the mirrored pair: consistency mask into valid, the
// filled disparities into filled, the final disparities into disp (all H*W).
cudaError_t launch_postprocess(const DevPlanes &PL, const float4 *labL, const float4 *labRm, float thr, int radius,
                               float gamma, uint8_t *valid, float *filled, float *disp, cudaStream_t st);
// dst (H*W*3 uint8, row stride 3W) = src mirrored horizontally (src row stride in bytes)
cudaError_t launch_mirror_rgb(const uint8_t *src, int64_t stride, int H, int W, uint8_t *dst, cudaStream_t st);
// packed 8-bit RGB (rows of 3 W bytes) from an image of element type dtype
// (LEM_IMG_*), srow / spx bytes between rows / pixels
cudaError_t launch_to_rgb8(const void *src, int64_t srow, int64_t spx, int dtype, int H, int W, uint8_t *dst,
                           cudaStream_t st);
// Batch min-cut whose region/offset/counter scratch is a static device array
// (no allocation); at most LEM_NOALLOC_MAX_REGIONS regions.
cudaError_t launch_mincut_noalloc(const KParams &kp, const lem_region *regions, int n_regions, int max_nodes,
                                  size_t smem, const int32_t *tcaps, const int32_t *ncaps, uint8_t *take,
                                  int64_t *flow, int32_t *status, cudaStream_t st);

// Forward pass of the proposal network on stream st (lem_cnn.cu); LEM_* status.
int cnn_forward_on(lem_cnn *net, const float *x, int H4, int W4, float *y, cudaStream_t st);
const char *cnn_error(const lem_cnn *net);

}  // namespace lem
