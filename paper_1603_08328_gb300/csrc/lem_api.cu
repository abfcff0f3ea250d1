// C ABI of the local-expansion-move library: handle management, argument
// checking and the host-side schedule of Algorithm 1.  All device work is in
// lem_kernels.cu.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "lem.h"
#include "lem_internal.h"

struct lem_handle {
    int B = 1;                          // pairs in the batch
    std::vector<lem::PairDesc> pairs;   // host copy
    lem::PairDesc *d_pairs = nullptr;
    int H = 0, W = 0;                   // pair 0 (the batch entry points work on pair 0)
    int maxH = 0, maxW = 0;
    long long total = 0;                // pixels over all pairs
    lem_params p{};
    cudaStream_t st = nullptr;
    void *L = nullptr, *R = nullptr;  // packed images, lem::px_bytes(p.store_dtype) per pixel
    float4 *gst = nullptr, *wfw = nullptr, *lab = nullptr;
    float *phiA = nullptr;
    float *phiB = nullptr;              // second data-term plane of the two-CTA visits
    // batched visits split into data-term and cut launches (lem::visit_split):
    // candidates_per_visit data-term planes and the candidate labels of a launch
    float *phiK = nullptr;
    float4 *alphaK = nullptr;
    int *d_queue = nullptr;             // work-queue counters of the 48 (level, group) launches
    unsigned *d_done = nullptr;         // dataflow launches: one done flag per cell of a level (all pairs)
    int done_cnt[3] = {0, 0, 0};        // cells of each level over all pairs
    bool split_level[3] = {false, false, false};
    float4 *prop = nullptr;             // proposal maps (allocated when some k_cnn > 0)
    bool prop_set = false;
    float *cnn_buf = nullptr;           // network input / output of one pair (lem_cnn_propose)
    long long *e_part = nullptr, *e_out = nullptr;
    lem::Counters *ctr = nullptr;
    int *n_fp64 = nullptr;
    int4 *d_regions = nullptr;
    int *d_img = nullptr;               // pair of each staged region
    int64_t *d_offsets = nullptr;
    size_t cap_regions = 0;
    // work items (pair, cell i, cell j) of every (level, group), concatenated
    int4 *d_items = nullptr;
    // levels whose regions take the cooperative multi-CTA path, and its buffers
    bool grid_level[3] = {false, false, false};
    int *grid_slots = nullptr;
    long long grid_slot_cap = 0;  // ints
    void *grid_sync = nullptr;
    int grid_sync_cap = 0;        // regions
    int item_off[3][16] = {};
    int item_cnt[3][16] = {};
    // one outer iteration as a CUDA graph; the iteration index lives on the device
    int *d_iter = nullptr;
    cudaStream_t cap_st = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    int iter = 0;
    int fp64_inverses = 0;
    // kernel timing (lem_set_kernel_timing): an event before the first launch of an
    // outer iteration and after each launch, with the kind of that launch
    bool ktime = false;
    std::vector<cudaEvent_t> kev;
    std::vector<int> kkind;
    int kn = 0;        // events recorded so far in the iteration being issued
    int kn_last = 0;   // events of the last iteration issued (direct or captured)
    int kn_graph = 0;  // events of the captured iteration
    bool capturing = false;
    cudaEvent_t it_ev[2] = {nullptr, nullptr};  // around the iterations of a lem_expand_iteration call
    lem::Counters last{};  // device counters at the previous stats read
    std::string err;
};

namespace {

thread_local std::string g_create_err;

int fail(lem_handle *h, int code, const std::string &msg) {
    if (h)
        h->err = msg;
    else
        g_create_err = msg;
    return code;
}

int cuda_fail(lem_handle *h, cudaError_t e, const char *what) {
    std::string m = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    return fail(h, e == cudaErrorMemoryAllocation ? LEM_ERR_OOM : LEM_ERR_CUDA, m);
}

#define LEM_CUDA(h, call)                                      \
    do {                                                       \
        cudaError_t e_ = (call);                               \
        if (e_ != cudaSuccess) return cuda_fail((h), e_, #call); \
    } while (0)

// planes of pair b (pointers offset to its pixels)
lem::DevPlanes planes(const lem_handle *h, int b = 0) {
    const lem::PairDesc &pd = h->pairs[b];
    lem::DevPlanes P;
    P.H = pd.H;
    P.W = pd.W;
    const size_t pb = lem::px_bytes(h->p.store_dtype);
    P.L = (const char *)h->L + pd.off * pb;
    P.R = (const char *)h->R + pd.off * pb;
    P.fmt = h->p.store_dtype;
    P.gst = h->gst + 3 * pd.off;
    P.wfw = h->wfw + pd.off;
    return P;
}

// base planes of the whole batch (the expansion kernel offsets per pair)
lem::DevPlanes planes_base(const lem_handle *h) {
    lem::DevPlanes P;
    P.H = h->maxH;
    P.W = h->maxW;
    P.L = h->L;
    P.R = h->R;
    P.fmt = h->p.store_dtype;
    P.gst = h->gst;
    P.wfw = h->wfw;
    return P;
}

lem::KParams kparams(const lem_handle *h) {
    const lem_params &p = h->p;
    lem::KParams k;
    k.r = p.gf_radius;
    k.tau_col = (float)p.tau_col;
    k.tau_grad = (float)p.tau_grad;
    k.alpha_grad = (float)p.alpha_grad;
    k.tau_dis = (float)p.tau_dis;
    k.S = (float)p.quant_scale;
    k.disp_min = p.disp_min;
    k.disp_max = p.disp_max;
    k.seed = p.seed;
    k.max_rounds = p.max_rounds;
    k.gr_interval = p.gr_interval;
    k.T = p.strip_rows;
    k.visit = p.candidates_per_visit;
    k.bf = p.data_term == LEM_DATA_BF ? 1 : 0;
    k.bf_log2e_inv_gamma = (float)(1.4426950408889634 / p.bf_gamma);
    // fixed-point scales of the warp data term: the largest powers of two for which
    // no window sum of (2r'+1)^2 raw-cost channel terms (|term| <= rho_max, the
    // largest raw cost, since |I/255 - c| <= 1) exceeds 2^31, and no window sum of
    // guided-filter coefficients exceeds 2^62; |a_k| <= sqrt(3) rho_max / e and
    // |b_k| <= rho_max (1 + 3 / e) bound the coefficients ((Sigma_k + eU)^-1 has
    // norm <= 1/e, guide values and their covariance with rho lie in [-1, 1] and
    // [-rho_max, rho_max]); margins of 1 % and 2x cover rounding
    {
        const double n = (2.0 * p.gf_radius + 1) * (2.0 * p.gf_radius + 1);
        const double rho_max = std::max(1e-30, std::fabs(1.0 - p.alpha_grad) * std::fabs(p.tau_col) +
                                                   std::fabs(p.alpha_grad) * std::fabs(p.tau_grad));
        const double coef_max = 2.0 * rho_max * (1.0 + 3.0 / p.gf_eps);
        auto pow2_floor = [](double x) {
            int e = 0;
            std::frexp(x, &e);
            return std::ldexp(1.0, e - 1);
        };
        k.q1 = (float)std::min(std::ldexp(1.0, 30), pow2_floor(2147483647.0 / (1.01 * n * rho_max)));
        k.q2 = (float)std::min(std::ldexp(1.0, 32), pow2_floor(std::ldexp(1.0, 62) / (n * coef_max)));
    }
    return k;
}

// the Level record of `level` with its launch overrides
lem::Level level_of(const lem_handle *h, int level) {
    lem::Level lv;
    lv.s = h->p.cell[level];
    lv.k_prop = h->p.k_prop[level];
    lv.k_rand = h->p.k_rand[level];
    lv.k_cnn = h->p.k_cnn[level];
    lv.k_rans = h->p.k_rans[level];
    lv.threads = h->p.level_threads[level];
    return lv;
}

lem::KParams kparams_level(const lem_handle *h, int level) {
    lem::KParams kp = kparams(h);
    // the multi-CTA path pays a region barrier per BFS level, so it relabels
    // less often by default (64 rounds: the fastest of 16..128 on the
    // 1500 x 1000 V3 levels; the interval never changes a result)
    if (h->grid_level[level]) kp.gr_interval = std::max(kp.gr_interval, 64);
    if (h->p.level_gr_interval[level] > 0) kp.gr_interval = h->p.level_gr_interval[level];
    if (h->p.level_strip_rows[level] > 0) kp.T = h->p.level_strip_rows[level];
    return kp;
}

bool level_uses_grid(const lem_handle *h, int level) {
    return lem::expand_uses_grid(kparams_level(h, level), level_of(h, level), h->maxW, h->maxH);
}

int check_params(const lem_params *p) {
    if (!p) return fail(nullptr, LEM_ERR_ARG, "params is NULL");
    if (p->gf_radius < 0 || p->gf_radius > 32) return fail(nullptr, LEM_ERR_ARG, "gf_radius out of range [0, 32]");
    if (!(p->gf_eps > 0)) return fail(nullptr, LEM_ERR_ARG, "gf_eps must be > 0");
    if (p->n_levels < 1 || p->n_levels > 3) return fail(nullptr, LEM_ERR_ARG, "n_levels must be 1..3");
    for (int l = 0; l < p->n_levels; ++l) {
        if (p->cell[l] < 1) return fail(nullptr, LEM_ERR_ARG, "cell size must be >= 1");
        if (p->cell[l] > LEM_MAX_CELL)
            return fail(nullptr, LEM_ERR_ARG, "cell size above LEM_MAX_CELL");
        if (p->k_prop[l] < 0 || p->k_rand[l] < 0 || p->k_cnn[l] < 0 || p->k_cnn[l] > 64 || p->k_rans[l] < 0 ||
            p->k_rans[l] > 64 || p->k_prop[l] + p->k_rand[l] < 1)
            return fail(nullptr, LEM_ERR_ARG,
                        "each level needs a propagation or perturbation proposal; k_cnn must be 0..64");
    }
    if (!(p->disp_max >= p->disp_min)) return fail(nullptr, LEM_ERR_ARG, "disp_max < disp_min");
    if (!(p->quant_scale > 0) || p->quant_scale > 1048576.0)
        return fail(nullptr, LEM_ERR_ARG, "quant_scale must be in (0, 2^20]");
    if (p->store_dtype != LEM_STORE_F32 && p->store_dtype != LEM_STORE_F16 && p->store_dtype != LEM_STORE_BF16)
        return fail(nullptr, LEM_ERR_ARG, "store_dtype must be LEM_STORE_F32, LEM_STORE_F16 or LEM_STORE_BF16");
    if (p->max_rounds < 1 || p->gr_interval < 1) return fail(nullptr, LEM_ERR_ARG, "max_rounds/gr_interval must be >= 1");
    if (p->strip_rows < 4 || p->strip_rows > 64 || p->strip_rows % 4)
        return fail(nullptr, LEM_ERR_ARG, "strip_rows must be a multiple of 4 in [4, 64]");
    if (p->data_term != LEM_DATA_GF && p->data_term != LEM_DATA_BF)
        return fail(nullptr, LEM_ERR_ARG, "data_term must be LEM_DATA_GF or LEM_DATA_BF");
    if (!(p->bf_gamma > 0)) return fail(nullptr, LEM_ERR_ARG, "bf_gamma must be > 0");
    if (p->cluster_visits != 0 && p->cluster_visits != 1) return fail(nullptr, LEM_ERR_ARG, "cluster_visits must be 0 or 1");
    if (p->split_visits != 0 && p->split_visits != 1) return fail(nullptr, LEM_ERR_ARG, "split_visits must be 0 or 1");
    if (p->work_queue != 0 && p->work_queue != 1) return fail(nullptr, LEM_ERR_ARG, "work_queue must be 0 or 1");
    if (p->dataflow != 0 && p->dataflow != 1) return fail(nullptr, LEM_ERR_ARG, "dataflow must be 0 or 1");
    if (p->candidates_per_visit < 1 || p->candidates_per_visit > 8)
        return fail(nullptr, LEM_ERR_ARG, "candidates_per_visit must be 1..8");
    if (p->threads < 32 || p->threads > 1024 || p->threads % 32)
        return fail(nullptr, LEM_ERR_ARG, "threads must be a multiple of 32 in [32, 1024]");
    for (int l = 0; l < 3; ++l) {
        const int t = p->level_threads[l];
        if (t != 0 && t != 32 && t != 64 && t != 128 && t != 256 && t != 512 && t != 1024)
            return fail(nullptr, LEM_ERR_ARG, "level_threads must be 0, 32, 64, 128, 256, 512 or 1024");
        if (p->level_gr_interval[l] < 0) return fail(nullptr, LEM_ERR_ARG, "level_gr_interval must be >= 0");
        if (p->level_strip_rows[l] < 0 || p->level_strip_rows[l] > 64 || p->level_strip_rows[l] % 4)
            return fail(nullptr, LEM_ERR_ARG, "level_strip_rows must be 0 or a multiple of 4 up to 64");
    }
    return LEM_OK;
}

// element size of a lem_image dtype (0: unknown)
size_t img_elem(int dtype) {
    return dtype == LEM_IMG_U8 ? 1 : (dtype == LEM_IMG_F16 || dtype == LEM_IMG_BF16) ? 2 : dtype == LEM_IMG_F32 ? 4 : 0;
}
int img_channels(const lem_image *im) { return im->channels ? im->channels : 3; }
int64_t img_stride_px(const lem_image *im) {
    return im->stride_px ? im->stride_px : (int64_t)img_channels(im) * (int64_t)img_elem(im->dtype);
}

int check_image(const lem_image *im, const char *name) {
    const std::string nm(name);
    if (!im || !im->data) return fail(nullptr, LEM_ERR_ARG, nm + " image is NULL");
    if (im->height < 1 || im->width < 2) return fail(nullptr, LEM_ERR_SHAPE, nm + " image too small");
    const int64_t es = (int64_t)img_elem(im->dtype);
    if (!es) return fail(nullptr, LEM_ERR_ARG, nm + " image dtype is not one of LEM_IMG_*");
    const int ch = img_channels(im);
    if (ch < 3 || ch > 16) return fail(nullptr, LEM_ERR_ARG, nm + " image channels must be 3..16");
    const int64_t spx = img_stride_px(im);
    if (spx < ch * es) return fail(nullptr, LEM_ERR_SHAPE, nm + " image stride_px < channels * element size");
    if (spx % es || im->stride_row % es || (uintptr_t)im->data % (uintptr_t)es)
        return fail(nullptr, LEM_ERR_ARG, nm + " image pointer or strides not a multiple of the element size");
    if (im->stride_row < (int64_t)(im->width - 1) * spx + ch * es)
        return fail(nullptr, LEM_ERR_SHAPE, nm + " image stride_row shorter than a row");
    if ((int64_t)im->height * im->width > (1LL << 30)) return fail(nullptr, LEM_ERR_SHAPE, "image too large");
    return LEM_OK;
}

// Device packed 8-bit RGB (rows of `*stride` bytes) of a checked image: the
// caller's own data when it already is that on the device, else a copy in
// *tmp (device memory the caller frees once the kernels reading it are done).
cudaError_t stage_rgb8(const lem_image *im, cudaStream_t st, uint8_t **tmp, const uint8_t **out, int64_t *stride) {
    const int H = im->height, W = im->width;
    const int64_t es = (int64_t)img_elem(im->dtype), spx = img_stride_px(im);
    *tmp = nullptr;
    const bool packed = im->dtype == LEM_IMG_U8 && spx == 3;
    if (packed && im->on_device) {
        *out = (const uint8_t *)im->data;
        *stride = im->stride_row;
        return cudaSuccess;
    }
    const size_t rgb = (size_t)H * W * 3;
    // host images that need converting are first copied as they are (rows cut
    // to their used bytes), then converted on the device
    const int64_t row_used = (int64_t)(W - 1) * spx + img_channels(im) * es;
    const int64_t pitch = (row_used + 15) & ~(int64_t)15;
    const size_t raw = (!packed && !im->on_device) ? (size_t)pitch * H : 0;
    cudaError_t e = cudaMalloc(tmp, rgb + raw);
    if (e != cudaSuccess) return e;
    if (packed) {
        e = cudaMemcpy2DAsync(*tmp, 3 * W, im->data, im->stride_row, 3 * W, H, cudaMemcpyHostToDevice, st);
    } else {
        const void *src = im->data;
        int64_t srow = im->stride_row;
        if (!im->on_device) {
            e = cudaMemcpy2DAsync(*tmp + rgb, pitch, im->data, im->stride_row, row_used, H, cudaMemcpyHostToDevice,
                                  st);
            src = *tmp + rgb;
            srow = pitch;
        }
        if (e == cudaSuccess) e = lem::launch_to_rgb8(src, srow, spx, im->dtype, H, W, *tmp, st);
    }
    if (e != cudaSuccess) {
        cudaStreamSynchronize(st);
        cudaFree(*tmp);
        *tmp = nullptr;
        return e;
    }
    *out = *tmp;
    *stride = 3 * W;
    return cudaSuccess;
}

void free_handle(lem_handle *h) {
    if (!h) return;
    cudaFree(h->L);
    cudaFree(h->R);
    cudaFree(h->gst);
    cudaFree(h->wfw);
    cudaFree(h->lab);
    cudaFree(h->phiA);
    cudaFree(h->phiB);
    cudaFree(h->phiK);
    cudaFree(h->alphaK);
    cudaFree(h->d_queue);
    cudaFree(h->d_done);
    cudaFree(h->prop);
    cudaFree(h->cnn_buf);
    cudaFree(h->e_part);
    cudaFree(h->e_out);
    cudaFree(h->ctr);
    cudaFree(h->n_fp64);
    cudaFree(h->d_regions);
    cudaFree(h->d_img);
    cudaFree(h->d_offsets);
    cudaFree(h->d_pairs);
    cudaFree(h->d_items);
    cudaFree(h->grid_slots);
    cudaFree(h->grid_sync);
    cudaFree(h->d_iter);
    if (h->gexec) cudaGraphExecDestroy(h->gexec);
    if (h->graph) cudaGraphDestroy(h->graph);
    if (h->cap_st) cudaStreamDestroy(h->cap_st);
    for (cudaEvent_t e : h->kev) cudaEventDestroy(e);
    for (cudaEvent_t e : h->it_ev)
        if (e) cudaEventDestroy(e);
    delete h;
}

// Uploads regions (host) and their packed offsets (K values per pixel).
int stage_regions(lem_handle *h, const lem_region *regions, int n, int K, int64_t *total, int *max_w, int *max_h,
                  int *max_n, size_t *max_cut_smem = nullptr) {
    if (!regions || n < 1) return fail(h, LEM_ERR_ARG, "regions is NULL or n_regions < 1");
    std::vector<int4> rg(n);
    std::vector<int> im(n);
    std::vector<int64_t> off(n);
    int64_t acc = 0;
    int mw = 0, mh = 0, mn = 0;
    for (int i = 0; i < n; ++i) {
        const lem_region &r = regions[i];
        if (r.img < 0 || r.img >= h->B)
            return fail(h, LEM_ERR_ARG, "region " + std::to_string(i) + ": img out of range");
        const lem::PairDesc &pd = h->pairs[r.img];
        if (r.w < 1 || r.h < 1 || r.x0 < 0 || r.y0 < 0 || r.x0 + r.w > pd.W || r.y0 + r.h > pd.H)
            return fail(h, LEM_ERR_SHAPE, "region " + std::to_string(i) + " is empty or outside its image");
        if ((r.cw != 0 || r.ch != 0) && (r.cw < 1 || r.ch < 1 || r.cx0 < r.x0 || r.cy0 < r.y0 ||
                                         r.cx0 + r.cw > r.x0 + r.w || r.cy0 + r.ch > r.y0 + r.h))
            return fail(h, LEM_ERR_SHAPE, "region " + std::to_string(i) + ": centre cell outside the region");
        rg[i] = make_int4(r.x0, r.y0, r.w, r.h);
        im[i] = r.img;
        off[i] = acc;
        acc += (int64_t)K * r.w * r.h;
        mw = std::max(mw, r.w);
        mh = std::max(mh, r.h);
        mn = std::max(mn, r.w * r.h);
        if (max_cut_smem) *max_cut_smem = std::max(*max_cut_smem, lem::cut_smem_bytes(r.w, r.h));
    }
    if ((size_t)n > h->cap_regions) {
        cudaFree(h->d_regions);
        cudaFree(h->d_img);
        cudaFree(h->d_offsets);
        h->d_regions = nullptr;
        h->d_img = nullptr;
        h->d_offsets = nullptr;
        h->cap_regions = 0;
        LEM_CUDA(h, cudaMalloc(&h->d_regions, sizeof(int4) * n));
        LEM_CUDA(h, cudaMalloc(&h->d_img, sizeof(int) * n));
        LEM_CUDA(h, cudaMalloc(&h->d_offsets, sizeof(int64_t) * n));
        h->cap_regions = n;
    }
    LEM_CUDA(h, cudaMemcpyAsync(h->d_regions, rg.data(), sizeof(int4) * n, cudaMemcpyHostToDevice, h->st));
    LEM_CUDA(h, cudaMemcpyAsync(h->d_img, im.data(), sizeof(int) * n, cudaMemcpyHostToDevice, h->st));
    LEM_CUDA(h, cudaMemcpyAsync(h->d_offsets, off.data(), sizeof(int64_t) * n, cudaMemcpyHostToDevice, h->st));
    // the staging vectors die on return: make sure the copies have read them
    LEM_CUDA(h, cudaStreamSynchronize(h->st));
    *total = acc;
    *max_w = mw;
    *max_h = mh;
    *max_n = mn;
    return LEM_OK;
}

// quantised energy of pair b, or of all pairs (b < 0)
int run_energy(lem_handle *h, long long *eq, int b = -1) {
    lem::KParams kp = kparams(h);
    long long tot = 0;
    for (int i = 0; i < h->B; ++i) {
        if (b >= 0 && i != b) continue;
        long long e = 0;
        LEM_CUDA(h, lem::launch_energy(planes(h, i), kp, h->lab + h->pairs[i].off, h->e_part, h->e_out, h->st));
        LEM_CUDA(h, cudaMemcpyAsync(&e, h->e_out, sizeof(long long), cudaMemcpyDeviceToHost, h->st));
        LEM_CUDA(h, cudaStreamSynchronize(h->st));
        tot += e;
    }
    *eq = tot;
    return LEM_OK;
}

// Reads the cumulative device counters; fills the deltas since the previous read.
int read_counters(lem_handle *h, lem_stats *stats) {
    lem::Counters c;
    LEM_CUDA(h, cudaMemcpyAsync(&c, h->ctr, sizeof(c), cudaMemcpyDeviceToHost, h->st));
    LEM_CUDA(h, cudaStreamSynchronize(h->st));
    stats->evals = (int64_t)(c.evals - h->last.evals);
    stats->accepted = (int64_t)(c.accepted - h->last.accepted);
    stats->maxflow_limit = (int64_t)(c.limit_hits - h->last.limit_hits);
    stats->pr_rounds = (int64_t)(c.rounds - h->last.rounds);
    stats->pr_global_relabels = (int64_t)(c.relabels - h->last.relabels);
    stats->pr_bfs_levels = (int64_t)(c.bfs_levels - h->last.bfs_levels);
    for (int k = 0; k < 4; ++k) stats->accepted_by_kind[k] = (int64_t)(c.accepted_kind[k] - h->last.accepted_kind[k]);
    stats->dep_waits_given_up = (int64_t)(c.dep_give_ups - h->last.dep_give_ups);
    stats->fp64_inverses = h->fp64_inverses;
    stats->iterations = h->iter;
    h->last = c;
    return LEM_OK;
}

}  // namespace

extern "C" {

void lem_default_params(lem_params *p) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->gf_radius = 10;
    p->gf_eps = 1e-4;
    p->tau_col = 10.0;
    p->tau_grad = 2.0;
    p->alpha_grad = 0.9;
    p->lambda = 1.0;
    p->tau_dis = 1.0;
    p->eps_w = 0.01;
    p->gamma = 10.0;
    p->disp_min = 0.0;
    p->disp_max = 60.0;
    p->n_levels = 3;
    p->cell[0] = 5;
    p->cell[1] = 15;
    p->cell[2] = 25;
    p->k_prop[0] = 1;
    p->k_prop[1] = 2;
    p->k_prop[2] = 2;
    p->k_rand[0] = 7;
    p->k_rand[1] = 0;
    p->k_rand[2] = 0;
    p->quant_scale = 65536.0;
    p->store_dtype = LEM_STORE_F32;
    p->cond_fp64 = 1e3;
    p->seed = 1;
    p->stream = nullptr;
    p->max_rounds = 200000;
    p->gr_interval = 32;
    p->strip_rows = 16;
    p->threads = 256;
    p->use_graph = 1;
    p->candidates_per_visit = 1;
    p->k_cnn[0] = p->k_cnn[1] = p->k_cnn[2] = 0;
    p->k_rans[0] = p->k_rans[1] = p->k_rans[2] = 0;
    p->data_term = LEM_DATA_GF;
    p->bf_gamma = 10.0;
    p->cluster_visits = 1;
}

const char *lem_last_error(const lem_handle *h) { return h ? h->err.c_str() : g_create_err.c_str(); }

int lem_create_batch(const lem_image *lefts, const lem_image *rights, int n_pairs, const lem_params *p,
                     lem_handle **out) {
    return lem_create_batch_ranges(lefts, rights, n_pairs, nullptr, p, out);
}

int lem_create_batch_ranges(const lem_image *lefts, const lem_image *rights, int n_pairs,
                            const double *disp_ranges, const lem_params *p, lem_handle **out) {
    if (!out) return fail(nullptr, LEM_ERR_ARG, "out is NULL");
    *out = nullptr;
    int rc;
    if ((rc = check_params(p)) != LEM_OK) return rc;
    if (!lefts || !rights || n_pairs < 1 || n_pairs > 4096)
        return fail(nullptr, LEM_ERR_ARG, "lefts/rights NULL or n_pairs outside [1, 4096]");
    if (disp_ranges)
        for (int b = 0; b < n_pairs; ++b)
            if (!(disp_ranges[2 * b + 1] >= disp_ranges[2 * b]) || !std::isfinite(disp_ranges[2 * b]) ||
                !std::isfinite(disp_ranges[2 * b + 1]))
                return fail(nullptr, LEM_ERR_ARG, "disparity range of pair " + std::to_string(b) + " is not finite with max >= min");
    for (int b = 0; b < n_pairs; ++b) {
        if ((rc = check_image(&lefts[b], "left")) != LEM_OK) return rc;
        if ((rc = check_image(&rights[b], "right")) != LEM_OK) return rc;
        if (lefts[b].height != rights[b].height || lefts[b].width != rights[b].width)
            return fail(nullptr, LEM_ERR_SHAPE, "left and right images differ in size (pair " + std::to_string(b) + ")");
        if (lefts[b].width < 2 * p->gf_radius + 1 || lefts[b].height < 2 * p->gf_radius + 1)
            return fail(nullptr, LEM_ERR_SHAPE, "image smaller than one regression window");
    }
    lem_handle *h = new lem_handle();
    h->B = n_pairs;
    h->p = *p;
    h->st = (cudaStream_t)p->stream;
    long long off = 0;
    for (int b = 0; b < n_pairs; ++b) {
        lem::PairDesc pd;
        pd.H = lefts[b].height;
        pd.W = lefts[b].width;
        pd.off = off;
        // pair 0 keeps the seed, so a batch of one reproduces lem_create
        pd.seed = p->seed + 0x9E3779B97F4A7C15ull * (unsigned long long)b;
        pd.disp_min = disp_ranges ? disp_ranges[2 * b] : p->disp_min;
        pd.disp_max = disp_ranges ? disp_ranges[2 * b + 1] : p->disp_max;
        off += (long long)pd.H * pd.W;
        h->pairs.push_back(pd);
        h->maxH = std::max(h->maxH, pd.H);
        h->maxW = std::max(h->maxW, pd.W);
    }
    h->total = off;
    h->H = h->pairs[0].H;
    h->W = h->pairs[0].W;
    const size_t n = (size_t)h->total;
    auto bail = [&](int code) {
        g_create_err = h->err;
        free_handle(h);
        return code;
    };
#define CREATE_CUDA(call)                                            \
    do {                                                             \
        cudaError_t e_ = (call);                                     \
        if (e_ != cudaSuccess) return bail(cuda_fail(h, e_, #call)); \
    } while (0)
    CREATE_CUDA(cudaMalloc(&h->L, lem::px_bytes(p->store_dtype) * n));
    CREATE_CUDA(cudaMalloc(&h->R, lem::px_bytes(p->store_dtype) * n));
    CREATE_CUDA(cudaMalloc(&h->gst, sizeof(float4) * 3 * n));
    CREATE_CUDA(cudaMalloc(&h->wfw, sizeof(float4) * n));
    CREATE_CUDA(cudaMalloc(&h->lab, sizeof(float4) * n));
    CREATE_CUDA(cudaMalloc(&h->phiA, sizeof(float) * n));
    CREATE_CUDA(cudaMalloc(&h->phiB, sizeof(float) * n));
    for (int l = 0; l < p->n_levels; ++l)
        if (p->k_cnn[l] > 0 && !h->prop) CREATE_CUDA(cudaMalloc(&h->prop, sizeof(float4) * n));
    CREATE_CUDA(cudaMalloc(&h->e_part, sizeof(long long) * lem::energy_partials(h->maxH, h->maxW)));
    CREATE_CUDA(cudaMalloc(&h->e_out, sizeof(long long)));
    CREATE_CUDA(cudaMalloc(&h->ctr, sizeof(lem::Counters)));
    CREATE_CUDA(cudaMalloc(&h->n_fp64, sizeof(int)));
    CREATE_CUDA(cudaMalloc(&h->d_pairs, sizeof(lem::PairDesc) * n_pairs));
    CREATE_CUDA(cudaMalloc(&h->d_iter, sizeof(int)));
    CREATE_CUDA(cudaMalloc(&h->d_queue, sizeof(int) * 2 * 48));
    CREATE_CUDA(cudaMemsetAsync(h->d_queue, 0, sizeof(int) * 2 * 48, h->st));
    CREATE_CUDA(cudaMemsetAsync(h->n_fp64, 0, sizeof(int), h->st));
    CREATE_CUDA(cudaMemsetAsync(h->ctr, 0, sizeof(lem::Counters), h->st));
    CREATE_CUDA(cudaMemcpyAsync(h->d_pairs, h->pairs.data(), sizeof(lem::PairDesc) * n_pairs, cudaMemcpyHostToDevice,
                                h->st));
    // work items of every (level, group): (pair, cell i, cell j, index of the
    // pair's cell (0, 0) among the level's done flags)
    {
        std::vector<int4> items;
        int max_cells = 1;
        for (int l = 0; l < p->n_levels; ++l) {
            const int s = p->cell[l];
            std::vector<int> base(n_pairs);
            int cells = 0;
            for (int b = 0; b < n_pairs; ++b) {
                base[b] = cells;
                cells += ((h->pairs[b].W + s - 1) / s) * ((h->pairs[b].H + s - 1) / s);
            }
            h->done_cnt[l] = cells;
            max_cells = std::max(max_cells, cells);
            for (int g = 0; g < 16; ++g) {
                h->item_off[l][g] = (int)items.size();
                const int gi = g & 3, gj = g >> 2;
                for (int b = 0; b < n_pairs; ++b) {
                    const int nx = (h->pairs[b].W + s - 1) / s, ny = (h->pairs[b].H + s - 1) / s;
                    for (int cj = gj; cj < ny; cj += 4)
                        for (int ci = gi; ci < nx; ci += 4) items.push_back(make_int4(b, ci, cj, base[b]));
                }
                h->item_cnt[l][g] = (int)items.size() - h->item_off[l][g];
                // largest regions first (the clipped border regions of every pair last), so
                // the block scheduler starts the longest work first; the regions of a group
                // are independent, so the order changes no result
                auto area = [&](const int4 &it) {
                    const lem::PairDesc &pd = h->pairs[it.x];
                    const int w = std::min(pd.W, (it.y + 2) * s) - std::max(0, (it.y - 1) * s);
                    const int hh = std::min(pd.H, (it.z + 2) * s) - std::max(0, (it.z - 1) * s);
                    return (long long)w * hh;
                };
                std::stable_sort(items.begin() + h->item_off[l][g], items.end(),
                                 [&](const int4 &a, const int4 &b) { return area(a) > area(b); });
            }
        }
        if (p->dataflow) CREATE_CUDA(cudaMalloc(&h->d_done, sizeof(unsigned) * max_cells));
        CREATE_CUDA(cudaMalloc(&h->d_items, sizeof(int4) * std::max<size_t>(1, items.size())));
        CREATE_CUDA(cudaMemcpy(h->d_items, items.data(), sizeof(int4) * items.size(), cudaMemcpyHostToDevice));
    }
    // levels above the shared-memory cut: global slots for as many regions as
    // one launch can hold co-resident (one CTA per SM at least)
    {
        int dev = 0, nsm = 0;
        CREATE_CUDA(cudaGetDevice(&dev));
        CREATE_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
        long long need = 0;
        int regions = 0;
        for (int l = 0; l < p->n_levels; ++l) {
            if (!h->grid_level[l] && !level_uses_grid(h, l)) continue;
            h->grid_level[l] = true;
            int most = 0;
            for (int g = 0; g < 16; ++g) most = std::max(most, h->item_cnt[l][g]);
            const int m = std::max(1, std::min(most, nsm));
            need = std::max(need, (long long)m * lem::grid_slot_ints_host(h->maxW, h->maxH, p->cell[l]));
            regions = std::max(regions, m);
        }
        if (need > 0) {
            CREATE_CUDA(cudaMalloc(&h->grid_slots, sizeof(int) * (size_t)need));
            CREATE_CUDA(cudaMalloc(&h->grid_sync, lem::grid_sync_bytes() * regions));
            h->grid_slot_cap = need;
            h->grid_sync_cap = regions;
        }
    }
    // levels whose batched visits run as data-term + cut launches: their planes
    // and candidate labels
    {
        int most = 0;
        for (int l = 0; l < p->n_levels; ++l) {
            h->split_level[l] = p->split_visits && !h->grid_level[l] &&
                                lem::visit_split(kparams_level(h, l), level_of(h, l), h->maxW, h->maxH);
            if (!h->split_level[l]) continue;
            for (int g = 0; g < 16; ++g) most = std::max(most, h->item_cnt[l][g]);
        }
        if (most > 0) {
            const int K = p->candidates_per_visit;
            CREATE_CUDA(cudaMalloc(&h->phiK, sizeof(float) * n * K));
            CREATE_CUDA(cudaMalloc(&h->alphaK, sizeof(float4) * (size_t)most * K));
        }
    }
    // per pair: images on the device, packing, guide statistics, random labels, costs
    for (int b = 0; b < n_pairs; ++b) {
        const lem_image *left = &lefts[b], *right = &rights[b];
        const lem::PairDesc &pd = h->pairs[b];
        const int H = pd.H, W = pd.W;
        const size_t np = (size_t)H * W;
        (void)np;
        // packed 8-bit RGB of both images on the device (uploaded / converted as needed)
        const uint8_t *dl = nullptr, *dr = nullptr;
        int64_t ls = 0, rs = 0;
        uint8_t *tmpl = nullptr, *tmpr = nullptr;
        cudaError_t ce = stage_rgb8(left, h->st, &tmpl, &dl, &ls);
        if (ce == cudaSuccess) ce = stage_rgb8(right, h->st, &tmpr, &dr, &rs);
        if (ce != cudaSuccess) {
            cudaStreamSynchronize(h->st);
            cudaFree(tmpl);
            return bail(cuda_fail(h, ce, "lem_create image upload"));
        }
        lem::DevPlanes P = planes(h, b);
        lem::KParams kp = kparams(h);
        kp.seed = pd.seed;
        cudaError_t e = lem::launch_preprocess(dl, ls, dr, rs, H, W, (float)p->lambda, (float)p->eps_w,
                                               (float)p->gamma, (void *)P.L, (void *)P.R, p->store_dtype,
                                               (float4 *)P.wfw, h->st);
        if (e == cudaSuccess)
            e = lem::launch_guide_stats(dl, ls, H, W, p->gf_radius, p->gf_eps, p->cond_fp64, (float4 *)P.gst,
                                        h->n_fp64, h->st);
        if (e == cudaSuccess)
            e = lem::launch_init_labels(H, W, pd.seed, pd.disp_min, pd.disp_max, h->lab + pd.off, h->st);
        if (e == cudaSuccess) e = lem::launch_pixel_costs(P, kp, h->lab + pd.off, std::min(p->threads, 128), h->st);
        // the temporary upload buffers must outlive the kernels that read them
        if (tmpl || tmpr) {
            if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
            cudaFree(tmpl);
            cudaFree(tmpr);
        }
        if (e != cudaSuccess) return bail(cuda_fail(h, e, "lem_create kernels"));
    }
    int nf = 0;
    CREATE_CUDA(cudaMemcpyAsync(&nf, h->n_fp64, sizeof(int), cudaMemcpyDeviceToHost, h->st));
    CREATE_CUDA(cudaStreamSynchronize(h->st));
#undef CREATE_CUDA
    h->fp64_inverses = nf;
    *out = h;
    return LEM_OK;
}

int lem_create(const lem_image *left, const lem_image *right, const lem_params *p, lem_handle **out) {
    if (!left || !right) {
        if (out) *out = nullptr;
        return fail(nullptr, LEM_ERR_ARG, "left or right image is NULL");
    }
    return lem_create_batch(left, right, 1, p, out);
}

int lem_create_right_view(const lem_image *left, const lem_image *right, const lem_params *p, lem_handle **out) {
    if (!out) return fail(nullptr, LEM_ERR_ARG, "out is NULL");
    *out = nullptr;
    int rc;
    if ((rc = check_params(p)) != LEM_OK) return rc;
    if ((rc = check_image(left, "left")) != LEM_OK) return rc;
    if ((rc = check_image(right, "right")) != LEM_OK) return rc;
    if (left->height != right->height || left->width != right->width)
        return fail(nullptr, LEM_ERR_SHAPE, "left and right images differ in size");
    const int H = left->height, W = left->width;
    const size_t img = (size_t)H * W * 3;
    cudaStream_t st = (cudaStream_t)p->stream;
    uint8_t *buf = nullptr;  // [mirrored right][mirrored left]
    cudaError_t e = cudaMalloc(&buf, 2 * img);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "lem_create_right_view");
    const lem_image *src[2] = {right, left};
    uint8_t *tmp[2] = {nullptr, nullptr};
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
        const uint8_t *d = nullptr;
        int64_t ds = 0;
        e = stage_rgb8(src[k], st, &tmp[k], &d, &ds);
        if (e == cudaSuccess) e = lem::launch_mirror_rgb(d, ds, H, W, buf + k * img, st);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(tmp[0]);
    cudaFree(tmp[1]);
    if (e != cudaSuccess) {
        cudaFree(buf);
        return cuda_fail(nullptr, e, "lem_create_right_view mirror");
    }
    // the mirrored right image is the reference view, the mirrored left the matched one
    lem_image l2{buf, H, W, 3LL * W, 1, 3, 3, LEM_IMG_U8}, r2{buf + img, H, W, 3LL * W, 1, 3, 3, LEM_IMG_U8};
    rc = lem_create_batch(&l2, &r2, 1, p, out);
    cudaFree(buf);
    return rc;
}

int lem_pair_count(const lem_handle *h) { return h ? h->B : -1; }

int lem_pair_info(const lem_handle *h, int pair, int *height, int *width, int64_t *pixel_offset) {
    if (!h || pair < 0 || pair >= h->B) return fail(nullptr, LEM_ERR_ARG, "lem_pair_info: bad handle or pair");
    if (height) *height = h->pairs[pair].H;
    if (width) *width = h->pairs[pair].W;
    if (pixel_offset) *pixel_offset = h->pairs[pair].off;
    return LEM_OK;
}

int lem_destroy(lem_handle *h) {
    if (h && h->st) cudaStreamSynchronize(h->st);
    free_handle(h);
    return LEM_OK;
}

int lem_unary_batch(lem_handle *h, const lem_region *regions, int n_regions, const float *labels, int K,
                    float *costs) {
    if (!h) return fail(nullptr, LEM_ERR_ARG, "handle is NULL");
    if (!labels || !costs || K < 1) return fail(h, LEM_ERR_ARG, "labels/costs NULL or K < 1");
    int64_t total;
    int mw, mh, mn, rc;
    if ((rc = stage_regions(h, regions, n_regions, K, &total, &mw, &mh, &mn)) != LEM_OK) return rc;
    if ((int64_t)n_regions * K > (1LL << 31) - 1) return fail(h, LEM_ERR_ARG, "too many region-label pairs");
    // a handle whose expansions use the warp data term (batched visits) gets the same
    // computation here
    const lem::KParams kp = kparams(h);
    if (h->p.split_visits && h->p.candidates_per_visit >= 2 && lem::unary_warp_fits(kp, h->maxW, mw)) {
        LEM_CUDA(h, lem::launch_unary_batch_warp(planes_base(h), kp, h->d_pairs, h->d_img, h->d_regions, h->d_offsets,
                                                 n_regions, K, mw, labels, costs, h->st));
        return LEM_OK;
    }
    LEM_CUDA(h, lem::launch_unary_batch(planes_base(h), kparams(h), h->d_pairs, h->d_img, h->d_regions, h->d_offsets,
                                        n_regions, K, mw, mh, labels, costs, h->p.threads, h->st));
    return LEM_OK;
}

int lem_pairwise_batch(lem_handle *h, const lem_region *regions, int n_regions, const float *alpha,
                       const float *costs_alpha, int32_t *tcaps, int32_t *ncaps, int64_t *const_term) {
    if (!h) return fail(nullptr, LEM_ERR_ARG, "handle is NULL");
    if (!alpha || !costs_alpha || !tcaps || !ncaps || !const_term) return fail(h, LEM_ERR_ARG, "NULL pointer");
    int64_t total;
    int mw, mh, mn, rc;
    if ((rc = stage_regions(h, regions, n_regions, 1, &total, &mw, &mh, &mn)) != LEM_OK) return rc;
    if (mn > LEM_MAX_REGION_NODES) return fail(h, LEM_ERR_SHAPE, "region larger than LEM_MAX_REGION_NODES");
    LEM_CUDA(h, lem::launch_pairwise_batch(planes_base(h), kparams(h), h->d_pairs, h->d_img, h->d_regions,
                                           h->d_offsets, n_regions, h->lab, alpha, costs_alpha, tcaps, ncaps,
                                           const_term, h->p.threads, h->st));
    return LEM_OK;
}

int lem_mincut_batch(lem_handle *h, const lem_region *regions, int n_regions, const int32_t *tcaps,
                     const int32_t *ncaps, uint8_t *take_alpha, int64_t *flow, int32_t *status) {
    if (!h) return fail(nullptr, LEM_ERR_ARG, "handle is NULL");
    if (!tcaps || !ncaps || !take_alpha || !flow || !status) return fail(h, LEM_ERR_ARG, "NULL pointer");
    int64_t total;
    int mw, mh, mn, rc;
    size_t smem = 0;
    if ((rc = stage_regions(h, regions, n_regions, 1, &total, &mw, &mh, &mn, &smem)) != LEM_OK) return rc;
    if (mn > LEM_MAX_REGION_NODES || smem > 227 * 1024) {
        // regions above the shared-memory cut: the multi-CTA path, with scratch
        // slots for as many regions as one launch holds
        int dev = 0, nsm = 0;
        LEM_CUDA(h, cudaGetDevice(&dev));
        LEM_CUDA(h, cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
        const int m = std::min(n_regions, nsm);
        const long long slot = lem::grid_slot_ints_wh(mw, mh);
        int *slots = nullptr;
        void *sync = nullptr;
        cudaError_t e = cudaMalloc(&slots, sizeof(int) * (size_t)slot * m);
        if (e == cudaSuccess) e = cudaMalloc(&sync, lem::grid_sync_bytes() * m);
        if (e == cudaSuccess)
            e = lem::launch_mincut_grid(kparams(h), h->d_regions, h->d_offsets, n_regions, mw, mh, tcaps, ncaps,
                                        take_alpha, flow, status, h->ctr, slots, slot * m, sync, m, h->st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
        cudaFree(slots);
        cudaFree(sync);
        if (e != cudaSuccess) return cuda_fail(h, e, "lem_mincut_batch (multi-CTA path)");
        return LEM_OK;
    }
    LEM_CUDA(h, lem::launch_mincut_batch(kparams(h), h->d_regions, h->d_offsets, n_regions, mn, smem, tcaps, ncaps,
                                         take_alpha, flow, status, h->ctr, h->st));
    return LEM_OK;
}

// kernel timing: records the next event of the iteration after a launch of `kind`
// (kind < 0: the event before the first launch).  In a stream capture the event
// becomes an event node of the graph.
static int ktime_mark(lem_handle *h, int kind, int level, cudaStream_t st) {
    if (!h->ktime) return LEM_OK;
    if (kind < 0) h->kn = 0;
    if (h->kn >= (int)h->kev.size()) {
        cudaEvent_t e = nullptr;
        LEM_CUDA(h, cudaEventCreate(&e));
        h->kev.push_back(e);
        h->kkind.push_back(-1);
    }
    h->kkind[h->kn] = kind < 0 ? -1 : kind + LEM_KERNEL_KINDS * level;
    LEM_CUDA(h, cudaEventRecordWithFlags(h->kev[h->kn], st, h->capturing ? cudaEventRecordExternal : 0));
    ++h->kn;
    return LEM_OK;
}

// one (level, group) launch over every pair; iter < 0: read from h->d_iter
static int expand_group_impl(lem_handle *h, int iter, int level, int group, cudaStream_t st) {
    const lem::Level lv = level_of(h, level);
    if (h->prop && !h->prop_set)
        return fail(h, LEM_ERR_ARG, "k_cnn > 0 but no proposal map was set (lem_set_proposals / lem_cnn_propose)");
    const lem::KParams kp = kparams_level(h, level);
    int rc;
    if (h->split_level[level]) {
        // batched visits: per visit, the data terms of its candidates, then its moves
        const int nprop = lv.k_prop + (h->prop ? lv.k_cnn : 0) + lv.k_rand;
        const int K = kp.visit;
        const int4 *items = h->d_items + h->item_off[level][group];
        const int n_items = h->item_cnt[level][group];
        for (int t0 = 0; t0 < nprop; t0 += K) {
            const int nK = std::min(K, nprop - t0);
            LEM_CUDA(h, lem::launch_visit_unary(planes_base(h), kp, lv, level, iter, h->d_iter, h->d_pairs, h->maxW,
                                                h->maxH, items, n_items, t0, nK, h->lab, h->phiK, h->total, h->prop,
                                                h->alphaK, st));
            if ((rc = ktime_mark(h, LEM_KERNEL_VISIT_UNARY, level, st)) != LEM_OK) return rc;
            LEM_CUDA(h, lem::launch_visit_cut(planes_base(h), kp, lv, h->d_pairs, h->maxW, h->maxH, items, n_items,
                                              t0, nK, h->prop ? lv.k_cnn : 0, h->lab, h->phiK, h->total, h->alphaK,
                                              h->ctr, st));
            if ((rc = ktime_mark(h, LEM_KERNEL_VISIT_CUT, level, st)) != LEM_OK) return rc;
        }
        return LEM_OK;
    }
    if (h->grid_level[level]) {
        if (iter < 0) return fail(h, LEM_ERR_ARG, "levels above the shared-memory cut are not graph-captured");
        LEM_CUDA(h, lem::launch_expand_grid(planes_base(h), kp, lv, level, iter, h->d_pairs, h->maxW, h->maxH,
                                            h->d_items + h->item_off[level][group], h->item_cnt[level][group],
                                            h->lab, h->phiA, h->prop, h->ctr, h->grid_slots, h->grid_slot_cap,
                                            h->grid_sync, h->grid_sync_cap, st));
        return ktime_mark(h, LEM_KERNEL_GRID, level, st);
    }
    LEM_CUDA(h, lem::launch_expand_group(planes_base(h), kp, lv, level, iter, h->d_iter, h->d_pairs, h->maxW,
                                         h->maxH, h->d_items + h->item_off[level][group], h->item_cnt[level][group],
                                         h->lab, h->phiA, h->prop, h->ctr, h->p.cluster_visits ? h->phiB : nullptr,
                                         h->p.work_queue ? h->d_queue + 2 * (16 * level + group) : nullptr, nullptr,
                                         st));
    return ktime_mark(h, LEM_KERNEL_EXPAND, level, st);
}

// all 16 groups of one level: one dataflow launch (dataflow = 1, on levels
// with one-kernel visits on the CTA cut), else 16 group launches
static int expand_level_impl(lem_handle *h, int iter, int level, cudaStream_t st) {
    if (!h->p.dataflow || h->split_level[level] || h->grid_level[level]) {
        int rc = LEM_OK;
        for (int g = 0; g < 16 && rc == LEM_OK; ++g) rc = expand_group_impl(h, iter, level, g, st);
        return rc;
    }
    if (h->prop && !h->prop_set)
        return fail(h, LEM_ERR_ARG, "k_cnn > 0 but no proposal map was set (lem_set_proposals / lem_cnn_propose)");
    const lem::Level lv = level_of(h, level);
    const lem::KParams kp = kparams_level(h, level);
    const int first = h->item_off[level][0];
    const int n_items = h->item_off[level][15] + h->item_cnt[level][15] - first;
    LEM_CUDA(h, cudaMemsetAsync(h->d_done, 0, sizeof(unsigned) * h->done_cnt[level], st));
    LEM_CUDA(h, lem::launch_expand_group(planes_base(h), kp, lv, level, iter, h->d_iter, h->d_pairs, h->maxW,
                                         h->maxH, h->d_items + first, n_items, h->lab, h->phiA, h->prop, h->ctr,
                                         nullptr, h->d_queue + 2 * (16 * level), h->d_done, st));
    return ktime_mark(h, LEM_KERNEL_EXPAND, level, st);
}

// Captures one outer iteration (every level and group, then the increment of
// the device iteration index) as a CUDA graph on a private stream.
static int build_graph(lem_handle *h) {
    if (!h->cap_st) LEM_CUDA(h, cudaStreamCreateWithFlags(&h->cap_st, cudaStreamNonBlocking));
    // kernel-timing events are created before the capture begins
    if (h->ktime)
        while ((int)h->kev.size() < h->kn_last + 1) {
            cudaEvent_t ev = nullptr;
            LEM_CUDA(h, cudaEventCreate(&ev));
            h->kev.push_back(ev);
            h->kkind.push_back(-1);
        }
    LEM_CUDA(h, cudaStreamBeginCapture(h->cap_st, cudaStreamCaptureModeThreadLocal));
    h->capturing = true;
    int rc = ktime_mark(h, -1, 0, h->cap_st);
    for (int l = 0; l < h->p.n_levels && rc == LEM_OK; ++l) rc = expand_level_impl(h, -1, l, h->cap_st);
    cudaError_t e = rc == LEM_OK ? lem::launch_increment(h->d_iter, h->cap_st) : cudaSuccess;
    cudaGraph_t graph = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(h->cap_st, &graph);
    h->capturing = false;
    h->kn_graph = h->kn;
    if (rc != LEM_OK) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
    }
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return e != cudaSuccess ? cuda_fail(h, e, "graph capture") : cuda_fail(h, e2, "cudaStreamEndCapture");
    }
    h->graph = graph;
    LEM_CUDA(h, cudaGraphInstantiate(&h->gexec, h->graph, 0));
    return LEM_OK;
}

int lem_expand_group(lem_handle *h, int iter, int level, int group, lem_stats *stats) {
    if (!h) return fail(nullptr, LEM_ERR_ARG, "handle is NULL");
    if (iter < 0 || level < 0 || level >= h->p.n_levels || group < 0 || group > 15)
        return fail(h, LEM_ERR_ARG, "iter/level/group out of range");
    // kernel timing covers lem_expand_iteration only
    const bool kt = h->ktime;
    h->ktime = false;
    int rc = expand_group_impl(h, iter, level, group, h->st);
    h->ktime = kt;
    if (rc != LEM_OK) return rc;
    if (stats) {
        std::memset(stats, 0, sizeof(*stats));
        return read_counters(h, stats);
    }
    return LEM_OK;
}

int lem_expand_iteration(lem_handle *h, int n_iters, lem_stats *stats) {
    if (!h) return fail(nullptr, LEM_ERR_ARG, "handle is NULL");
    if (n_iters < 0) return fail(h, LEM_ERR_ARG, "n_iters < 0");
    if (stats) {
        for (cudaEvent_t &e : h->it_ev)
            if (!e) LEM_CUDA(h, cudaEventCreate(&e));
        LEM_CUDA(h, cudaEventRecord(h->it_ev[0], h->st));
    }
    int done = 0;
    // cooperative launches of the multi-CTA levels run directly, never as a graph
    const bool graph_ok = !(h->grid_level[0] || h->grid_level[1] || h->grid_level[2]);
    if (n_iters > 0 && h->p.use_graph && graph_ok && !h->gexec) {
        // the first iteration runs directly (it also sets the kernels' shared
        // memory limits), the graph is captured for the following ones
        int rc = ktime_mark(h, -1, 0, h->st);
        for (int l = 0; l < h->p.n_levels && rc == LEM_OK; ++l) rc = expand_level_impl(h, h->iter, l, h->st);
        if (rc != LEM_OK) return rc;
        h->kn_last = h->kn;
        ++h->iter;
        ++done;
        if ((rc = build_graph(h)) != LEM_OK) return rc;
    }
    if (done < n_iters && h->gexec) {
        // the device iteration index follows the host one
        LEM_CUDA(h, cudaMemcpyAsync(h->d_iter, &h->iter, sizeof(int), cudaMemcpyHostToDevice, h->st));
        for (; done < n_iters; ++done) {
            LEM_CUDA(h, cudaGraphLaunch(h->gexec, h->st));
            h->kn_last = h->kn_graph;
            ++h->iter;
        }
    }
    for (; done < n_iters; ++done) {
        int rc = ktime_mark(h, -1, 0, h->st);
        for (int l = 0; l < h->p.n_levels && rc == LEM_OK; ++l) rc = expand_level_impl(h, h->iter, l, h->st);
        if (rc != LEM_OK) return rc;
        h->kn_last = h->kn;
        ++h->iter;
    }
    if (stats) {
        LEM_CUDA(h, cudaEventRecord(h->it_ev[1], h->st));
        long long eq = 0;
        int rc = run_energy(h, &eq);
        if (rc != LEM_OK) return rc;
        if ((rc = read_counters(h, stats)) != LEM_OK) return rc;
        float ms = 0.f;
        LEM_CUDA(h, cudaEventElapsedTime(&ms, h->it_ev[0], h->it_ev[1]));
        stats->ms = ms;
        stats->energy_q = eq;
        stats->energy = (double)eq / h->p.quant_scale;
        if (stats->dep_waits_given_up > 0)
            return fail(h, LEM_ERR_CUDA, "a dataflow region gave up waiting for a neighbour; the labels are not valid");
    }
    return LEM_OK;
}

int lem_set_kernel_timing(lem_handle *h, int on) {
    if (!h) return fail(nullptr, LEM_ERR_ARG, "handle is NULL");
    if (on != 0 && on != 1) return fail(h, LEM_ERR_ARG, "on must be 0 or 1");
    if ((on != 0) != h->ktime) {
        // the captured graph is recaptured with (or without) the event nodes
        if (h->gexec) cudaGraphExecDestroy(h->gexec);
        if (h->graph) cudaGraphDestroy(h->graph);
        h->gexec = nullptr;
        h->graph = nullptr;
    }
    h->ktime = on != 0;
    h->kn = h->kn_last = h->kn_graph = 0;
    return LEM_OK;
}

int lem_get_kernel_times(lem_handle *h, lem_kernel_times *out) {
    if (!h || !out) return fail(h, LEM_ERR_ARG, "handle or output is NULL");
    std::memset(out, 0, sizeof(*out));
    if (!h->ktime || h->kn_last < 2) return LEM_OK;
    LEM_CUDA(h, cudaStreamSynchronize(h->st));
    for (int i = 1; i < h->kn_last; ++i) {
        float ms = 0.f;
        LEM_CUDA(h, cudaEventElapsedTime(&ms, h->kev[i - 1], h->kev[i]));
        const int k = h->kkind[i];
        if (k < 0 || k >= 3 * LEM_KERNEL_KINDS) continue;
        out->ms[k / LEM_KERNEL_KINDS][k % LEM_KERNEL_KINDS] += ms;
        out->launches[k / LEM_KERNEL_KINDS][k % LEM_KERNEL_KINDS] += 1;
    }
    return LEM_OK;
}

// labels of every pair into device buffers (pairs in order, each row-major)
static cudaError_t labels_out_all(lem_handle *h, float *abc, float *disp, float *cost) {
    for (int b = 0; b < h->B; ++b) {
        const lem::PairDesc &pd = h->pairs[b];
        cudaError_t e = lem::launch_labels_out(pd.H, pd.W, h->lab + pd.off, abc ? abc + 3 * pd.off : nullptr,
                                               disp ? disp + pd.off : nullptr, cost ? cost + pd.off : nullptr, h->st);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

int lem_get_labels(lem_handle *h, float *abc, float *disp, float *cost, int on_device) {
    if (!h) return fail(nullptr, LEM_ERR_ARG, "handle is NULL");
    const size_t n = (size_t)h->total;
    if (on_device) {
        LEM_CUDA(h, labels_out_all(h, abc, disp, cost));
        return LEM_OK;
    }
    float *d = nullptr;
    LEM_CUDA(h, cudaMalloc(&d, sizeof(float) * n * 5));
    cudaError_t e = labels_out_all(h, d, d + 3 * n, d + 4 * n);
    if (e == cudaSuccess && abc) e = cudaMemcpyAsync(abc, d, sizeof(float) * 3 * n, cudaMemcpyDeviceToHost, h->st);
    if (e == cudaSuccess && disp)
        e = cudaMemcpyAsync(disp, d + 3 * n, sizeof(float) * n, cudaMemcpyDeviceToHost, h->st);
    if (e == cudaSuccess && cost)
        e = cudaMemcpyAsync(cost, d + 4 * n, sizeof(float) * n, cudaMemcpyDeviceToHost, h->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
    cudaFree(d);
    if (e != cudaSuccess) return cuda_fail(h, e, "lem_get_labels");
    return LEM_OK;
}

int lem_set_labels(lem_handle *h, const float *abc, const float *cost, int on_device) {
    if (!h) return fail(nullptr, LEM_ERR_ARG, "handle is NULL");
    if (!abc) return fail(h, LEM_ERR_ARG, "abc is NULL");
    const size_t n = (size_t)h->total;
    const float *dabc = abc, *dcost = cost;
    float *tmp = nullptr;
    if (!on_device) {
        LEM_CUDA(h, cudaMalloc(&tmp, sizeof(float) * n * 4));
        cudaError_t e = cudaMemcpyAsync(tmp, abc, sizeof(float) * 3 * n, cudaMemcpyHostToDevice, h->st);
        if (e == cudaSuccess && cost)
            e = cudaMemcpyAsync(tmp + 3 * n, cost, sizeof(float) * n, cudaMemcpyHostToDevice, h->st);
        if (e != cudaSuccess) {
            cudaFree(tmp);
            return cuda_fail(h, e, "lem_set_labels copy");
        }
        dabc = tmp;
        dcost = cost ? tmp + 3 * n : nullptr;
    }
    cudaError_t e = cudaSuccess;
    for (int b = 0; b < h->B && e == cudaSuccess; ++b) {
        const lem::PairDesc &pd = h->pairs[b];
        e = lem::launch_labels_in(pd.H, pd.W, dabc + 3 * pd.off, dcost ? dcost + pd.off : nullptr, h->lab + pd.off,
                                  h->st);
        if (e == cudaSuccess && !dcost) {
            lem::KParams kp = kparams(h);
            e = lem::launch_pixel_costs(planes(h, b), kp, h->lab + pd.off, std::min(h->p.threads, 128), h->st);
        }
    }
    if (tmp) {
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
        cudaFree(tmp);
    }
    if (e != cudaSuccess) return cuda_fail(h, e, "lem_set_labels");
    return LEM_OK;
}

int lem_energy(lem_handle *h, double *energy, int64_t *energy_q) {
    if (!h) return fail(nullptr, LEM_ERR_ARG, "handle is NULL");
    long long eq = 0;
    int rc = run_energy(h, &eq);
    if (rc != LEM_OK) return rc;
    if (energy_q) *energy_q = eq;
    if (energy) *energy = (double)eq / h->p.quant_scale;
    return LEM_OK;
}

int lem_energy_pair(lem_handle *h, int pair, double *energy, int64_t *energy_q) {
    if (!h) return fail(nullptr, LEM_ERR_ARG, "handle is NULL");
    if (pair < 0 || pair >= h->B) return fail(h, LEM_ERR_ARG, "pair out of range");
    long long eq = 0;
    int rc = run_energy(h, &eq, pair);
    if (rc != LEM_OK) return rc;
    if (energy_q) *energy_q = eq;
    if (energy) *energy = (double)eq / h->p.quant_scale;
    return LEM_OK;
}

int lem_get_planes(lem_handle *h, float *left, float *right, float *guide, float *weights) {
    if (!h) return fail(nullptr, LEM_ERR_ARG, "handle is NULL");
    for (int b = 0; b < h->B; ++b) {
        const long long o = h->pairs[b].off;
        LEM_CUDA(h, lem::launch_planes_out(h->pairs[b].H, h->pairs[b].W, planes(h, b), left ? left + 4 * o : nullptr,
                                           right ? right + 4 * o : nullptr, guide ? guide + 9 * o : nullptr,
                                           weights ? weights + 4 * o : nullptr, h->st));
    }
    return LEM_OK;
}

int lem_mincut_batch_noalloc(const lem_region *regions, int n_regions, const int32_t *tcaps, const int32_t *ncaps,
                             uint8_t *take_alpha, int64_t *flow, int32_t *status, int max_rounds, int gr_interval,
                             void *stream) {
    if (!regions || !tcaps || !ncaps || !take_alpha || !flow || !status)
        return fail(nullptr, LEM_ERR_ARG, "lem_mincut_batch_noalloc: NULL pointer");
    if (n_regions < 1 || n_regions > LEM_NOALLOC_MAX_REGIONS)
        return fail(nullptr, LEM_ERR_ARG,
                    "lem_mincut_batch_noalloc: n_regions must be in [1, LEM_NOALLOC_MAX_REGIONS = " +
                        std::to_string(LEM_NOALLOC_MAX_REGIONS) + "], got " + std::to_string(n_regions));
    if (max_rounds < 1 || gr_interval < 1)
        return fail(nullptr, LEM_ERR_ARG, "lem_mincut_batch_noalloc: max_rounds/gr_interval must be >= 1");
    int max_nodes = 0;
    size_t smem = 0;
    for (int i = 0; i < n_regions; ++i) {
        const lem_region &r = regions[i];
        if (r.w < 1 || r.h < 1 || (int64_t)r.w * r.h > LEM_MAX_REGION_NODES)
            return fail(nullptr, LEM_ERR_SHAPE,
                        "lem_mincut_batch_noalloc: region " + std::to_string(i) + " is empty or too large");
        max_nodes = std::max(max_nodes, r.w * r.h);
        smem = std::max(smem, lem::cut_smem_bytes(r.w, r.h));
    }
    if (smem > 227 * 1024)
        return fail(nullptr, LEM_ERR_SHAPE, "lem_mincut_batch_noalloc: region shape needs more shared memory");
    lem::KParams kp{};
    kp.max_rounds = max_rounds;
    kp.gr_interval = gr_interval;
    cudaError_t e = lem::launch_mincut_noalloc(kp, regions, n_regions, max_nodes, smem, tcaps, ncaps, take_alpha,
                                               flow, status, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "lem_mincut_batch_noalloc");
    return LEM_OK;
}

int lem_set_proposals(lem_handle *h, int pair, const float *abc_dev) {
    if (!h) return fail(nullptr, LEM_ERR_ARG, "handle is NULL");
    if (!abc_dev || pair < 0 || pair >= h->B) return fail(h, LEM_ERR_ARG, "abc is NULL or pair out of range");
    if (!h->prop) return fail(h, LEM_ERR_ARG, "every k_cnn is 0: the handle keeps no proposal map");
    const lem::PairDesc &pd = h->pairs[pair];
    LEM_CUDA(h, lem::launch_props_in(pd.H * pd.W, abc_dev, h->prop + pd.off, h->st));
    // a batch needs every pair's map; pairs not set keep what the buffer holds
    h->prop_set = true;
    return LEM_OK;
}

int lem_get_proposals(lem_handle *h, int pair, float *abc_dev) {
    if (!h) return fail(nullptr, LEM_ERR_ARG, "handle is NULL");
    if (!abc_dev || pair < 0 || pair >= h->B) return fail(h, LEM_ERR_ARG, "abc is NULL or pair out of range");
    if (!h->prop || !h->prop_set) return fail(h, LEM_ERR_ARG, "no proposal map was set");
    const lem::PairDesc &pd = h->pairs[pair];
    LEM_CUDA(h, lem::launch_props_out(pd.H * pd.W, h->prop + pd.off, abc_dev, h->st));
    return LEM_OK;
}

int lem_cnn_features(lem_handle *h, int pair, float *x) {
    if (!h) return fail(nullptr, LEM_ERR_ARG, "handle is NULL");
    if (!x || pair < 0 || pair >= h->B) return fail(h, LEM_ERR_ARG, "x is NULL or pair out of range");
    const lem::PairDesc &pd = h->pairs[pair];
    if (!(pd.disp_max > 0)) return fail(h, LEM_ERR_ARG, "the network input needs disp_max > 0");
    LEM_CUDA(h, lem::launch_cnn_features(planes(h, pair), h->lab + pd.off, (float)pd.disp_max, x, h->st));
    return LEM_OK;
}

int lem_cnn_targets(lem_handle *h, int pair, float *t) {
    if (!h) return fail(nullptr, LEM_ERR_ARG, "handle is NULL");
    if (!t || pair < 0 || pair >= h->B) return fail(h, LEM_ERR_ARG, "t is NULL or pair out of range");
    const lem::PairDesc &pd = h->pairs[pair];
    if (!(pd.disp_max > 0)) return fail(h, LEM_ERR_ARG, "the network target needs disp_max > 0");
    LEM_CUDA(h, lem::launch_cnn_targets(h->lab + pd.off, pd.H, pd.W, (float)pd.disp_max, t, h->st));
    return LEM_OK;
}

int lem_cnn_propose(lem_cnn *net, lem_handle *h) {
    if (!h) return fail(nullptr, LEM_ERR_ARG, "handle is NULL");
    if (!net) return fail(h, LEM_ERR_ARG, "network is NULL");
    if (!h->prop) return fail(h, LEM_ERR_ARG, "every k_cnn is 0: the handle keeps no proposal map");
    for (const lem::PairDesc &pd : h->pairs)
        if (!(pd.disp_max > 0)) return fail(h, LEM_ERR_ARG, "the network input needs disp_max > 0");
    // quarter-resolution buffers sized for the largest pair, kept by the handle
    const size_t n4 = (size_t)((h->maxH + 3) / 4) * ((h->maxW + 3) / 4);
    if (!h->cnn_buf) LEM_CUDA(h, cudaMalloc(&h->cnn_buf, sizeof(float) * n4 * 10));
    float *x = h->cnn_buf, *y = h->cnn_buf + 7 * n4;
    int rc = LEM_OK;
    for (int b = 0; b < h->B && rc == LEM_OK; ++b) {
        const lem::PairDesc &pd = h->pairs[b];
        const float dmax = (float)pd.disp_max;
        cudaError_t e = lem::launch_cnn_features(planes(h, b), h->lab + pd.off, dmax, x, h->st);
        if (e != cudaSuccess) {
            rc = cuda_fail(h, e, "lem_cnn_propose features");
            break;
        }
        rc = lem::cnn_forward_on(net, x, (pd.H + 3) / 4, (pd.W + 3) / 4, y, h->st);
        if (rc != LEM_OK) {
            fail(h, rc, std::string("lem_cnn_propose forward: ") + lem::cnn_error(net));
            break;
        }
        e = lem::launch_cnn_upsample(y, pd.H, pd.W, dmax, h->prop + pd.off, h->st);
        if (e != cudaSuccess) rc = cuda_fail(h, e, "lem_cnn_propose upsample");
    }
    if (rc != LEM_OK) return rc;
    h->prop_set = true;
    return LEM_OK;
}

int lem_v3_params(lem_params *p, int width) {
    if (!p || width < 1) return fail(nullptr, LEM_ERR_ARG, "params NULL or width < 1");
    static const double kFrac[3] = {0.01, 0.03, 0.09};
    for (int l = 0; l < 3; ++l) {
        p->cell[l] = std::max(1, (int)std::lround(kFrac[l] * width));
        p->k_rans[l] = 1;
    }
    p->n_levels = 3;
    p->lambda = 0.5;
    return LEM_OK;
}

int lem_autotune(lem_handle *h, int repeats, lem_tuning *out) {
    if (!h) return fail(nullptr, LEM_ERR_ARG, "handle is NULL");
    if (repeats < 1 || repeats > 100) return fail(h, LEM_ERR_ARG, "repeats must be 1..100");
    if (h->prop && !h->prop_set) return fail(h, LEM_ERR_ARG, "k_cnn > 0 but no proposal map was set");
    const size_t n = (size_t)h->total;
    float4 *save = nullptr;
    LEM_CUDA(h, cudaMalloc(&save, sizeof(float4) * n));
    cudaEvent_t ev[2] = {nullptr, nullptr};
    lem::Counters ctr0{};
    cudaError_t e = cudaEventCreate(&ev[0]);
    if (e == cudaSuccess) e = cudaEventCreate(&ev[1]);
    if (e == cudaSuccess) e = cudaMemcpyAsync(save, h->lab, sizeof(float4) * n, cudaMemcpyDeviceToDevice, h->st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&ctr0, h->ctr, sizeof(ctr0), cudaMemcpyDeviceToHost, h->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
    lem_tuning res{};
    int rc = e == cudaSuccess ? LEM_OK : cuda_fail(h, e, "lem_autotune setup");
    const lem_params keep = h->p;
    // trial launches record no kernel-timing events
    const bool keep_ktime = h->ktime;
    h->ktime = false;
    static const int kThreads[4] = {128, 256, 512, 1024}, kGr[4] = {8, 16, 32, 64}, kRows[5] = {8, 12, 16, 24, 32};
    static const int kThreadsSplit[6] = {32, 64, 128, 256, 512, 1024};
    // time of `repeats` launches of groups 0 and 10 at `level` (with dataflow launches:
    // of the level's one launch), state restored after each; < 0 when the configuration
    // cannot launch
    auto trial = [&](int level, float &ms) -> int {
        float tot = 0.f;
        const bool whole = h->p.dataflow && !h->split_level[level] && !h->grid_level[level];
        const int ng = whole ? 1 : 2;
        for (int r = 0; r < repeats; ++r)
            for (int gi = 0; gi < ng; ++gi) {
                cudaError_t ce = cudaEventRecord(ev[0], h->st);
                if (ce != cudaSuccess) return cuda_fail(h, ce, "lem_autotune event");
                int rr = whole ? expand_level_impl(h, h->iter, level, h->st)
                               : expand_group_impl(h, h->iter, level, gi == 0 ? 0 : 10, h->st);
                if (rr != LEM_OK) {
                    cudaGetLastError();
                    ms = -1.f;
                    return LEM_OK;  // configuration does not launch: skipped
                }
                ce = cudaEventRecord(ev[1], h->st);
                if (ce == cudaSuccess) ce = cudaEventSynchronize(ev[1]);
                float t = 0.f;
                if (ce == cudaSuccess) ce = cudaEventElapsedTime(&t, ev[0], ev[1]);
                if (ce == cudaSuccess)
                    ce = cudaMemcpyAsync(h->lab, save, sizeof(float4) * n, cudaMemcpyDeviceToDevice, h->st);
                if (ce != cudaSuccess) return cuda_fail(h, ce, "lem_autotune trial");
                tot += t;
            }
        ms = tot / (float)(ng * repeats);
        return LEM_OK;
    };
    for (int l = 0; l < h->p.n_levels && rc == LEM_OK; ++l) {
        if (h->grid_level[l]) {
            // the multi-CTA path has no tuned parameters
            res.ms[l] = res.ms_default[l] = -1.f;
            continue;
        }
        // the default configuration first
        h->p.level_threads[l] = 0;
        h->p.level_gr_interval[l] = 0;
        h->p.level_strip_rows[l] = 0;
        float best = -1.f;
        rc = trial(l, best);
        res.ms_default[l] = best;
        const int s3 = 3 * h->p.cell[l];
        const int nodes = std::min(h->maxW, s3) * std::min(h->maxH, s3);
        int bt = h->split_level[l] ? lem::visit_cut_threads(nodes) : lem::threads_for_nodes(nodes);
        int bg = keep.gr_interval, bs = keep.strip_rows;
        // split levels: the cut CTA's size (32 .. 1024) and the relabel interval (the
        // warp data term has no strip rows); one-kernel levels: all three
        const int *threads = h->split_level[l] ? kThreadsSplit : kThreads;
        const int nthreads = h->split_level[l] ? 6 : 4, nrows = h->split_level[l] ? 1 : 5;
        for (int ti = 0; ti < nthreads && rc == LEM_OK; ++ti)
            for (int gi = 0; gi < 4 && rc == LEM_OK; ++gi)
                for (int si = 0; si < nrows && rc == LEM_OK; ++si) {
                    h->p.level_threads[l] = threads[ti];
                    h->p.level_gr_interval[l] = kGr[gi];
                    h->p.level_strip_rows[l] = h->split_level[l] ? 0 : kRows[si];
                    float ms = -1.f;
                    rc = trial(l, ms);
                    ++res.configs_tried;
                    if (rc == LEM_OK && ms >= 0.f && (best < 0.f || ms < best)) {
                        best = ms;
                        bt = threads[ti];
                        bg = kGr[gi];
                        bs = h->p.level_strip_rows[l];
                    }
                }
        h->p.level_threads[l] = bt;
        h->p.level_gr_interval[l] = bg;
        h->p.level_strip_rows[l] = bs;
        res.threads[l] = bt;
        res.gr_interval[l] = bg;
        res.strip_rows[l] = bs;
        res.ms[l] = best;
    }
    // statistics counters back to their values before tuning
    lem::Counters ctr1{};
    if (rc == LEM_OK) {
        e = cudaMemcpyAsync(&ctr1, h->ctr, sizeof(ctr1), cudaMemcpyDeviceToHost, h->st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(h->ctr, &ctr0, sizeof(ctr0), cudaMemcpyHostToDevice, h->st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
        if (e != cudaSuccess) rc = cuda_fail(h, e, "lem_autotune restore");
        else if (ctr1.limit_hits != ctr0.limit_hits)
            rc = fail(h, LEM_ERR_MAXFLOW_LIMIT, "a trial cut hit the push-relabel round limit");
        else if (ctr1.dep_give_ups != ctr0.dep_give_ups)
            rc = fail(h, LEM_ERR_CUDA, "a trial region gave up waiting for a neighbour");
    }
    h->ktime = keep_ktime;
    if (rc != LEM_OK) {
        // a failed trial may have left its moves in the labels
        h->p = keep;
        if (cudaMemcpyAsync(h->lab, save, sizeof(float4) * n, cudaMemcpyDeviceToDevice, h->st) == cudaSuccess)
            cudaStreamSynchronize(h->st);
    }
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    cudaFree(save);
    if (rc != LEM_OK) return rc;
    // the captured graph holds the old launch configuration
    if (h->gexec) cudaGraphExecDestroy(h->gexec);
    if (h->graph) cudaGraphDestroy(h->graph);
    h->gexec = nullptr;
    h->graph = nullptr;
    if (out) *out = res;
    return LEM_OK;
}

int lem_propose_batch(lem_handle *h, int iter, int level, const int *cells, int n_cells, float *alpha) {
    if (!h) return fail(nullptr, LEM_ERR_ARG, "handle is NULL");
    if (!cells || !alpha || n_cells < 1 || iter < 0 || level < 0 || level >= h->p.n_levels)
        return fail(h, LEM_ERR_ARG, "cells/alpha NULL, n_cells < 1, or iter/level out of range");
    if (h->prop && !h->prop_set) return fail(h, LEM_ERR_ARG, "k_cnn > 0 but no proposal map was set");
    const lem::PairDesc &pd = h->pairs[0];
    const int s = h->p.cell[level];
    const int nx = (pd.W + s - 1) / s, ny = (pd.H + s - 1) / s;
    for (int k = 0; k < n_cells; ++k)
        if (cells[2 * k] < 0 || cells[2 * k] >= nx || cells[2 * k + 1] < 0 || cells[2 * k + 1] >= ny)
            return fail(h, LEM_ERR_SHAPE, "cell " + std::to_string(k) + " is outside the grid");
    lem::Level lv;
    lv.s = s;
    lv.k_prop = h->p.k_prop[level];
    lv.k_rand = h->p.k_rand[level];
    lv.k_cnn = h->p.k_cnn[level];
    lv.k_rans = h->p.k_rans[level];
    lv.threads = 0;
    lem::KParams kp = kparams(h);
    kp.seed = pd.seed;
    kp.disp_min = pd.disp_min;
    kp.disp_max = pd.disp_max;
    int2 *dc = nullptr;
    long long *dq = nullptr;
    LEM_CUDA(h, cudaMalloc(&dc, sizeof(int2) * n_cells));
    cudaError_t e = cudaSuccess;
    if (lv.k_rans > 0 && s * s > lem::kRansacSmemCell)
        e = cudaMalloc(&dq, sizeof(long long) * (size_t)s * s * n_cells);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dc, cells, sizeof(int2) * n_cells, cudaMemcpyHostToDevice, h->st);
    if (e == cudaSuccess)
        e = lem::launch_propose_batch(planes(h, 0), kp, lv, level, iter, dc, n_cells, h->lab + pd.off,
                                      h->prop ? h->prop + pd.off : nullptr, alpha, dq, h->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
    cudaFree(dc);
    if (dq) cudaFree(dq);
    if (e != cudaSuccess) return cuda_fail(h, e, "lem_propose_batch");
    return LEM_OK;
}

void lem_default_post_params(lem_post_params *pp) {
    if (!pp) return;
    pp->lr_threshold = 1.0f;
    pp->median_radius = 20;
    pp->median_gamma = 10.0f;
}

int lem_postprocess(lem_handle *hL, lem_handle *hR, const lem_post_params *pp, float *disp, uint8_t *valid) {
    if (!hL || !hR) return fail(nullptr, LEM_ERR_ARG, "handle is NULL");
    if (!pp || !disp) return fail(hL, LEM_ERR_ARG, "params or disp is NULL");
    if (!(pp->lr_threshold >= 0.f) || pp->median_radius < 0 || pp->median_radius > 64 || !(pp->median_gamma > 0.f))
        return fail(hL, LEM_ERR_ARG, "lr_threshold >= 0, median_radius in [0, 64] and median_gamma > 0 are required");
    if (hL->pairs[0].H != hR->pairs[0].H || hL->pairs[0].W != hR->pairs[0].W)
        return fail(hL, LEM_ERR_SHAPE, "the two views differ in size");
    const size_t n = (size_t)hL->pairs[0].H * hL->pairs[0].W;
    // the right view's labels must be final before the left stream reads them
    if (hR->st != hL->st) LEM_CUDA(hL, cudaStreamSynchronize(hR->st));
    char *tmp = nullptr;
    LEM_CUDA(hL, cudaMalloc(&tmp, n * sizeof(float) + n));
    float *filled = (float *)tmp;
    uint8_t *vbuf = valid ? valid : (uint8_t *)(tmp + n * sizeof(float));
    cudaError_t e = lem::launch_postprocess(planes(hL, 0), hL->lab, hR->lab, pp->lr_threshold, pp->median_radius,
                                            pp->median_gamma, vbuf, filled, disp, hL->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(hL->st);
    cudaFree(tmp);
    if (e != cudaSuccess) return cuda_fail(hL, e, "lem_postprocess");
    return LEM_OK;
}

int64_t lem_evals_per_iteration(const lem_handle *h) {
    if (!h) return -1;
    int64_t tot = 0;
    for (const lem::PairDesc &pd : h->pairs)
        for (int l = 0; l < h->p.n_levels; ++l) {
            const int s = h->p.cell[l];
            const int nx = (pd.W + s - 1) / s, ny = (pd.H + s - 1) / s;
            const int np = h->p.k_prop[l] + h->p.k_rand[l] + h->p.k_rans[l] + (h->prop ? h->p.k_cnn[l] : 0);
            for (int j = 0; j < ny; ++j)
                for (int i = 0; i < nx; ++i) {
                    const int x0 = std::max(0, (i - 1) * s), x1 = std::min(pd.W, (i + 2) * s);
                    const int y0 = std::max(0, (j - 1) * s), y1 = std::min(pd.H, (j + 2) * s);
                    tot += (int64_t)(x1 - x0) * (y1 - y0) * np;
                }
        }
    return tot;
}

}  // extern "C"
