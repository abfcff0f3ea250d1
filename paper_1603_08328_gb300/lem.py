"""Python binding of the C ABI in ``include/lem.h`` (ctypes, argument marshalling only).

Every function of the header is exposed under the same name.  ``Stereo`` is a
thin convenience wrapper that keeps one handle and allocates the device
buffers of the batch calls as torch tensors; every step of the computation
runs in the CUDA library.  There is no CPU fallback: without the built library
or without a CUDA device these calls raise.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "liblem.so")

LEM_OK = 0
LEM_ERR_ARG = -1
LEM_ERR_SHAPE = -2
LEM_ERR_CUDA = -3
LEM_ERR_MAXFLOW_LIMIT = -4
LEM_ERR_OOM = -5
LEM_STORE_F32, LEM_STORE_F16, LEM_STORE_BF16 = 0, 1, 2
LEM_DATA_GF, LEM_DATA_BF = 0, 1
LEM_MAX_REGION_NODES = 5625
LEM_NOALLOC_MAX_REGIONS = 4096


LEM_IMG_U8, LEM_IMG_F16, LEM_IMG_BF16, LEM_IMG_F32 = 0, 1, 2, 3


class lem_image(C.Structure):
    _fields_ = [("data", C.c_void_p), ("height", C.c_int), ("width", C.c_int), ("stride_row", C.c_int64),
                ("on_device", C.c_int), ("channels", C.c_int), ("stride_px", C.c_int64), ("dtype", C.c_int)]


class lem_params(C.Structure):
    _fields_ = [
        ("gf_radius", C.c_int), ("gf_eps", C.c_double), ("tau_col", C.c_double), ("tau_grad", C.c_double),
        ("alpha_grad", C.c_double), ("lam", C.c_double), ("tau_dis", C.c_double), ("eps_w", C.c_double),
        ("gamma", C.c_double), ("disp_min", C.c_double), ("disp_max", C.c_double), ("n_levels", C.c_int),
        ("cell", C.c_int * 3), ("k_prop", C.c_int * 3), ("k_rand", C.c_int * 3), ("quant_scale", C.c_double),
        ("store_dtype", C.c_int), ("cond_fp64", C.c_double), ("seed", C.c_uint64), ("stream", C.c_void_p),
        ("max_rounds", C.c_int), ("gr_interval", C.c_int), ("strip_rows", C.c_int), ("threads", C.c_int),
        ("use_graph", C.c_int), ("candidates_per_visit", C.c_int), ("k_cnn", C.c_int * 3),
        ("level_threads", C.c_int * 3), ("level_gr_interval", C.c_int * 3), ("level_strip_rows", C.c_int * 3),
        ("k_rans", C.c_int * 3), ("data_term", C.c_int), ("bf_gamma", C.c_double), ("cluster_visits", C.c_int),
        ("split_visits", C.c_int), ("work_queue", C.c_int), ("dataflow", C.c_int),
    ]


class lem_post_params(C.Structure):
    _fields_ = [("lr_threshold", C.c_float), ("median_radius", C.c_int), ("median_gamma", C.c_float)]


class lem_tuning(C.Structure):
    _fields_ = [("threads", C.c_int * 3), ("gr_interval", C.c_int * 3), ("strip_rows", C.c_int * 3),
                ("ms", C.c_float * 3), ("ms_default", C.c_float * 3), ("configs_tried", C.c_int)]


class lem_region(C.Structure):
    _fields_ = [("x0", C.c_int), ("y0", C.c_int), ("w", C.c_int), ("h", C.c_int), ("img", C.c_int),
                ("cx0", C.c_int), ("cy0", C.c_int), ("cw", C.c_int), ("ch", C.c_int)]


LEM_KERNEL_EXPAND, LEM_KERNEL_VISIT_UNARY, LEM_KERNEL_VISIT_CUT, LEM_KERNEL_GRID = 0, 1, 2, 3
KERNEL_KIND_NAMES = ("k_expand_group", "k_visit_unary", "k_visit_cut", "k_expand_grid")


class lem_kernel_times(C.Structure):
    _fields_ = [("ms", (C.c_double * 4) * 3), ("launches", (C.c_int64 * 4) * 3)]


class lem_stats(C.Structure):
    _fields_ = [("energy_q", C.c_int64), ("energy", C.c_double), ("evals", C.c_int64), ("accepted", C.c_int64),
                ("maxflow_limit", C.c_int64), ("fp64_inverses", C.c_int32), ("iterations", C.c_int32),
                ("pr_rounds", C.c_int64), ("pr_global_relabels", C.c_int64), ("pr_bfs_levels", C.c_int64),
                ("accepted_by_kind", C.c_int64 * 4), ("dep_waits_given_up", C.c_int64),
                ("ms", C.c_double)]


_lib = None


def lib():
    """The loaded CUDA library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library not built: {LIB_PATH} (run __graft_entry__.build())")
        L = C.CDLL(LIB_PATH)
        P, vp, H = C.POINTER, C.c_void_p, C.c_void_p
        L.lem_default_params.argtypes = [P(lem_params)]
        L.lem_default_params.restype = None
        L.lem_create.argtypes = [P(lem_image), P(lem_image), P(lem_params), P(H)]
        L.lem_create_batch.argtypes = [P(lem_image), P(lem_image), C.c_int, P(lem_params), P(H)]
        L.lem_create_batch_ranges.argtypes = [P(lem_image), P(lem_image), C.c_int, P(C.c_double), P(lem_params),
                                              P(H)]
        L.lem_create_batch_ranges.restype = C.c_int
        L.lem_pair_count.argtypes = [H]
        L.lem_pair_info.argtypes = [H, C.c_int, P(C.c_int), P(C.c_int), P(C.c_int64)]
        L.lem_energy_pair.argtypes = [H, C.c_int, P(C.c_double), P(C.c_int64)]
        L.lem_destroy.argtypes = [H]
        L.lem_last_error.argtypes = [H]
        L.lem_last_error.restype = C.c_char_p
        L.lem_unary_batch.argtypes = [H, P(lem_region), C.c_int, vp, C.c_int, vp]
        L.lem_pairwise_batch.argtypes = [H, P(lem_region), C.c_int, vp, vp, vp, vp, vp]
        L.lem_mincut_batch.argtypes = [H, P(lem_region), C.c_int, vp, vp, vp, vp, vp]
        L.lem_expand_group.argtypes = [H, C.c_int, C.c_int, C.c_int, P(lem_stats)]
        L.lem_expand_iteration.argtypes = [H, C.c_int, P(lem_stats)]
        L.lem_get_labels.argtypes = [H, vp, vp, vp, C.c_int]
        L.lem_set_labels.argtypes = [H, vp, vp, C.c_int]
        L.lem_energy.argtypes = [H, P(C.c_double), P(C.c_int64)]
        L.lem_get_planes.argtypes = [H, vp, vp, vp, vp]
        L.lem_mincut_batch_noalloc.argtypes = [P(lem_region), C.c_int, vp, vp, vp, vp, vp, C.c_int, C.c_int, vp]
        L.lem_mincut_batch_noalloc.restype = C.c_int
        L.lem_evals_per_iteration.argtypes = [H]
        L.lem_evals_per_iteration.restype = C.c_int64
        L.lem_set_proposals.argtypes = [H, C.c_int, vp]
        L.lem_get_proposals.argtypes = [H, C.c_int, vp]
        N = C.c_void_p
        L.lem_cnn_create.argtypes = [C.c_uint64, vp, P(N)]
        L.lem_cnn_destroy.argtypes = [N]
        L.lem_cnn_last_error.argtypes = [N]
        L.lem_cnn_last_error.restype = C.c_char_p
        L.lem_cnn_check.argtypes = [N]
        L.lem_cnn_check.restype = C.c_int
        L.lem_cnn_num_params.argtypes = []
        L.lem_cnn_num_params.restype = C.c_int64
        L.lem_cnn_get_params.argtypes = [N, vp]
        L.lem_cnn_set_params.argtypes = [N, vp]
        L.lem_cnn_forward.argtypes = [N, vp, C.c_int, C.c_int, vp]
        L.lem_cnn_gradients.argtypes = [N, vp, vp, C.c_int, C.c_int, C.c_int, vp, vp, vp]
        L.lem_cnn_train_step.argtypes = [N, vp, vp, C.c_int, C.c_int, C.c_int, vp, C.c_float, vp]
        L.lem_cnn_features.argtypes = [H, C.c_int, vp]
        L.lem_cnn_targets.argtypes = [H, C.c_int, vp]
        L.lem_cnn_propose.argtypes = [N, H]
        L.lem_propose_batch.argtypes = [H, C.c_int, C.c_int, vp, C.c_int, vp]
        L.lem_propose_batch.restype = C.c_int
        L.lem_create_right_view.argtypes = [P(lem_image), P(lem_image), P(lem_params), P(H)]
        L.lem_create_right_view.restype = C.c_int
        L.lem_default_post_params.argtypes = [P(lem_post_params)]
        L.lem_default_post_params.restype = None
        L.lem_postprocess.argtypes = [H, H, P(lem_post_params), vp, vp]
        L.lem_postprocess.restype = C.c_int
        L.lem_autotune.argtypes = [H, C.c_int, P(lem_tuning)]
        L.lem_autotune.restype = C.c_int
        L.lem_v3_params.argtypes = [P(lem_params), C.c_int]
        L.lem_v3_params.restype = C.c_int
        L.lem_measure_peaks.argtypes = [vp, P(C.c_double), P(C.c_double)]
        L.lem_measure_peaks.restype = C.c_int
        L.lem_set_kernel_timing.argtypes = [H, C.c_int]
        L.lem_set_kernel_timing.restype = C.c_int
        L.lem_get_kernel_times.argtypes = [H, P(lem_kernel_times)]
        L.lem_get_kernel_times.restype = C.c_int
        for name in ("lem_set_proposals", "lem_get_proposals", "lem_cnn_create", "lem_cnn_destroy",
                     "lem_cnn_get_params", "lem_cnn_set_params", "lem_cnn_forward", "lem_cnn_gradients",
                     "lem_cnn_train_step", "lem_cnn_features", "lem_cnn_targets", "lem_cnn_propose"):
            getattr(L, name).restype = C.c_int
        for name in ("lem_create", "lem_create_batch", "lem_pair_count", "lem_pair_info", "lem_energy_pair",
                     "lem_destroy", "lem_unary_batch", "lem_pairwise_batch", "lem_mincut_batch",
                     "lem_expand_group", "lem_expand_iteration", "lem_get_labels", "lem_set_labels", "lem_energy",
                     "lem_get_planes"):
            getattr(L, name).restype = C.c_int
        _lib = L
    return _lib


class LemError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"lem error {code}: {msg}")
        self.code = code


# --- same-name wrappers of the C functions ------------------------------------

def lem_v3_params(p: lem_params, width: int) -> lem_params:
    _check(lib().lem_v3_params(C.byref(p), int(width)))
    return p


def lem_default_params(**overrides) -> lem_params:
    """The paper's defaults with `overrides` applied; v3_width=W first applies the
    Middlebury V3 settings for images W pixels wide (lem_v3_params)."""
    p = lem_params()
    lib().lem_default_params(C.byref(p))
    if "v3_width" in overrides:
        lem_v3_params(p, overrides.pop("v3_width"))
    for k, v in overrides.items():
        if k == "lambda":
            k = "lam"
        if k in ("cell", "k_prop", "k_rand", "k_cnn", "k_rans", "level_threads", "level_gr_interval",
                 "level_strip_rows"):
            v = list(v) + [0] * (3 - len(v))
            v = (C.c_int * 3)(*v)
        setattr(p, k, v)
    return p


def lem_last_error(h) -> str:
    s = lib().lem_last_error(h)
    return s.decode() if s else ""


def _check(rc, h=None):
    if rc != LEM_OK:
        raise LemError(rc, lem_last_error(h))
    return rc


def lem_create(left: lem_image, right: lem_image, params: lem_params):
    h = C.c_void_p()
    rc = lib().lem_create(C.byref(left), C.byref(right), C.byref(params), C.byref(h))
    _check(rc, None)
    return h


def lem_create_batch(lefts, rights, params: lem_params):
    n = len(lefts)
    la = (lem_image * n)(*lefts)
    ra = (lem_image * n)(*rights)
    h = C.c_void_p()
    rc = lib().lem_create_batch(la, ra, n, C.byref(params), C.byref(h))
    _check(rc, None)
    return h


def lem_create_batch_ranges(lefts, rights, disp_ranges, params: lem_params):
    n = len(lefts)
    la = (lem_image * n)(*lefts)
    ra = (lem_image * n)(*rights)
    rg = None
    if disp_ranges is not None:
        flat = [float(x) for r in disp_ranges for x in r]
        assert len(flat) == 2 * n
        rg = (C.c_double * (2 * n))(*flat)
    h = C.c_void_p()
    rc = lib().lem_create_batch_ranges(la, ra, n, rg, C.byref(params), C.byref(h))
    _check(rc, None)
    return h


def lem_pair_count(h) -> int:
    return lib().lem_pair_count(h)


def lem_pair_info(h, pair):
    hh, ww, off = C.c_int(), C.c_int(), C.c_int64()
    rc = lib().lem_pair_info(h, pair, C.byref(hh), C.byref(ww), C.byref(off))
    return rc, hh.value, ww.value, off.value


def lem_energy_pair(h, pair):
    e = C.c_double()
    q = C.c_int64()
    rc = lib().lem_energy_pair(h, pair, C.byref(e), C.byref(q))
    return rc, e.value, q.value


def lem_destroy(h):
    return lib().lem_destroy(h)


def _regions(regions):
    """(x0, y0, w, h[, img[, cx0, cy0, cw, ch]]) tuples -> lem_region array."""
    arr = (lem_region * len(regions))()
    for i, r in enumerate(regions):
        arr[i] = lem_region(*[int(x) for x in r])
    return arr


def lem_unary_batch(h, regions, labels_ptr, K, costs_ptr):
    return lib().lem_unary_batch(h, _regions(regions), len(regions), labels_ptr, K, costs_ptr)


def lem_pairwise_batch(h, regions, alpha_ptr, costs_alpha_ptr, tcaps_ptr, ncaps_ptr, const_ptr):
    return lib().lem_pairwise_batch(h, _regions(regions), len(regions), alpha_ptr, costs_alpha_ptr, tcaps_ptr,
                                    ncaps_ptr, const_ptr)


def lem_mincut_batch(h, regions, tcaps_ptr, ncaps_ptr, take_ptr, flow_ptr, status_ptr):
    return lib().lem_mincut_batch(h, _regions(regions), len(regions), tcaps_ptr, ncaps_ptr, take_ptr, flow_ptr,
                                  status_ptr)


def lem_expand_group(h, it, level, group, stats=None):
    return lib().lem_expand_group(h, it, level, group, C.byref(stats) if stats is not None else None)


def lem_expand_iteration(h, n_iters, stats=None):
    return lib().lem_expand_iteration(h, n_iters, C.byref(stats) if stats is not None else None)


def lem_get_labels(h, abc_ptr, disp_ptr, cost_ptr, on_device):
    return lib().lem_get_labels(h, abc_ptr, disp_ptr, cost_ptr, on_device)


def lem_set_labels(h, abc_ptr, cost_ptr, on_device):
    return lib().lem_set_labels(h, abc_ptr, cost_ptr, on_device)


def lem_energy(h):
    e = C.c_double()
    q = C.c_int64()
    rc = lib().lem_energy(h, C.byref(e), C.byref(q))
    return rc, e.value, q.value


def lem_get_planes(h, left_ptr, right_ptr, guide_ptr, weights_ptr):
    return lib().lem_get_planes(h, left_ptr, right_ptr, guide_ptr, weights_ptr)


def lem_mincut_batch_noalloc(regions, tcaps_ptr, ncaps_ptr, take_ptr, flow_ptr, status_ptr, max_rounds, gr_interval,
                             stream):
    return lib().lem_mincut_batch_noalloc(_regions(regions), len(regions), tcaps_ptr, ncaps_ptr, take_ptr, flow_ptr,
                                          status_ptr, max_rounds, gr_interval, stream)


def lem_set_kernel_timing(h, on):
    return lib().lem_set_kernel_timing(h, on)


def lem_get_kernel_times(h, out):
    return lib().lem_get_kernel_times(h, C.byref(out))


def lem_measure_peaks(stream=None):
    """(FP32 FMA TFLOP/s, shared-memory GB/s) of the current device, measured by the
    library's microbenchmarks on `stream` (a torch stream, a raw handle or None)."""
    st = getattr(stream, "cuda_stream", stream)
    f = C.c_double()
    b = C.c_double()
    _check(lib().lem_measure_peaks(C.c_void_p(st), C.byref(f), C.byref(b)))
    return f.value, b.value


def lem_evals_per_iteration(h) -> int:
    return lib().lem_evals_per_iteration(h)


def lem_propose_batch(h, it, level, cells, alpha_ptr):
    arr = np.ascontiguousarray(np.asarray(cells, np.int32).reshape(-1, 2))
    return lib().lem_propose_batch(h, it, level, C.c_void_p(arr.ctypes.data), arr.shape[0], alpha_ptr)


def lem_create_right_view(left: lem_image, right: lem_image, params: lem_params):
    h = C.c_void_p()
    rc = lib().lem_create_right_view(C.byref(left), C.byref(right), C.byref(params), C.byref(h))
    _check(rc, None)
    return h


def lem_default_post_params(**overrides) -> lem_post_params:
    pp = lem_post_params()
    lib().lem_default_post_params(C.byref(pp))
    for k, v in overrides.items():
        setattr(pp, k, v)
    return pp


def lem_postprocess(hL, hR, pp: lem_post_params, disp_ptr, valid_ptr):
    return lib().lem_postprocess(hL, hR, C.byref(pp), disp_ptr, valid_ptr)


def lem_autotune(h, repeats, out=None):
    return lib().lem_autotune(h, repeats, C.byref(out) if out is not None else None)


def lem_set_proposals(h, pair, abc_ptr):
    return lib().lem_set_proposals(h, pair, abc_ptr)


def lem_get_proposals(h, pair, abc_ptr):
    return lib().lem_get_proposals(h, pair, abc_ptr)


def lem_cnn_create(seed, stream=None):
    n = C.c_void_p()
    rc = lib().lem_cnn_create(seed, stream, C.byref(n))
    if rc != LEM_OK:
        raise LemError(rc, lem_cnn_last_error(None))
    return n


def lem_cnn_destroy(net):
    return lib().lem_cnn_destroy(net)


def lem_cnn_last_error(net) -> str:
    s = lib().lem_cnn_last_error(net)
    return s.decode() if s else ""


def lem_cnn_check(net):
    return lib().lem_cnn_check(net)


def lem_cnn_num_params() -> int:
    return lib().lem_cnn_num_params()


def lem_cnn_get_params(net, host_ptr):
    return lib().lem_cnn_get_params(net, host_ptr)


def lem_cnn_set_params(net, host_ptr):
    return lib().lem_cnn_set_params(net, host_ptr)


def lem_cnn_forward(net, x_ptr, H4, W4, y_ptr):
    return lib().lem_cnn_forward(net, x_ptr, H4, W4, y_ptr)


def lem_cnn_gradients(net, x_ptr, t_ptr, n_images, H4, W4, scale_ptr, loss_ptr, grads_ptr):
    return lib().lem_cnn_gradients(net, x_ptr, t_ptr, n_images, H4, W4, scale_ptr, loss_ptr, grads_ptr)


def lem_cnn_train_step(net, x_ptr, t_ptr, n_images, H4, W4, scale_ptr, lr, loss_ptr):
    return lib().lem_cnn_train_step(net, x_ptr, t_ptr, n_images, H4, W4, scale_ptr, lr, loss_ptr)


def lem_cnn_features(h, pair, x_ptr):
    return lib().lem_cnn_features(h, pair, x_ptr)


def lem_cnn_targets(h, pair, t_ptr):
    return lib().lem_cnn_targets(h, pair, t_ptr)


def lem_cnn_propose(net, h):
    return lib().lem_cnn_propose(net, h)


# --- convenience wrapper ------------------------------------------------------

def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


def _on_own_stream(fn):
    """Runs a method with the object's stream current, so that the tensors it
    allocates and copies are ordered with the library calls it makes."""
    import functools

    @functools.wraps(fn)
    def wrapped(self, *args, **kwargs):
        with self.torch.cuda.stream(self.stream):
            return fn(self, *args, **kwargs)
    return wrapped


class Stereo:
    """One handle on one pair.  Images are numpy uint8 (H, W, 3) host arrays or
    CUDA uint8 tensors; batch outputs are CUDA tensors.  Every call runs on
    `stream` (default: the current stream at construction), the tensor copies and
    allocations this wrapper makes included; results are ready in that stream's
    order."""

    def __init__(self, left, right, stream=None, disp_ranges=None, view="left", **params):
        """left/right: one image each, or lists of images (a batch of pairs); disp_ranges:
        optional (disp_min, disp_max) per pair of a batch.  view="right" estimates the right
        image's labels (lem_create_right_view: labels in mirrored coordinates)."""
        import torch
        self.torch = torch
        if not torch.cuda.is_available():
            raise RuntimeError("no CUDA device: the library has no CPU path")
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        self.params = lem_default_params(**params)
        self.params.stream = C.c_void_p(stream.cuda_stream)
        self._keep = []
        if isinstance(left, (list, tuple)):
            lis = [self._image(x) for x in left]
            ris = [self._image(x) for x in right]
            if disp_ranges is not None:
                self.h = lem_create_batch_ranges(lis, ris, disp_ranges, self.params)
            else:
                self.h = lem_create_batch(lis, ris, self.params)
            li = lis[0]
        else:
            li, ri = self._image(left), self._image(right)
            if view == "right":
                self.h = lem_create_right_view(li, ri, self.params)
            else:
                self.h = lem_create(li, ri, self.params)
        self.view = view
        self.H, self.W = li.height, li.width
        self.pairs = [lem_pair_info(self.h, b)[1:] for b in range(lem_pair_count(self.h))]
        self.total = sum(hh * ww for hh, ww, _ in self.pairs)

    def _image(self, img):
        """An (H, W, C >= 3) image: a CUDA tensor (uint8, float16, bfloat16, float32; any strides
        with a unit channel step) or a host array (uint8, float16, float32), passed as it is."""
        torch = self.torch
        if isinstance(img, torch.Tensor):
            codes = {torch.uint8: LEM_IMG_U8, torch.float16: LEM_IMG_F16, torch.bfloat16: LEM_IMG_BF16,
                     torch.float32: LEM_IMG_F32}
            assert img.is_cuda and img.dim() == 3 and img.dtype in codes and img.stride(2) == 1
            self._keep.append(img)
            es = img.element_size()
            return lem_image(img.data_ptr(), img.shape[0], img.shape[1], img.stride(0) * es, 1, img.shape[2],
                             img.stride(1) * es, codes[img.dtype])
        a = np.asarray(img)
        codes = {np.dtype(np.uint8): LEM_IMG_U8, np.dtype(np.float16): LEM_IMG_F16, np.dtype(np.float32): LEM_IMG_F32}
        if a.dtype not in codes:
            a = a.astype(np.uint8)
        a = np.ascontiguousarray(a)
        self._keep.append(a)
        return lem_image(a.ctypes.data, a.shape[0], a.shape[1], a.strides[0], 0, a.shape[2], a.strides[1],
                         codes[a.dtype])

    def close(self):
        if getattr(self, "h", None):
            lem_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def check(self, rc):
        return _check(rc, self.h)

    # batch calls ------------------------------------------------------------
    @_on_own_stream
    def unary(self, regions, labels):
        """labels: (n_regions, K, 3) float32 -> list of (K, h, w) cost tensors."""
        torch = self.torch
        lab = torch.as_tensor(np.ascontiguousarray(labels, np.float32)).cuda()
        n, K = lab.shape[0], lab.shape[1]
        sizes = [r[2] * r[3] for r in regions]
        out = torch.empty(K * sum(sizes), dtype=torch.float32, device="cuda")
        self.check(lem_unary_batch(self.h, regions, _ptr(lab), K, _ptr(out)))
        res, off = [], 0
        for r, s in zip(regions, sizes):
            res.append(out[off:off + K * s].view(K, r[3], r[2]))
            off += K * s
        return res

    @_on_own_stream
    def pairwise(self, regions, alpha, costs_alpha):
        torch = self.torch
        al = torch.as_tensor(np.ascontiguousarray(alpha, np.float32)).cuda()
        ca = torch.cat([torch.as_tensor(c, dtype=torch.float32).reshape(-1).cuda() for c in costs_alpha])
        n = sum(r[2] * r[3] for r in regions)
        tc = torch.empty(2 * n, dtype=torch.int32, device="cuda")
        nc = torch.empty(4 * n, dtype=torch.int32, device="cuda")
        ct = torch.empty(len(regions), dtype=torch.int64, device="cuda")
        self.check(lem_pairwise_batch(self.h, regions, _ptr(al), _ptr(ca), _ptr(tc), _ptr(nc), _ptr(ct)))
        return tc, nc, ct

    @_on_own_stream
    def mincut(self, regions, tcaps, ncaps):
        torch = self.torch
        n = sum(r[2] * r[3] for r in regions)
        tc = torch.as_tensor(tcaps, dtype=torch.int32).reshape(-1).cuda().contiguous()
        nc = torch.as_tensor(ncaps, dtype=torch.int32).reshape(-1).cuda().contiguous()
        take = torch.empty(n, dtype=torch.uint8, device="cuda")
        flow = torch.empty(len(regions), dtype=torch.int64, device="cuda")
        st = torch.empty(len(regions), dtype=torch.int32, device="cuda")
        self.check(lem_mincut_batch(self.h, regions, _ptr(tc), _ptr(nc), _ptr(take), _ptr(flow), _ptr(st)))
        return take, flow, st

    # method ---------------------------------------------------------------------
    def expand_group(self, it, level, group):
        s = lem_stats()
        self.check(lem_expand_group(self.h, it, level, group, s))
        return s

    def iterate(self, n=1, stats=True):
        s = lem_stats() if stats else None
        self.check(lem_expand_iteration(self.h, n, s))
        return s

    @_on_own_stream
    def labels(self, pair=None):
        """(abc, disp, cost) of pair 0 (single pair) or of `pair`; pair='all' gives flat arrays."""
        torch = self.torch
        abc = torch.empty(self.total, 3, dtype=torch.float32, device="cuda")
        disp = torch.empty(self.total, dtype=torch.float32, device="cuda")
        cost = torch.empty(self.total, dtype=torch.float32, device="cuda")
        self.check(lem_get_labels(self.h, _ptr(abc), _ptr(disp), _ptr(cost), 1))
        if pair == "all":
            return abc, disp, cost
        b = 0 if pair is None else pair
        hh, ww, off = self.pairs[b]
        n = hh * ww
        return abc[off:off + n].view(hh, ww, 3), disp[off:off + n].view(hh, ww), cost[off:off + n].view(hh, ww)

    @_on_own_stream
    def set_labels(self, abc, cost=None):
        torch = self.torch
        a = torch.as_tensor(np.ascontiguousarray(abc, np.float32)).cuda()
        c = torch.as_tensor(np.ascontiguousarray(cost, np.float32)).cuda() if cost is not None else None
        self.check(lem_set_labels(self.h, _ptr(a), _ptr(c), 1))

    def energy(self, pair=None):
        rc, e, q = lem_energy(self.h) if pair is None else lem_energy_pair(self.h, pair)
        self.check(rc)
        return e, q

    @_on_own_stream
    def planes(self):
        torch = self.torch
        n = self.total
        L = torch.empty(n, 4, device="cuda")
        R = torch.empty(n, 4, device="cuda")
        G = torch.empty(n, 9, device="cuda")
        Wt = torch.empty(n, 4, device="cuda")
        self.check(lem_get_planes(self.h, _ptr(L), _ptr(R), _ptr(G), _ptr(Wt)))
        if len(self.pairs) == 1:
            H, W = self.H, self.W
            return L.view(H, W, 4), R.view(H, W, 4), G.view(H, W, 9), Wt.view(H, W, 4)
        return L, R, G, Wt

    def evals_per_iteration(self):
        return lem_evals_per_iteration(self.h)

    def set_kernel_timing(self, on=True):
        """Events between the expansion launches of every outer iteration (lem_set_kernel_timing)."""
        self.check(lem_set_kernel_timing(self.h, 1 if on else 0))

    def kernel_times(self):
        """{(level, kernel name): (ms, launches)} of the last outer iteration (lem_get_kernel_times)."""
        t = lem_kernel_times()
        self.check(lem_get_kernel_times(self.h, t))
        return {(l, n): (t.ms[l][k], t.launches[l][k]) for l in range(3) for k, n in enumerate(KERNEL_KIND_NAMES)
                if t.launches[l][k]}

    @_on_own_stream
    def proposals_of(self, it, level, cells, nprop):
        """Candidates of one visit of each cell (lem_propose_batch): (n_cells, nprop, 3) numpy."""
        out = self.torch.empty(len(cells) * nprop * 3, dtype=self.torch.float32, device="cuda")
        self.check(lem_propose_batch(self.h, it, level, cells, _ptr(out)))
        return out.cpu().numpy().reshape(len(cells), nprop, 3)

    @_on_own_stream
    def postprocess(self, right_view: "Stereo", **pp):
        """Consistency check with the right view, occlusion filling and weighted median
        (lem_postprocess); returns (disparity (H, W), consistent (H, W) bool) CUDA tensors."""
        torch = self.torch
        disp = torch.empty(self.H, self.W, dtype=torch.float32, device="cuda")
        valid = torch.empty(self.H, self.W, dtype=torch.uint8, device="cuda")
        self.check(lem_postprocess(self.h, right_view.h, lem_default_post_params(**pp), _ptr(disp), _ptr(valid)))
        return disp, valid.bool()

    def autotune(self, repeats=2):
        """Picks the per-level launch configuration (lem_autotune); returns the lem_tuning."""
        t = lem_tuning()
        self.check(lem_autotune(self.h, repeats, t))
        for k in ("level_threads", "level_gr_interval", "level_strip_rows"):
            src = {"level_threads": t.threads, "level_gr_interval": t.gr_interval,
                   "level_strip_rows": t.strip_rows}[k]
            setattr(self.params, k, (C.c_int * 3)(*src))
        return t

    # learned proposer -------------------------------------------------------------
    @_on_own_stream
    def set_proposals(self, abc, pair=0):
        """Proposal map (H, W, 3) of plane labels for the k_cnn map candidates."""
        torch = self.torch
        a = torch.as_tensor(np.ascontiguousarray(abc, np.float32)).cuda().contiguous()
        self._prop_keep = a
        self.check(lem_set_proposals(self.h, pair, _ptr(a)))

    @_on_own_stream
    def proposals(self, pair=0):
        hh, ww, _ = self.pairs[pair]
        out = self.torch.empty(hh, ww, 3, dtype=self.torch.float32, device="cuda")
        self.check(lem_get_proposals(self.h, pair, _ptr(out)))
        return out

    def quarter_shape(self, pair=0):
        hh, ww, _ = self.pairs[pair]
        return (hh + 3) // 4, (ww + 3) // 4

    @_on_own_stream
    def cnn_features(self, pair=0):
        H4, W4 = self.quarter_shape(pair)
        x = self.torch.empty(H4, W4, 7, dtype=self.torch.float32, device="cuda")
        self.check(lem_cnn_features(self.h, pair, _ptr(x)))
        return x

    @_on_own_stream
    def cnn_targets(self, pair=0):
        H4, W4 = self.quarter_shape(pair)
        t = self.torch.empty(H4, W4, 3, dtype=self.torch.float32, device="cuda")
        self.check(lem_cnn_targets(self.h, pair, _ptr(t)))
        return t

    def cnn_propose(self, net: "ProposalNet"):
        self.check(lem_cnn_propose(net.net, self.h))


class ProposalNet:
    """The proposal network (lem_cnn_* entry points).  Inputs and outputs are CUDA tensors."""

    def __init__(self, seed=0, stream=None):
        import torch
        self.torch = torch
        if not torch.cuda.is_available():
            raise RuntimeError("no CUDA device: the library has no CPU path")
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        self.net = lem_cnn_create(seed, C.c_void_p(stream.cuda_stream))

    def close(self):
        if getattr(self, "net", None):
            lem_cnn_destroy(self.net)
            self.net = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def check(self, rc):
        if rc != LEM_OK:
            raise LemError(rc, lem_cnn_last_error(self.net))
        return rc

    def sync_check(self):
        """Synchronise and raise if a convolution tile gave up waiting for the tensor core."""
        self.check(lem_cnn_check(self.net))

    def get_params(self) -> np.ndarray:
        out = np.empty(lem_cnn_num_params(), np.float32)
        self.check(lem_cnn_get_params(self.net, C.c_void_p(out.ctypes.data)))
        return out

    def set_params(self, flat):
        a = np.ascontiguousarray(flat, np.float32)
        assert a.size == lem_cnn_num_params()
        self.check(lem_cnn_set_params(self.net, C.c_void_p(a.ctypes.data)))

    @_on_own_stream
    def forward(self, x):
        """x: (H4, W4, 7) CUDA float32 -> (H4, W4, 3)."""
        x = x.contiguous()
        H4, W4 = x.shape[:2]
        y = self.torch.empty(H4, W4, 3, dtype=self.torch.float32, device="cuda")
        self.check(lem_cnn_forward(self.net, _ptr(x), H4, W4, _ptr(y)))
        return y

    @_on_own_stream
    def gradients(self, x, t, scale=(1.0, 1.0, 1.0)):
        """x: (n, H4, W4, 7), t: (n, H4, W4, 3) CUDA -> (loss, flat gradients in get_params order)."""
        x, t = x.contiguous(), t.contiguous()
        n, H4, W4 = x.shape[:3]
        sc = np.ascontiguousarray(scale, np.float32)
        loss = np.zeros(1, np.float32)
        g = np.empty(lem_cnn_num_params(), np.float32)
        self.check(lem_cnn_gradients(self.net, _ptr(x), _ptr(t), n, H4, W4, C.c_void_p(sc.ctypes.data),
                                     C.c_void_p(loss.ctypes.data), C.c_void_p(g.ctypes.data)))
        return float(loss[0]), g

    @_on_own_stream
    def train_step(self, x, t, lr, scale=(1.0, 1.0, 1.0)):
        x, t = x.contiguous(), t.contiguous()
        n, H4, W4 = x.shape[:3]
        sc = np.ascontiguousarray(scale, np.float32)
        loss = np.zeros(1, np.float32)
        self.check(lem_cnn_train_step(self.net, _ptr(x), _ptr(t), n, H4, W4, C.c_void_p(sc.ctypes.data), lr,
                                      C.c_void_p(loss.ctypes.data)))
        return float(loss[0])

    @staticmethod
    def unflatten(flat):
        """Flat parameters -> list of (w (3, 3, Cin, Cout), b (Cout,))."""
        out, o = [], 0
        for ci, co in LAYERS:
            w = np.asarray(flat[o:o + 9 * ci * co]).reshape(3, 3, ci, co)
            o += 9 * ci * co
            b = np.asarray(flat[o:o + co])
            o += co
            out.append((w, b))
        return out


LAYERS = [(7, 32), (32, 32), (32, 32), (32, 32), (32, 32), (32, 3)]
