"""FP64 CPU oracle for local-expansion-move stereo (arXiv 1603.08328).

TEST INFRASTRUCTURE ONLY.  The tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` are the only users.  The product library never
loads this module, and this module never loads the product library: the two
share no code.  ``lem_oracle.c`` is the implementation; this file compiles it
with gcc and binds it with ctypes.

Parity pins for every function are in ``tests/test_oracle_*.py``.  Functions
with no pin: none.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lem_oracle.c")
_LIB = os.path.join(_HERE, "liblem_oracle.so")


def build(force: bool = False) -> str:
    """Compile the oracle (gcc, OpenMP, no fused multiply-add)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fopenmp",
               _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class Params(C.Structure):
    _fields_ = [
        ("gf_radius", C.c_int),
        ("gf_eps", C.c_double),
        ("tau_col", C.c_double),
        ("tau_grad", C.c_double),
        ("alpha_grad", C.c_double),
        ("lam", C.c_double),
        ("tau_dis", C.c_double),
        ("eps_w", C.c_double),
        ("gamma", C.c_double),
        ("disp_min", C.c_double),
        ("disp_max", C.c_double),
        ("n_levels", C.c_int),
        ("cell", C.c_int * 3),
        ("k_prop", C.c_int * 3),
        ("k_rand", C.c_int * 3),
        ("quant_scale", C.c_double),
        ("seed", C.c_uint64),
        ("n_threads", C.c_int),
        ("reverse_order", C.c_int),
        ("visit", C.c_int),
        ("k_cnn", C.c_int * 3),
        ("k_rans", C.c_int * 3),
        ("data_term", C.c_int),
        ("bf_gamma", C.c_double),
    ]


# parameter values of the paper's experiments (Sec. 4, settings)
PAPER_DEFAULTS = dict(gf_radius=10, gf_eps=1e-4, tau_col=10.0, tau_grad=2.0, alpha_grad=0.9,
                      lam=1.0, tau_dis=1.0, eps_w=0.01, gamma=10.0, disp_min=0.0, disp_max=60.0,
                      n_levels=3, cell=(5, 15, 25), k_prop=(1, 2, 2), k_rand=(7, 0, 0),
                      quant_scale=65536.0, seed=1, n_threads=0, reverse_order=0, visit=1,
                      k_cnn=(0, 0, 0), k_rans=(0, 0, 0), data_term=0, bf_gamma=10.0)


def make_params(**kw) -> Params:
    d = dict(PAPER_DEFAULTS)
    d.update(kw)
    p = Params()
    for k, v in d.items():
        if k in ("cell", "k_prop", "k_rand", "k_cnn", "k_rans"):
            v = list(v) + [0] * (3 - len(v))
            setattr(p, k, (C.c_int * 3)(*v))
        else:
            setattr(p, k, v)
    return p


_lib = None


def lib():
    global _lib
    if _lib is None:
        # LEM_ORACLE_LIB: a separately compiled copy (the mutation tests load copies
        # with planted mistakes to show that the pins catch them)
        _lib = C.CDLL(os.environ.get("LEM_ORACLE_LIB") or build())
        L = _lib
        P = C.POINTER
        dp, fp, ip, i32p, u8p, i64p = (P(C.c_double), P(C.c_float), P(C.c_int), P(C.c_int32),
                                       P(C.c_uint8), P(C.c_int64))
        L.lo_create.restype = C.c_void_p
        L.lo_create.argtypes = [u8p, u8p, C.c_int, C.c_int, P(Params)]
        L.lo_create_f64.restype = C.c_void_p
        L.lo_create_f64.argtypes = [dp, dp, C.c_int, C.c_int, P(Params)]
        L.lo_destroy.argtypes = [C.c_void_p]
        L.lo_get_planes.argtypes = [C.c_void_p, dp, dp, dp, dp, dp]
        L.lo_rho.restype = C.c_double
        L.lo_rho.argtypes = [C.c_void_p, C.c_double, C.c_double, C.c_double, C.c_int, C.c_int]
        L.lo_gf_coeffs.argtypes = [C.c_void_p, C.c_double, C.c_double, C.c_double, C.c_int, C.c_int, dp]
        L.lo_phi_def.restype = C.c_double
        L.lo_phi_def.argtypes = [C.c_void_p, C.c_double, C.c_double, C.c_double, C.c_int, C.c_int]
        L.lo_phi_weights.argtypes = [C.c_void_p, C.c_int, C.c_int, dp]
        L.lo_phi_bf.restype = C.c_double
        L.lo_phi_bf.argtypes = [C.c_void_p, C.c_double, C.c_double, C.c_double, C.c_int, C.c_int]
        L.lo_region_cost.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, fp, dp]
        L.lo_psibar.restype = C.c_double
        L.lo_psibar.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, fp, fp]
        L.lo_psi.restype = C.c_double
        L.lo_psi.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int, fp, fp]
        L.lo_energy_of.argtypes = [C.c_void_p, fp, dp, dp, i64p]
        L.lo_energy.argtypes = [C.c_void_p, dp, i64p]
        L.lo_build_graph.restype = C.c_int64
        L.lo_build_graph.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, fp, fp, dp, dp,
                                     i32p, i32p, ip, u8p]
        for name in ("lo_maxflow_dinic", "lo_maxflow_ek", "lo_mincut_enum"):
            f = getattr(L, name)
            f.restype = C.c_int64
            f.argtypes = [C.c_int, C.c_int, i32p, i32p, u8p]
        L.lo_splitmix64_next.restype = C.c_uint64
        L.lo_splitmix64_next.argtypes = [P(C.c_uint64)]
        L.lo_proposal_stream.restype = C.c_uint64
        L.lo_proposal_stream.argtypes = [C.c_uint64, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int]
        L.lo_init_stream.restype = C.c_uint64
        L.lo_init_stream.argtypes = [C.c_uint64, C.c_int64]
        L.lo_init_label.argtypes = [C.c_uint64, C.c_int, C.c_int, C.c_int, C.c_double, C.c_double, fp]
        L.lo_propose.argtypes = [fp, C.c_int, C.c_uint64, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int,
                                 C.c_double, C.c_double, C.c_double, C.c_double, fp]
        L.lo_propose_map.argtypes = [fp, C.c_int, C.c_uint64, C.c_int, C.c_int, C.c_int, C.c_int, fp]
        L.lo_set_proposals.argtypes = [C.c_void_p, fp]
        L.lo_propose_ransac.argtypes = [fp, C.c_int, C.c_uint64, C.c_int, C.c_int, C.c_int, C.c_int, fp]
        L.lo_init_state.argtypes = [C.c_void_p]
        L.lo_set_labels.argtypes = [C.c_void_p, fp]
        L.lo_get_state.argtypes = [C.c_void_p, fp, dp]
        L.lo_put_state.argtypes = [C.c_void_p, fp, dp]
        L.lo_expand_group.restype = C.c_longlong
        L.lo_expand_group.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int, P(C.c_longlong)]
        L.lo_expand_cells.restype = C.c_longlong
        L.lo_expand_cells.argtypes = [C.c_void_p, C.c_int, C.c_int, ip, C.c_int, P(C.c_longlong)]
        L.lo_visit_candidates.restype = C.c_int
        L.lo_visit_candidates.argtypes = [C.c_void_p, fp, C.c_int, C.c_int, C.c_int, C.c_int, fp]
        L.lo_iterate.restype = C.c_longlong
        L.lo_iterate.argtypes = [C.c_void_p, C.c_int, P(C.c_longlong)]
        L.lo_region_of.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, ip, ip]
        L.lo_group_cells.restype = C.c_int
        L.lo_group_cells.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, ip]
        L.lo_openmp_threads.restype = C.c_int
    return _lib


def _ptr(a: np.ndarray, ct):
    return a.ctypes.data_as(C.POINTER(ct))


def _f32(x):
    return np.ascontiguousarray(np.asarray(x, dtype=np.float32))


class Oracle:
    """One stereo pair preprocessed in FP64, plus the method's state (labels, cost cache)."""

    def __init__(self, left, right, **params):
        L = lib()
        self.params = make_params(**params)
        self.p = dict(PAPER_DEFAULTS, **params)
        left = np.ascontiguousarray(left)
        right = np.ascontiguousarray(right)
        self.H, self.W = left.shape[:2]
        if left.dtype == np.uint8:
            self.h = L.lo_create(_ptr(left, C.c_uint8), _ptr(right, C.c_uint8), self.H, self.W,
                                 C.byref(self.params))
        else:
            l64 = np.ascontiguousarray(left, dtype=np.float64)
            r64 = np.ascontiguousarray(right, dtype=np.float64)
            self.h = L.lo_create_f64(_ptr(l64, C.c_double), _ptr(r64, C.c_double), self.H, self.W,
                                     C.byref(self.params))

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            lib().lo_destroy(h)
            self.h = None

    # --- preprocessed planes -------------------------------------------------
    def planes(self):
        H, W = self.H, self.W
        Lc = np.empty((H, W, 4)); Rc = np.empty((H, W, 4)); mu = np.empty((H, W, 3))
        A = np.empty((H, W, 3, 3)); wq = np.empty((H, W, 4))
        lib().lo_get_planes(self.h, *[_ptr(x, C.c_double) for x in (Lc, Rc, mu, A, wq)])
        return dict(L=Lc, R=Rc, mu=mu, A=A, w=wq)

    # --- data term -----------------------------------------------------------
    def rho(self, abc, u, v):
        a, b, c = (float(x) for x in _f32(abc))
        return lib().lo_rho(self.h, a, b, c, int(u), int(v))

    def gf_coeffs(self, abc, kx, ky):
        out = np.empty(4)
        a, b, c = (float(x) for x in _f32(abc))
        lib().lo_gf_coeffs(self.h, a, b, c, int(kx), int(ky), _ptr(out, C.c_double))
        return out

    def phi_def(self, abc, u, v):
        a, b, c = (float(x) for x in _f32(abc))
        return lib().lo_phi_def(self.h, a, b, c, int(u), int(v))

    def phi_bf(self, abc, u, v):
        a, b, c = (float(x) for x in _f32(abc))
        return lib().lo_phi_bf(self.h, a, b, c, int(u), int(v))

    def phi_weights(self, u, v):
        r = self.p["gf_radius"]
        out = np.empty((4 * r + 1, 4 * r + 1))
        lib().lo_phi_weights(self.h, int(u), int(v), _ptr(out, C.c_double))
        return out

    def region_cost(self, x0, y0, w, h, abc):
        out = np.empty((h, w))
        lab = _f32(abc)
        lib().lo_region_cost(self.h, x0, y0, w, h, _ptr(lab, C.c_float), _ptr(out, C.c_double))
        return out

    # --- smoothness / energy -------------------------------------------------
    def psi(self, u, v, d, fp, fq):
        fp = _f32(fp); fq = _f32(fq)
        return lib().lo_psi(self.h, u, v, d, _ptr(fp, C.c_float), _ptr(fq, C.c_float))

    def energy_of(self, lab, cost):
        lab = _f32(lab); cost = np.ascontiguousarray(cost, dtype=np.float64)
        e = C.c_double(); q = C.c_int64()
        lib().lo_energy_of(self.h, _ptr(lab, C.c_float), _ptr(cost, C.c_double), C.byref(e), C.byref(q))
        return e.value, q.value

    def energy(self):
        e = C.c_double(); q = C.c_int64()
        lib().lo_energy(self.h, C.byref(e), C.byref(q))
        return e.value, q.value

    def build_graph(self, x0, y0, w, h, alpha, lab, cost, phi_alpha):
        tcap = np.zeros((h, w, 2), np.int32)
        ncap = np.zeros((h, w, 4), np.int32)
        mask = np.zeros((h, w), np.uint8)
        ncl = C.c_int()
        a = _f32(alpha); lab = _f32(lab)
        cost = np.ascontiguousarray(cost, dtype=np.float64)
        phA = np.ascontiguousarray(phi_alpha, dtype=np.float64)
        const = lib().lo_build_graph(self.h, x0, y0, w, h, _ptr(a, C.c_float), _ptr(lab, C.c_float),
                                     _ptr(cost, C.c_double), _ptr(phA, C.c_double), _ptr(tcap, C.c_int32),
                                     _ptr(ncap, C.c_int32), C.byref(ncl), _ptr(mask, C.c_uint8))
        return dict(tcap=tcap, ncap=ncap, const=const, nclamp=ncl.value, clamp_mask=mask)

    # --- method state --------------------------------------------------------
    def init_state(self):
        lib().lo_init_state(self.h)

    def state(self):
        lab = np.empty((self.H, self.W, 3), np.float32)
        cost = np.empty((self.H, self.W))
        lib().lo_get_state(self.h, _ptr(lab, C.c_float), _ptr(cost, C.c_double))
        return lab, cost

    def put_state(self, lab, cost):
        lab = _f32(lab); cost = np.ascontiguousarray(cost, dtype=np.float64)
        lib().lo_put_state(self.h, _ptr(lab, C.c_float), _ptr(cost, C.c_double))

    def set_labels(self, lab):
        lab = _f32(lab)
        lib().lo_set_labels(self.h, _ptr(lab, C.c_float))

    def set_proposals(self, abc):
        """Proposal map (H, W, 3) of plane labels for the k_cnn map candidates; None clears it."""
        if abc is None:
            lib().lo_set_proposals(self.h, None)
            return
        self._prop = _f32(abc).reshape(self.H, self.W, 3)
        lib().lo_set_proposals(self.h, _ptr(self._prop, C.c_float))

    def expand_cells(self, it, level, cells):
        """Algorithm 2 on the listed cells (i, j) of one group; returns (switched, evals)."""
        arr = np.ascontiguousarray(np.asarray(cells, np.int32).reshape(-1, 2))
        ev = C.c_longlong()
        acc = lib().lo_expand_cells(self.h, it, level, _ptr(arr, C.c_int), arr.shape[0], C.byref(ev))
        return acc, ev.value

    def expand_group(self, it, level, group):
        ev = C.c_longlong()
        acc = lib().lo_expand_group(self.h, it, level, group, C.byref(ev))
        return acc, ev.value

    def visit_candidates(self, lab, it, level, ci, cj):
        """Every candidate of the visit of cell (ci, cj), drawn from `lab` with no move in
        between (Algorithm 2 with the outer perturbation sizes of iteration `it`)."""
        lab = _f32(lab)
        n = lib().lo_visit_candidates(self.h, _ptr(lab, C.c_float), it, level, ci, cj, None)
        out = np.empty((n, 3), np.float32)
        lib().lo_visit_candidates(self.h, _ptr(lab, C.c_float), it, level, ci, cj, _ptr(out, C.c_float))
        return out

    def iterate(self, it):
        ev = C.c_longlong()
        acc = lib().lo_iterate(self.h, it, C.byref(ev))
        return acc, ev.value


# --- free functions -----------------------------------------------------------

def maxflow(w, h, tcap, ncap, method="dinic"):
    """(flow, cut) for the region grid graph; cut[p] = 1 iff p reaches the sink."""
    tcap = np.ascontiguousarray(tcap, dtype=np.int32)
    ncap = np.ascontiguousarray(ncap, dtype=np.int32)
    cut = np.zeros(w * h, np.uint8)
    f = {"dinic": lib().lo_maxflow_dinic, "ek": lib().lo_maxflow_ek, "enum": lib().lo_mincut_enum}[method]
    flow = f(w, h, _ptr(tcap, C.c_int32), _ptr(ncap, C.c_int32), _ptr(cut, C.c_uint8))
    return flow, cut.reshape(h, w)


def splitmix64(state: int, n: int):
    st = C.c_uint64(state)
    return [lib().lo_splitmix64_next(C.byref(st)) for _ in range(n)]


def proposal_stream(seed, it, level, ci, cj, proposal):
    return lib().lo_proposal_stream(seed, it, level, ci, cj, proposal)


def init_label(seed, W, u, v, dmin, dmax):
    out = np.empty(3, np.float32)
    lib().lo_init_label(seed, W, u, v, dmin, dmax, _ptr(out, C.c_float))
    return out


def propose(lab, stream, cell, perturb, rd, rn, dmin, dmax):
    lab = _f32(lab)
    H, W = lab.shape[:2]
    out = np.empty(3, np.float32)
    cx0, cy0, cw, ch = cell
    lib().lo_propose(_ptr(lab, C.c_float), W, stream, cx0, cy0, cw, ch, int(perturb), rd, rn, dmin, dmax,
                     _ptr(out, C.c_float))
    return out


def propose_map(prop, stream, cell):
    """Map candidate: the proposal map's label at a pixel drawn from the centre cell."""
    prop = _f32(prop)
    W = prop.shape[1]
    out = np.empty(3, np.float32)
    cx0, cy0, cw, ch = cell
    lib().lo_propose_map(_ptr(prop, C.c_float), W, stream, cx0, cy0, cw, ch, _ptr(out, C.c_float))
    return out


def propose_ransac(lab, stream, cell):
    """RANSAC candidate: a plane fitted to the disparities of the centre cell's labels."""
    lab = _f32(lab)
    W = lab.shape[1]
    out = np.empty(3, np.float32)
    cx0, cy0, cw, ch = cell
    lib().lo_propose_ransac(_ptr(lab, C.c_float), W, stream, cx0, cy0, cw, ch, _ptr(out, C.c_float))
    return out


def region_of(H, W, s, ci, cj):
    R = (C.c_int * 4)(); Cc = (C.c_int * 4)()
    lib().lo_region_of(H, W, s, ci, cj, R, Cc)
    return tuple(R), tuple(Cc)


def group_cells(H, W, s, group):
    n = lib().lo_group_cells(H, W, s, group, None)
    out = np.zeros((max(n, 1), 2), np.int32)
    lib().lo_group_cells(H, W, s, group, out.ctypes.data_as(C.POINTER(C.c_int)))
    return out[:n]


def openmp_threads():
    return lib().lo_openmp_threads()
