"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks an oracle function against something other than itself: a
closed form, an invariant stated in the paper, a textbook routine written
independently here (integral-image guided filter, ridge regression), a library
routine (scipy max-flow) or brute force on tiny inputs.
"""
import os

import numpy as np
import pytest

import oracle
from tests.conftest import TINY_PARAMS

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --- random draws -------------------------------------------------------------

def test_splitmix64_published_outputs():
    """SplitMix64 (Steele et al. 2014) from state 0: the published first outputs."""
    vals = [int(l, 16) for l in open(os.path.join(GOLDEN, "splitmix64_seed0.txt")) if l.startswith("0x")]
    assert oracle.splitmix64(0, len(vals)) == vals


# --- preprocessing --------------------------------------------------------------

def _gray_ramp(H, W, k):
    # R = G = B so the BT.601 gray value equals the channel value
    u = np.arange(W, dtype=np.float64)
    img = np.repeat((20.0 + k * u)[None, :, None], 3, axis=2)
    return np.repeat(img, H, axis=0)


def test_gradient_kernel_on_ramp():
    """[-0.5 0 0.5] on a ramp of slope k: k inside, k/2 at the replicated border (Sec. 3.2)."""
    H, W, k = 6, 12, 3.5
    img = _gray_ramp(H, W, k)
    o = oracle.Oracle(img, img, gf_radius=1)
    g = o.planes()["L"][..., 3]
    assert np.allclose(g[:, 1:-1], k, atol=1e-12)
    assert np.allclose(g[:, [0, -1]], k / 2, atol=1e-12)


def test_guide_stats_against_numpy(tiny_pair):
    """mu_k and (Sigma_k + eU)^-1 over the clipped window, vs numpy mean/cov/inv."""
    r = 2
    o = oracle.Oracle(tiny_pair["left"], tiny_pair["right"], gf_radius=r)
    pl = o.planes()
    I = tiny_pair["left"].astype(np.float64) / 255.0
    H, W = I.shape[:2]
    for (y, x) in [(0, 0), (5, 7), (71, 95), (30, 0), (40, 60)]:
        win = I[max(0, y - r):y + r + 1, max(0, x - r):x + r + 1].reshape(-1, 3)
        mu = win.mean(0)
        S = np.cov(win.T, bias=True) + 1e-4 * np.eye(3)
        assert np.allclose(pl["mu"][y, x], mu, rtol=0, atol=1e-14)
        assert np.allclose(pl["A"][y, x], np.linalg.inv(S), rtol=1e-9)


def test_contrast_weight_closed_form():
    """w_pq = exp(-|I_p - I_q|_1 / gamma) with the lower bound eps (Eq. smweight)."""
    H, W = 4, 5
    img = np.full((H, W, 3), 100.0)
    img[:, 3:, :] += np.array([4.0, 3.0, 2.0])   # step of L1 = 9 between columns 2 and 3
    img[2:, :, 0] += 60.0                          # step of 60 between rows 1 and 2 (weight floor)
    o = oracle.Oracle(img, img, gf_radius=1, gamma=10.0, eps_w=0.01)
    w = o.planes()["w"]
    assert w[0, 0, 0] == pytest.approx(1.0)                 # flat
    assert w[0, 2, 0] == pytest.approx(np.exp(-0.9))        # right across the colour step
    assert w[1, 0, 2] == pytest.approx(0.01)                # down across the 60 step: exp(-6) < eps
    assert w[0, 4, 0] == 0.0                                # right neighbour outside the image


# --- raw cost rho ---------------------------------------------------------------

def test_rho_zero_for_integer_fronto_parallel_shift(tiny_pair):
    """Noise-free right view = left shifted by an integer d: rho(s|(0,0,d)) = 0 exactly."""
    L = tiny_pair["left"].astype(np.float64)
    d = 6
    R = np.empty_like(L)
    R[:, :-d] = L[:, d:]
    R[:, -d:] = L[:, -1:]
    o = oracle.Oracle(L, R, gf_radius=2)
    H, W = L.shape[:2]
    for v in range(0, H, 7):
        for u in range(d + 1, W - 1, 5):
            assert o.rho((0, 0, d), u, v) == 0.0


def test_rho_zero_on_slanted_plane_with_affine_texture():
    """Slanted plane, texture affine in u with constant gray: the exact right view gives rho = 0."""
    H, W = 20, 64
    a, b, c = 0.12, -0.05, 9.0
    rng = np.random.default_rng(3)
    base = rng.uniform(60, 160, size=(H, 1, 3))
    # per-row colour slopes whose BT.601 gray slope is zero, so both gradients vanish
    sR = rng.uniform(-1, 1, size=(H, 1))
    sB = rng.uniform(-1, 1, size=(H, 1))
    sG = -(0.299 * sR + 0.114 * sB) / 0.587
    slope = np.concatenate([sR, sG, sB], axis=1)[:, None, :]
    u = np.arange(W, dtype=np.float64)[None, :, None]
    L = base + slope * u
    v = np.arange(H, dtype=np.float64)[:, None, None]
    ul = (u + b * v + c) / (1.0 - a)           # left position seen by right pixel u
    R = base + slope * ul
    o = oracle.Oracle(L, R, gf_radius=2)
    for vv in range(H):
        for uu in range(W):
            up = uu - (a * uu + b * vv + c)
            if 0.0 <= up <= W - 1:
                assert abs(o.rho(np.float32([a, b, c]), uu, vv)) < 1e-5   # labels are float32
    # with the float32-rounded label the residual is the label rounding only
    lab = np.float32([a, b, c])
    o2 = oracle.Oracle(L, base + slope * ((u + float(lab[1]) * v + float(lab[2])) / (1.0 - float(lab[0]))),
                       gf_radius=2)
    assert max(abs(o2.rho(lab, uu, 10)) for uu in range(W // 2, W)) < 1e-10


def test_rho_bounded_by_linear_interpolation_error():
    """Smooth sinusoid, non-integer shift: rho <= the linear-interpolation error bound h^2/8 max|f''|."""
    H, W = 3, 80
    A, om, ph = 40.0, 0.3, 0.4
    delta = 3.37
    u = np.arange(W, dtype=np.float64)
    f = lambda x: 120.0 + A * np.sin(om * x + ph)
    L = np.repeat(np.repeat(f(u)[None, :, None], 3, axis=2), H, axis=0)
    R = np.repeat(np.repeat(f(u + delta)[None, :, None], 3, axis=2), H, axis=0)
    o = oracle.Oracle(L, R, gf_radius=1)
    # colour: 3 channels, each |f - lerp f| <= A om^2 / 8; gradient: central difference
    # of a sinusoid is A sin(om) cos(.), whose lerp error is <= A om^2 sin(om) / 8
    bound = 0.1 * 3 * A * om ** 2 / 8 + 0.9 * A * om ** 2 * np.sin(om) / 8
    worst = max(o.rho((0, 0, delta), uu, 1) for uu in range(6, W - 2))
    assert worst <= bound + 1e-9
    assert worst > 0.05 * bound           # and the bound is not vacuous


# --- data term: guided-filter aggregation ---------------------------------------

def _box_mean(x, r):
    """Count-normalised box mean over (2r+1)^2 windows clipped to the image, by integral images."""
    H, W = x.shape[:2]
    ii = np.zeros((H + 1, W + 1) + x.shape[2:])
    ii[1:, 1:] = x.cumsum(0).cumsum(1)
    ys = np.arange(H); xs = np.arange(W)
    y0 = np.clip(ys - r, 0, H); y1 = np.clip(ys + r + 1, 0, H)
    x0 = np.clip(xs - r, 0, W); x1 = np.clip(xs + r + 1, 0, W)
    s = ii[y1][:, x1] - ii[y0][:, x1] - ii[y1][:, x0] + ii[y0][:, x0]
    n = (y1 - y0)[:, None] * (x1 - x0)[None, :]
    return s / n.reshape(n.shape + (1,) * (x.ndim - 2))


def _guided_filter(I, p, r, eps):
    """He et al. (TPAMI 2013) guided filter, colour guide, box means by integral images."""
    mI = _box_mean(I, r)
    mp = _box_mean(p, r)
    mIp = _box_mean(I * p[..., None], r)
    cov_Ip = mIp - mI * mp[..., None]
    II = I[..., :, None] * I[..., None, :]
    var = _box_mean(II.reshape(I.shape[:2] + (9,)), r).reshape(I.shape[:2] + (3, 3)) \
        - mI[..., :, None] * mI[..., None, :]
    a = np.linalg.solve(var + eps * np.eye(3), cov_Ip[..., None])[..., 0]
    b = mp - (a * mI).sum(-1)
    return (_box_mean(a, r) * I).sum(-1) + _box_mean(b[..., None], r)[..., 0]


@pytest.mark.parametrize("c", [4.0, 6.63])
def test_fronto_parallel_region_cost_is_cost_volume_filtering(tiny_pair, c):
    """alpha = (0,0,c): phi over a region equals the guided-filtered cost-volume slice."""
    r = 2
    o = oracle.Oracle(tiny_pair["left"], tiny_pair["right"], gf_radius=r)
    H, W = o.H, o.W
    slice_ = np.array([[o.rho((0, 0, c), u, v) for u in range(W)] for v in range(H)])
    I = tiny_pair["left"].astype(np.float64) / 255.0
    ref = _guided_filter(I, slice_, r, 1e-4)
    for (x0, y0, w, h) in [(0, 0, 15, 15), (40, 30, 15, 15), (81, 57, 15, 15), (20, 60, 9, 12)]:
        reg = o.region_cost(x0, y0, w, h, (0, 0, c))
        assert np.allclose(reg, ref[y0:y0 + h, x0:x0 + w], rtol=0, atol=1e-9)


def test_gf_coefficients_are_the_ridge_regression(tiny_pair):
    """a_k, b_k minimise sum_s (a.I_s + b - rho_s)^2 + e |W'_k| |a|^2 (He et al. 2013)."""
    r = 2
    o = oracle.Oracle(tiny_pair["left"], tiny_pair["right"], gf_radius=r)
    I = tiny_pair["left"].astype(np.float64) / 255.0
    lab = np.float32([0.07, -0.03, 5.2])
    for (kx, ky) in [(0, 0), (10, 10), (95, 71), (50, 3)]:
        xs = range(max(0, kx - r), min(o.W, kx + r + 1))
        ys = range(max(0, ky - r), min(o.H, ky + r + 1))
        X, y = [], []
        for v in ys:
            for u in xs:
                X.append([*I[v, u], 1.0])
                y.append(o.rho(lab, u, v))
        X = np.array(X); y = np.array(y); n = len(y)
        Pen = np.diag([1e-4 * n] * 3 + [0.0])
        sol = np.linalg.solve(X.T @ X + Pen, X.T @ y)
        assert np.allclose(o.gf_coeffs(lab, kx, ky), sol, rtol=1e-7, atol=1e-9)


def test_region_cost_equals_definition_brute_force(tiny_pair):
    """The region scheme over M reproduces phi_p(alpha) by definition at every p, borders included."""
    o = oracle.Oracle(tiny_pair["left"], tiny_pair["right"], gf_radius=2)
    lab = np.float32([0.05, 0.02, 8.4])
    for (x0, y0, w, h) in [(0, 0, 10, 10), (86, 62, 10, 10), (37, 21, 15, 15), (90, 0, 6, 4)]:
        reg = o.region_cost(x0, y0, w, h, lab)
        d = np.array([[o.phi_def(lab, x0 + x, y0 + y) for x in range(w)] for y in range(h)])
        assert np.abs(reg - d).max() < 1e-12


def test_definition_equals_explicit_weights_of_eq_gf(tiny_pair):
    """Interior p: phi_p = sum_s omega_ps rho(s) with omega from Eq. gf, and the weights sum to 1."""
    r = 2
    o = oracle.Oracle(tiny_pair["left"], tiny_pair["right"], gf_radius=r)
    lab = np.float32([-0.04, 0.06, 7.1])
    for (u, v) in [(20, 20), (50, 33), (80, 60)]:
        w = o.phi_weights(u, v)
        rho = np.array([[o.rho(lab, u + dx, v + dy) for dx in range(-2 * r, 2 * r + 1)]
                        for dy in range(-2 * r, 2 * r + 1)])
        assert w.sum() == pytest.approx(1.0, abs=1e-12)
        assert (w * rho).sum() == pytest.approx(o.phi_def(lab, u, v), abs=1e-12)


# --- smoothness term --------------------------------------------------------------

def _rand_label(rng):
    return np.float32([rng.uniform(-1, 1), rng.uniform(-1, 1), rng.uniform(-30, 60)])


def test_psi_lemma1_and_special_cases(tiny_pair):
    """Lemma 1 (psi(a,a) + psi(b,g) <= psi(b,a) + psi(a,g)), psi(f,f) = 0, and a=b=0 -> 2|c_p - c_q|."""
    o = oracle.Oracle(tiny_pair["left"], tiny_pair["right"], gf_radius=2, tau_dis=1e9, eps_w=1.0)
    o_t = oracle.Oracle(tiny_pair["left"], tiny_pair["right"], gf_radius=2)
    rng = np.random.default_rng(5)
    for _ in range(400):
        u, v, d = int(rng.integers(1, 90)), int(rng.integers(0, 70)), int(rng.integers(0, 4))
        al, be, ga = (_rand_label(rng) for _ in range(3))
        for oo in (o, o_t):
            lhs = oo.psi(u, v, d, al, al) + oo.psi(u, v, d, be, ga)
            rhs = oo.psi(u, v, d, be, al) + oo.psi(u, v, d, al, ga)
            assert lhs <= rhs + 1e-9
            assert oo.psi(u, v, d, be, be) == 0.0
        cp, cq = rng.uniform(0, 60, 2)
        # untruncated, unit weight: psi-bar = 2 |c_p - c_q|
        assert o.psi(u, v, d, (0, 0, cp), (0, 0, cq)) == pytest.approx(
            2 * abs(np.float32(cp) - np.float32(cq)), rel=1e-12)


# --- the binary move ---------------------------------------------------------------

def _random_state(o, rng, spread=0.6):
    H, W = o.H, o.W
    lab = np.empty((H, W, 3), np.float32)
    base = [_rand_label(rng) for _ in range(4)]
    for y in range(H):
        for x in range(W):
            f = base[rng.integers(0, 4)].astype(np.float64)
            f = f + rng.normal(0, [0.02, 0.02, spread])
            lab[y, x] = f
    return lab


def _smooth_state(o, rng):
    """Labels close to one plane: neighbouring pairs stay below the truncation tau_dis, so
    A, B and C of a pair differ (the random state truncates nearly every pair)."""
    H, W = o.H, o.W
    lab = np.empty((H, W, 3), np.float32)
    lab[..., 0] = 0.05 + rng.normal(0, 0.002, (H, W))
    lab[..., 1] = -0.03 + rng.normal(0, 0.002, (H, W))
    lab[..., 2] = 6.0 + rng.normal(0, 0.03, (H, W))
    return lab


@pytest.mark.parametrize("labels", ["rough", "smooth"])
def test_move_graph_encodes_the_energy_exactly(tiny_pair, labels):
    """|R| = 16: for all 2^16 moves x, const + cut(x) equals the quantised energy of f (+) x summed
    term by term from the definitions (phi by definition, psi of Eq. smooth_phi), except one unit
    less for each pair that was lowered to B + C (submodularity after rounding) and stays at (0,0).
    Rough labels truncate nearly every pair at tau_dis; smooth ones keep them below it, where the
    pair's A, B and C differ and the edge p->q carries B + C - A > 0."""
    o = oracle.Oracle(tiny_pair["left"], tiny_pair["right"], gf_radius=2)
    S, lam = 65536.0, o.p["lam"]
    rng = np.random.default_rng(9)
    lab = _random_state(o, rng) if labels == "rough" else _smooth_state(o, rng)
    x0, y0, w, h = 34, 24, 4, 4
    cost = np.zeros((o.H, o.W))
    for y in range(y0, y0 + h):
        for x in range(x0, x0 + w):
            cost[y, x] = o.phi_def(lab[y, x], x, y)
    alpha = lab[y0 + 1, x0 + 1].copy()
    alpha[2] += 0.3 if labels == "rough" else 0.1
    alpha[0] += 0.01 if labels == "rough" else 0.002
    phiA = np.array([[o.phi_def(alpha, x0 + x, y0 + y) for x in range(w)] for y in range(h)])
    g = o.build_graph(x0, y0, w, h, alpha, lab, cost, phiA)
    if labels == "smooth":
        assert (g["ncap"] > 0).sum() >= 30      # untruncated pairs with an edge of their own
    tcap, ncap = g["tcap"].reshape(-1, 2).astype(np.int64), g["ncap"].reshape(-1, 4).astype(np.int64)
    Q = lambda z: int(np.rint(S * z))
    fdx, fdy = [1, -1, 0, 1], [0, 1, 1, 1]
    n = w * h
    X = ((np.arange(1 << n)[:, None] >> np.arange(n)[None, :]) & 1).astype(np.int64)   # all moves
    idx = lambda x, y: (y - y0) * w + (x - x0)
    inR = lambda x, y: x0 <= x < x0 + w and y0 <= y < y0 + h
    # energy of f (+) x from the definitions, restricted to the terms that touch R
    E = np.zeros(1 << n, np.int64)
    for y in range(y0, y0 + h):
        for x in range(x0, x0 + w):
            i = idx(x, y)
            E += np.where(X[:, i] == 1, Q(phiA[y - y0, x - x0]), Q(cost[y, x]))
    for y in range(y0 - 1, y0 + h + 1):
        for x in range(x0 - 1, x0 + w + 1):
            for d in range(4):
                qx, qy = x + fdx[d], y + fdy[d]
                if not (inR(x, y) or inR(qx, qy)):
                    continue
                lp = [lab[y, x], alpha] if inR(x, y) else [lab[y, x], lab[y, x]]
                lq = [lab[qy, qx], alpha] if inR(qx, qy) else [lab[qy, qx], lab[qy, qx]]
                xp = X[:, idx(x, y)] if inR(x, y) else np.zeros(1 << n, np.int64)
                xq = X[:, idx(qx, qy)] if inR(qx, qy) else np.zeros(1 << n, np.int64)
                for bp in (0, 1):
                    for bq in (0, 1):
                        term = Q(lam * o.psi(x, y, d, lp[bp], lq[bq]))
                        E += np.where((xp == bp) & (xq == bq), term, 0)
    # cut of every move
    cut = np.where(X == 1, tcap[None, :, 0], tcap[None, :, 1]).sum(1)
    lowered = np.zeros(1 << n, np.int64)
    clamp = g["clamp_mask"].reshape(-1)
    for i in range(n):
        iy, ix = divmod(i, w)
        for d in range(4):
            jx, jy = ix + fdx[d], iy + fdy[d]
            if 0 <= jx < w and jy < h:
                j = jy * w + jx
                cut += np.where((X[:, i] == 0) & (X[:, j] == 1), ncap[i, d], 0)
                if (clamp[i] >> d) & 1:
                    lowered += (X[:, i] == 0) & (X[:, j] == 0)
    assert (g["const"] + cut == E - lowered).all()
    # and the min-cut solvers find the minimum of this energy
    f, c = oracle.maxflow(w, h, g["tcap"], g["ncap"], "dinic")
    assert f == cut.min()


def _random_grid(rng, w, h, cap=2000, tmax=5000):
    tcap = rng.integers(0, tmax, size=(h, w, 2)).astype(np.int32)
    tcap[rng.random((h, w)) < 0.5, 0] = 0
    tcap[tcap[..., 0] > 0, 1] = 0
    ncap = rng.integers(0, cap, size=(h, w, 4)).astype(np.int32)
    ncap[rng.random((h, w, 4)) < 0.3] = 0
    return tcap, ncap


@pytest.mark.parametrize("seed", range(12))
def test_mincut_small_exhaustive(seed):
    """<= 16 nodes: Dinic, Edmonds-Karp and enumeration agree on the value and the minimal cut."""
    rng = np.random.default_rng(seed)
    w, h = [(4, 4), (3, 5), (5, 3), (1, 16), (16, 1), (2, 2)][seed % 6]
    tcap, ncap = _random_grid(rng, w, h, cap=int(rng.integers(1, 3000)))
    f1, c1 = oracle.maxflow(w, h, tcap, ncap, "dinic")
    f2, c2 = oracle.maxflow(w, h, tcap, ncap, "ek")
    f3, c3 = oracle.maxflow(w, h, tcap, ncap, "enum")
    assert f1 == f2 == f3
    assert (c1 == c3).all() and (c2 == c3).all()


def _scipy_maxflow(w, h, tcap, ncap):
    sp = pytest.importorskip("scipy.sparse")
    csg = pytest.importorskip("scipy.sparse.csgraph")
    n = w * h
    rows, cols, caps = [], [], []
    fdx, fdy = [1, -1, 0, 1], [0, 1, 1, 1]
    for y in range(h):
        for x in range(w):
            i = y * w + x
            if tcap[y, x, 0]:
                rows.append(n); cols.append(i); caps.append(tcap[y, x, 0])
            if tcap[y, x, 1]:
                rows.append(i); cols.append(n + 1); caps.append(tcap[y, x, 1])
            for d in range(4):
                jx, jy = x + fdx[d], y + fdy[d]
                if 0 <= jx < w and jy < h and ncap[y, x, d]:
                    rows.append(i); cols.append(jy * w + jx); caps.append(ncap[y, x, d])
    m = sp.csr_matrix((np.array(caps, np.int32), (rows, cols)), shape=(n + 2, n + 2))
    return csg.maximum_flow(m, n, n + 1).flow_value


@pytest.mark.parametrize("w,h,seed", [(15, 15, 0), (45, 45, 1), (75, 75, 2), (33, 7, 3)])
def test_mincut_large_against_ek_and_scipy(w, h, seed):
    """Random grid graphs up to 75x75: Dinic = Edmonds-Karp (value and cut) = scipy max-flow value."""
    rng = np.random.default_rng(100 + seed)
    tcap, ncap = _random_grid(rng, w, h)
    f1, c1 = oracle.maxflow(w, h, tcap, ncap, "dinic")
    f2, c2 = oracle.maxflow(w, h, tcap, ncap, "ek")
    assert f1 == f2
    assert (c1 == c2).all()
    assert f1 == _scipy_maxflow(w, h, tcap, ncap)


# --- the method: Algorithms 1 and 2 -------------------------------------------------

def test_groups_are_disjoint_with_one_cell_gaps():
    """Eq. groupindex: the 16 groups partition the cells; regions of one group are separated by >= 1 cell."""
    for (H, W, s) in [(72, 96, 5), (375, 450, 15), (375, 450, 25), (40, 41, 5)]:
        nx, ny = -(-W // s), -(-H // s)
        seen = np.zeros((ny, nx), int)
        for g in range(16):
            cells = oracle.group_cells(H, W, s, g)
            for (i, j) in cells:
                seen[j, i] += 1
                assert 4 * (j % 4) + (i % 4) == g
            rects = [oracle.region_of(H, W, s, i, j)[0] for (i, j) in cells]
            for a in range(len(rects)):
                for b in range(a + 1, len(rects)):
                    (ax, ay, aw, ah), (bx, by, bw, bh) = rects[a], rects[b]
                    gapx = max(bx - (ax + aw), ax - (bx + bw))
                    gapy = max(by - (ay + ah), ay - (by + bh))
                    assert max(gapx, gapy) >= s
        assert (seen == 1).all()


def test_init_labels_pass_through_a_disparity_in_range():
    """Random init (Sec. 3.4): the plane passes through (u, v, z0), z0 in [dmin, dmax]."""
    for (u, v) in [(0, 0), (17, 3), (449, 374), (200, 100)]:
        f = oracle.init_label(7, 450, u, v, 0.0, 60.0).astype(np.float64)
        d = f[0] * u + f[1] * v + f[2]
        assert -1e-3 <= d <= 60.0 + 1e-3


def test_proposals_propagation_and_perturbation(tiny_pair):
    """Propagation returns the label of a pixel r of the centre cell (Algorithm 2); perturbation
    (Sec. 3.4) moves the disparity at r by at most r_d (then clamps it to the range) and tilts the
    normal by at most asin(r_n)."""
    rng = np.random.default_rng(2)
    o = oracle.Oracle(tiny_pair["left"], tiny_pair["right"], **TINY_PARAMS)
    lab = _random_state(o, rng)
    cell = (10, 15, 5, 5)
    where = {tuple(lab[y, x]): (x, y) for y in range(15, 20) for x in range(10, 15)}
    rd, rn = 2.0, 0.5
    for k in range(40):
        st = oracle.proposal_stream(11, 0, 0, 2, 3, k)
        a = oracle.propose(lab, st, cell, 0, 0, 0, 0.0, 15.0)
        assert tuple(a) in where
        x, y = where[tuple(a)]            # the same stream draws the same pixel first
        b = oracle.propose(lab, st, cell, 1, rd, rn, 0.0, 15.0).astype(np.float64)
        a = a.astype(np.float64)
        d0 = a[0] * x + a[1] * y + a[2]
        d1 = b[0] * x + b[1] * y + b[2]
        lo, hi = min(max(d0 - rd, 0.0), 15.0), min(max(d0 + rd, 0.0), 15.0)
        assert lo - 1e-3 <= d1 <= hi + 1e-3
        n0 = np.array([-a[0], -a[1], 1.0]); n0 /= np.linalg.norm(n0)
        n1 = np.array([-b[0], -b[1], 1.0]); n1 /= np.linalg.norm(n1)
        ang = np.arccos(np.clip(abs(n0 @ n1), -1, 1))
        assert ang <= np.arcsin(rn) + 1e-4


def test_energy_never_increases_and_group_order_is_irrelevant(tiny_pair):
    """Subproblem optimality (Sec. 3.3): E never increases over the moves of Algorithm 1;
    independence (Lemma 3): reversing the order of the regions of a group changes nothing."""
    kw = dict(TINY_PARAMS)
    o1 = oracle.Oracle(tiny_pair["left"], tiny_pair["right"], **kw)
    o2 = oracle.Oracle(tiny_pair["left"], tiny_pair["right"], reverse_order=1, n_threads=1,
                       **{k: v for k, v in kw.items()})
    o1.init_state(); o2.init_state()
    e_prev, q_prev = o1.energy()
    for it in range(2):
        for g in range(16):
            o1.expand_group(it, 0, g)
            o2.expand_group(it, 0, g)
            e, q = o1.energy()
            assert q <= q_prev
            assert e <= e_prev + 1e-9
            e_prev, q_prev = e, q
    l1, c1 = o1.state(); l2, c2 = o2.state()
    assert (l1 == l2).all() and (c1 == c2).all()


def test_cost_cache_matches_definition_after_moves(tiny_pair):
    """The cached phi_p(f_p) equals phi_p by definition for the current labels."""
    o = oracle.Oracle(tiny_pair["left"], tiny_pair["right"], **TINY_PARAMS)
    o.init_state()
    o.iterate(0)
    lab, cost = o.state()
    rng = np.random.default_rng(0)
    for _ in range(60):
        y, x = int(rng.integers(0, o.H)), int(rng.integers(0, o.W))
        assert cost[y, x] == pytest.approx(o.phi_def(lab[y, x], x, y), abs=1e-11)


def test_method_recovers_ground_truth_disparity(tiny_pair):
    """After 4 iterations on the tiny scene most pixels are within 1 px of the rendered disparity."""
    o = oracle.Oracle(tiny_pair["left"], tiny_pair["right"], **TINY_PARAMS)
    o.init_state()
    for it in range(4):
        o.iterate(it)
    lab, _ = o.state()
    v, u = np.mgrid[0:o.H, 0:o.W]
    d = lab[..., 0] * u + lab[..., 1] * v + lab[..., 2]
    assert (np.abs(d - tiny_pair["disp"]) > 1.0).mean() < 0.2


def test_batched_visits_are_exact_moves(tiny_pair):
    """Batched schedule (candidates of a visit drawn from the visit-start labels): every move
    is still an exact expansion, so the energy never increases and the cost cache stays exact;
    with visit = 1 it is Algorithm 2 as printed (bit-identical to the default)."""
    kw = dict(TINY_PARAMS)
    o4 = oracle.Oracle(tiny_pair["left"], tiny_pair["right"], visit=4, **kw)
    o1 = oracle.Oracle(tiny_pair["left"], tiny_pair["right"], visit=1, **kw)
    o0 = oracle.Oracle(tiny_pair["left"], tiny_pair["right"], **kw)
    for o in (o4, o1, o0):
        o.init_state()
    q_prev = o4.energy()[1]
    for g in range(16):
        o4.expand_group(0, 0, g)
        q = o4.energy()[1]
        assert q <= q_prev
        q_prev = q
    o1.iterate(0)
    o0.iterate(0)
    l1, c1 = o1.state(); l0, c0 = o0.state()
    assert (l1 == l0).all() and (c1 == c0).all()
    lab, cost = o4.state()
    rng = np.random.default_rng(1)
    for _ in range(30):
        y, x = int(rng.integers(0, o4.H)), int(rng.integers(0, o4.W))
        assert cost[y, x] == pytest.approx(o4.phi_def(lab[y, x], x, y), abs=1e-11)


def test_map_proposals_draw_the_propagation_pixel(tiny_pair):
    """A map candidate is the proposal map's label at a pixel r of the centre cell, drawn
    exactly as the propagation proposal draws r; a constant map gives its constant."""
    rng = np.random.default_rng(5)
    o = oracle.Oracle(tiny_pair["left"], tiny_pair["right"], **TINY_PARAMS)
    M = _random_state(o, rng)
    const = np.broadcast_to(np.float32([0.25, -0.5, 7.0]), M.shape)
    cell = (20, 10, 5, 5)
    for k in range(30):
        st = oracle.proposal_stream(11, 1, 0, 4, 2, k)
        assert (oracle.propose_map(M, st, cell) == oracle.propose(M, st, cell, 0, 0, 0, 0.0, 15.0)).all()
        assert (oracle.propose_map(const, st, cell) == np.float32([0.25, -0.5, 7.0])).all()


def test_map_proposals_are_exact_moves_and_help(tiny_pair):
    """Map candidates sit between propagation and perturbation: every move stays an exact
    expansion (energy never increases), a cleared map reproduces k_cnn = 0 bit for bit, and a
    map of the true disparities (fronto-parallel planes) beats one iteration without it."""
    kw = dict(TINY_PARAMS)
    gt = tiny_pair["disp"].astype(np.float32)
    gt_map = np.stack([np.zeros_like(gt), np.zeros_like(gt), gt], axis=-1)
    om = oracle.Oracle(tiny_pair["left"], tiny_pair["right"], k_cnn=(2,), **kw)
    oc = oracle.Oracle(tiny_pair["left"], tiny_pair["right"], k_cnn=(2,), **kw)
    o0 = oracle.Oracle(tiny_pair["left"], tiny_pair["right"], **kw)
    for o in (om, oc, o0):
        o.init_state()
    om.set_proposals(gt_map)
    oc.set_proposals(gt_map)
    oc.set_proposals(None)
    q_prev = om.energy()[1]
    for g in range(16):
        om.expand_group(0, 0, g)
        q = om.energy()[1]
        assert q <= q_prev
        q_prev = q
    oc.iterate(0)
    o0.iterate(0)
    lc, cc = oc.state(); l0, c0 = o0.state()
    assert (lc == l0).all() and (cc == c0).all()
    v, u = np.mgrid[0:om.H, 0:om.W]

    def bad(o):
        lab, _ = o.state()
        return (np.abs(lab[..., 0] * u + lab[..., 1] * v + lab[..., 2] - gt) > 1.0).mean()
    assert bad(om) < bad(o0) - 0.02
    assert om.energy()[1] < o0.energy()[1]


def _plane_labels(H, W, a, b, c):
    lab = np.empty((H, W, 3), np.float32)
    lab[..., 0], lab[..., 1], lab[..., 2] = a, b, c
    return lab


def test_ransac_recovers_a_plane_among_outliers():
    """Algorithm 2, RANSAC proposal (LO-RANSAC on the centre cell): labels of one plane, 30 % of
    them replaced by labels 5-20 px off it, give back that plane."""
    rng = np.random.default_rng(3)
    H, W = 40, 60
    a, b, c = 0.125, -0.0625, 17.5           # multiples of 2^-10: exact disparities
    lab = _plane_labels(H, W, a, b, c)
    mask = rng.random((H, W)) < 0.3
    off = rng.uniform(5, 20, size=(H, W)).astype(np.float32)
    lab[..., 2] = np.where(mask, lab[..., 2] + off, lab[..., 2])
    for k in range(20):
        st = oracle.proposal_stream(4, 0, 2, 1, 1, k)
        al = oracle.propose_ransac(lab, st, (25, 10, 25, 25))
        assert np.allclose(al, [a, b, c], rtol=0, atol=2e-6), al


def test_ransac_degenerate_cell_falls_back_to_a_drawn_label():
    """A one-pixel-wide cell has only collinear points: every hypothesis is void and the
    candidate is the label of the first drawn pixel (one of the cell's labels)."""
    rng = np.random.default_rng(4)
    lab = rng.normal(size=(10, 8, 3)).astype(np.float32)
    for k in range(10):
        al = oracle.propose_ransac(lab, oracle.proposal_stream(1, 0, 0, 0, 0, k), (3, 2, 1, 5))
        assert any((al == lab[y, 3]).all() for y in range(2, 7))


def test_ransac_candidates_are_exact_moves(tiny_pair):
    """K_RANS = 1 (between propagation and perturbation): every move is still an exact
    expansion, so the energy never increases, and the cost cache stays exact."""
    kw = dict(TINY_PARAMS, k_rans=(1,))
    o = oracle.Oracle(tiny_pair["left"], tiny_pair["right"], **kw)
    o.init_state()
    q_prev = o.energy()[1]
    for g in range(16):
        o.expand_group(0, 0, g)
        q = o.energy()[1]
        assert q <= q_prev
        q_prev = q
    lab, cost = o.state()
    rng = np.random.default_rng(2)
    for _ in range(20):
        y, x = int(rng.integers(0, o.H)), int(rng.integers(0, o.W))
        assert cost[y, x] == pytest.approx(o.phi_def(lab[y, x], x, y), abs=1e-11)


def test_le_bf_uniform_colours_give_the_plain_window_sum(tiny_pair):
    """LE-BF (Sec. 4): with one colour everywhere in the left view every bilateral weight is
    exp(0) = 1, so phi_p is the unnormalised sum of rho over the (4r'+1)^2 window clipped
    to the image; with a large gamma the weights of a textured view tend to 1 as well."""
    H, W = 20, 30
    L = np.full((H, W, 3), 120.0)
    rng = np.random.default_rng(9)
    R = rng.uniform(0, 255, size=(H, W, 3))
    o = oracle.Oracle(L, R, gf_radius=2, data_term=1)
    for (u, v) in [(0, 0), (15, 10), (29, 19), (4, 17)]:
        ref = sum(o.rho((0.1, 0.0, 3.2), su, sv) for sv in range(max(0, v - 4), min(H, v + 5))
                  for su in range(max(0, u - 4), min(W, u + 5)))
        assert o.phi_bf((0.1, 0.0, 3.2), u, v) == pytest.approx(ref, rel=1e-13)
    o2 = oracle.Oracle(tiny_pair["left"], tiny_pair["right"], gf_radius=2, data_term=1, bf_gamma=1e12)
    u, v = 40, 30
    ref = sum(o2.rho((0, 0, 5.0), su, sv) for sv in range(v - 4, v + 5) for su in range(u - 4, u + 5))
    assert o2.phi_bf((0, 0, 5.0), u, v) == pytest.approx(ref, rel=1e-9)


def test_le_bf_zero_at_an_integer_shift_and_region_dispatch(tiny_pair):
    """rho = 0 at the true fronto-parallel label of a noise-free shifted pair, so the
    LE-BF cost is 0 there; the region computation of LE-BF is the per-pixel definition."""
    L = tiny_pair["left"].astype(np.float64)
    d = 6
    R = np.empty_like(L)
    R[:, :-d] = L[:, d:]
    R[:, -d:] = L[:, -1:]
    o = oracle.Oracle(L, R, gf_radius=2, data_term=1)
    assert o.phi_bf((0, 0, d), 40, 30) == 0.0
    o3 = oracle.Oracle(tiny_pair["left"], tiny_pair["right"], gf_radius=2, data_term=1)
    reg = o3.region_cost(10, 20, 6, 4, (0.05, -0.02, 7.5))
    for y in range(4):
        for x in range(6):
            assert reg[y, x] == o3.phi_bf((0.05, -0.02, 7.5), 10 + x, 20 + y)


def test_le_bf_colour_step_weight():
    """A left view of two colours differing by (10, 20, 10), an L1 distance of 40: each
    window pixel on the other side of the step weighs exp(-40 / gamma) and each pixel on
    the same side 1 (an L2 distance, a 0..1 colour scale or a normalised sum would all
    give other values)."""
    H, W = 16, 24
    L = np.full((H, W, 3), 100.0)
    L[:, 12:] += (10.0, 20.0, 10.0)
    rng = np.random.default_rng(4)
    R = rng.uniform(0, 255, size=(H, W, 3))
    for gamma in (10.0, 25.0):
        o = oracle.Oracle(L, R, gf_radius=2, data_term=1, bf_gamma=gamma)
        f = (0.05, 0.02, 2.7)
        for (u, v) in [(10, 8), (13, 3), (11, 15)]:
            same = other = 0.0
            for sv in range(max(0, v - 4), min(H, v + 5)):
                for su in range(max(0, u - 4), min(W, u + 5)):
                    if (su >= 12) == (u >= 12):
                        same += o.rho(f, su, sv)
                    else:
                        other += o.rho(f, su, sv)
            assert other > 0
            ref = same + np.exp(-40.0 / gamma) * other
            assert o.phi_bf(f, u, v) == pytest.approx(ref, rel=1e-12)


# --- pins found missing by planting mistakes (tests/test_oracle_mutants.py) ---------

# forward neighbour offsets (each unordered 8-neighbour pair once) and their direction index
_FWD = {(1, 0): 0, (-1, 1): 1, (0, 1): 2, (1, 1): 3}


def test_energy_is_the_sum_of_its_terms(tiny_pair):
    """Eq. mrf with lambda = 2.5: E = sum_p phi_p(f_p) + lambda sum over unordered 8-neighbour
    pairs of psi_pq.  Here every pixel's 8 neighbours are visited and the sum halved (each pair
    seen from both ends, psi being symmetric in (p, f_p) <-> (q, f_q)); the quantised energy is
    sum Q(phi_p) + sum Q(lambda psi_pq), Q(x) = rne(S x)."""
    lam, S = 2.5, 65536.0
    left = np.ascontiguousarray(tiny_pair["left"][:30, :40])
    right = np.ascontiguousarray(tiny_pair["right"][:30, :40])
    o = oracle.Oracle(left, right, gf_radius=2, lam=lam, disp_max=15.0)
    rng = np.random.default_rng(8)
    lab = _random_state(o, rng)
    cost = rng.uniform(0.0, 3.0, size=(o.H, o.W))
    E, Eq = o.energy_of(lab, cost)
    H, W = o.H, o.W
    both = 0.0
    q = int(np.rint(S * cost).astype(np.int64).sum())
    for y in range(H):
        for x in range(W):
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    qx, qy = x + dx, y + dy
                    if (dx, dy) == (0, 0) or not (0 <= qx < W and 0 <= qy < H):
                        continue
                    if (dx, dy) in _FWD:
                        v = o.psi(x, y, _FWD[(dx, dy)], lab[y, x], lab[qy, qx])
                        q += int(np.rint(S * (lam * v)))
                    else:
                        v = o.psi(qx, qy, _FWD[(-dx, -dy)], lab[qy, qx], lab[y, x])
                    both += v
    assert E == pytest.approx(cost.sum() + lam * both / 2.0, rel=1e-12)
    assert Eq == q


def test_visit_candidates_follow_algorithms_1_and_2(tiny_pair):
    """The candidates of one visit at the 5 px level (K_prop = 1, K_rand = 7): the propagation
    proposal is the label f_r of a pixel r of the centre cell C_ij; the k-th perturbation
    (k = 0 .. 6) moves the disparity at its pixel r by at most r_d 2^-k (then clamps it to the
    range) and tilts the normal by at most asin(r_n 2^-k), where r_d = (d_max - d_min)/2 and
    r_n = 1 are halved after every outer iteration (Algorithm 1) and after every perturbation
    of the visit (Algorithm 2)."""
    o = oracle.Oracle(tiny_pair["left"], tiny_pair["right"], **TINY_PARAMS)
    H, W, s = o.H, o.W, 5
    rng = np.random.default_rng(12)
    lab = np.empty((H, W, 3), np.float32)
    lab[..., 0] = rng.uniform(-0.2, 0.2, (H, W))
    lab[..., 1] = rng.uniform(-0.2, 0.2, (H, W))
    v, u = np.mgrid[0:H, 0:W]
    lab[..., 2] = rng.uniform(2.0, 13.0, (H, W)) - lab[..., 0] * u - lab[..., 1] * v
    where = {tuple(lab[y, x]): (x, y) for y in range(H) for x in range(W)}
    assert len(where) == H * W
    for it in (0, 2):
        rd0, rn0 = 7.5 * 2.0 ** -it, 2.0 ** -it
        for (ci, cj) in [(3, 4), (0, 0), (19, 14), (10, 7), (6, 13)]:
            _, cell = oracle.region_of(H, W, s, ci, cj)
            cx0, cy0, cw, ch = cell
            cands = o.visit_candidates(lab, it, 0, ci, cj).astype(np.float64)
            assert cands.shape == (8, 3)
            x, y = where[tuple(np.float32(cands[0]))]
            assert cx0 <= x < cx0 + cw and cy0 <= y < cy0 + ch
            for k in range(7):
                st = oracle.proposal_stream(TINY_PARAMS["seed"], it, 0, ci, cj, 1 + k)
                f = oracle.propose(lab, st, cell, 0, 0.0, 0.0, 0.0, 15.0)   # the same stream's pixel r
                x, y = where[tuple(f)]
                f, b = f.astype(np.float64), cands[1 + k]
                rd, rn = rd0 * 2.0 ** -k, rn0 * 2.0 ** -k
                d0 = f[0] * x + f[1] * y + f[2]
                d1 = b[0] * x + b[1] * y + b[2]
                lo, hi = min(max(d0 - rd, 0.0), 15.0), min(max(d0 + rd, 0.0), 15.0)
                assert lo - 1e-3 <= d1 <= hi + 1e-3, (it, ci, cj, k)
                n0 = np.array([-f[0], -f[1], 1.0]); n0 /= np.linalg.norm(n0)
                n1 = np.array([-b[0], -b[1], 1.0]); n1 /= np.linalg.norm(n1)
                assert np.arccos(np.clip(abs(n0 @ n1), -1, 1)) <= np.arcsin(min(rn, 1.0)) + 1e-4


def test_ransac_refines_by_least_squares_on_inliers():
    """LO-RANSAC (Algorithm 2, RANSAC proposal; the least-squares refinement on the inliers
    within 1 px): 60 % of the cell's disparities lie on a plane with Gaussian noise of 0.2 px,
    20 % sit 2.5 px above it (no plane's 1 px band holds both groups) and 20 % 5-20 px off.  The
    refined plane is the least-squares fit of the noisy inliers: slopes within 6e-3 and the
    disparity at the cell centre within 0.06 px of the true plane in every trial, far closer
    than a plane through three noisy points, and unbiased by the points at 2.5 px."""
    rng = np.random.default_rng(6)
    H, W = 40, 60
    a, b, c = 0.125, -0.0625, 17.5
    lab = _plane_labels(H, W, a, b, c)
    kind = rng.random((H, W))
    off = np.where(kind < 0.6, rng.normal(0.0, 0.2, (H, W)),
                   np.where(kind < 0.8, 2.5 + rng.normal(0.0, 0.05, (H, W)), rng.uniform(5, 20, (H, W))))
    lab[..., 2] = lab[..., 2] + off.astype(np.float32)
    cell = (25, 10, 25, 25)
    uc, vc = 25 + 12, 10 + 12
    for k in range(20):
        al = oracle.propose_ransac(lab, oracle.proposal_stream(9, 0, 2, 1, 1, k), cell).astype(np.float64)
        assert abs(al[0] - a) <= 6e-3 and abs(al[1] - b) <= 6e-3, al
        assert abs((al[0] * uc + al[1] * vc + al[2]) - (a * uc + b * vc + c)) <= 0.06, al


def test_rounding_above_b_plus_c_is_lowered():
    """Lemma 1 makes psi(f_p, f_q) <= psi(f_p, alpha) + psi(alpha, f_q), but after rounding
    Q(A) can exceed Q(B) + Q(C) by one unit.  For fronto-parallel labels d1 < d_alpha < d2 the
    real terms are exactly additive; picking the gaps so the rounding goes up for A and down
    for B and C, the pair's A is lowered to B + C: the pair is counted as lowered and its edge
    capacity is 0, never negative."""
    img = np.full((8, 8, 3), 100, np.uint8)
    o = oracle.Oracle(img, img, gf_radius=1)
    S = 65536.0
    rng = np.random.default_rng(10)
    lab = np.zeros((8, 8, 3), np.float32)
    for _ in range(1000):
        d1 = np.float32(5.0)
        da = np.float32(d1 + rng.uniform(0.01, 0.2))
        d2 = np.float32(da + rng.uniform(0.01, 0.2))
        fp, fa, fq = (np.float32([0, 0, d]) for d in (d1, da, d2))
        A = np.rint(S * o.psi(3, 3, 0, fp, fq))
        B = np.rint(S * o.psi(3, 3, 0, fp, fa))
        C = np.rint(S * o.psi(3, 3, 0, fa, fq))
        if A > B + C:
            break
    else:
        pytest.fail("no rounding case found")
    lab[3, 3], lab[3, 4] = fp, fq
    g = o.build_graph(3, 3, 2, 1, fa, lab, np.zeros((8, 8)), np.zeros((1, 2)))
    assert g["nclamp"] == 1 and g["clamp_mask"][0, 0] == 1
    assert g["ncap"][0, 0, 0] == 0
    assert (g["ncap"] >= 0).all() and (g["tcap"] >= 0).all()


def test_visit_order_propagation_ransac_map_perturbation(tiny_pair):
    """Order of the proposals in a visit: K_prop propagation, K_RANS RANSAC, k_cnn map
    candidates, then K_rand perturbations with the size halved after each (Algorithm 2 with
    the RANSAC and map proposals in the candidate slots).  The visit's draw equals the
    single-proposal functions composed in that order, each with proposal index t's stream."""
    kw = dict(TINY_PARAMS, k_prop=(2,), k_rans=(1,), k_cnn=(2,), k_rand=(3,))
    o = oracle.Oracle(tiny_pair["left"], tiny_pair["right"], **kw)
    rng = np.random.default_rng(14)
    lab = _random_state(o, rng)
    prop = _random_state(o, rng)
    o.set_proposals(prop)
    H, W, s = o.H, o.W, 5
    for it in (0, 1):
        for (ci, cj) in [(2, 3), (19, 14), (7, 0)]:
            _, cell = oracle.region_of(H, W, s, ci, cj)
            got = o.visit_candidates(lab, it, 0, ci, cj)
            rd, rn = 7.5 * 2.0 ** -it, 2.0 ** -it
            want = []
            for t in range(8):
                st = oracle.proposal_stream(TINY_PARAMS["seed"], it, 0, ci, cj, t)
                if t < 2:
                    want.append(oracle.propose(lab, st, cell, 0, 0.0, 0.0, 0.0, 15.0))
                elif t < 3:
                    want.append(oracle.propose_ransac(lab, st, cell))
                elif t < 5:
                    want.append(oracle.propose_map(prop, st, cell))
                else:
                    want.append(oracle.propose(lab, st, cell, 1, rd, rn, 0.0, 15.0))
                    rd, rn = rd * 0.5, rn * 0.5
            assert (got == np.array(want)).all(), (it, ci, cj)


def test_disparity_range_with_a_nonzero_minimum(tiny_pair):
    """Disparity range [20, 60] (reading R20: the range is [d_min, d_max], r_d starts at
    (d_max - d_min)/2 = 20): the initial planes pass through disparities drawn over the whole
    range (Sec. 3.4), and every perturbed disparity stays within r_d 2^-k of its pixel's
    disparity and inside the range (R10), reaching d_min when labels sit just above it."""
    dmin, dmax = 20.0, 60.0
    d = []
    for k in range(3000):
        u, v = k % 96, k // 96
        f = oracle.init_label(5, 96, u, v, dmin, dmax).astype(np.float64)
        d.append(f[0] * u + f[1] * v + f[2])
    d = np.array(d)
    assert d.min() >= dmin - 1e-3 and d.max() <= dmax + 1e-3
    assert d.min() < dmin + 1.0 and d.max() > dmax - 1.0
    o = oracle.Oracle(tiny_pair["left"], tiny_pair["right"], **dict(TINY_PARAMS, disp_min=dmin, disp_max=dmax))
    H, W, s = o.H, o.W, 5
    rng = np.random.default_rng(13)
    lab = np.empty((H, W, 3), np.float32)
    lab[..., 0] = rng.uniform(-0.05, 0.05, (H, W))
    lab[..., 1] = rng.uniform(-0.05, 0.05, (H, W))
    v, u = np.mgrid[0:H, 0:W]
    lab[..., 2] = rng.uniform(20.5, 22.0, (H, W)) - lab[..., 0] * u - lab[..., 1] * v
    where = {tuple(lab[y, x]): (x, y) for y in range(H) for x in range(W)}
    at_min = 0
    for (ci, cj) in [(3, 4), (0, 0), (19, 14), (10, 7), (6, 13), (12, 2)]:
        _, cell = oracle.region_of(H, W, s, ci, cj)
        cands = o.visit_candidates(lab, 0, 0, ci, cj).astype(np.float64)
        for k in range(7):
            st = oracle.proposal_stream(TINY_PARAMS["seed"], 0, 0, ci, cj, 1 + k)
            f = oracle.propose(lab, st, cell, 0, 0.0, 0.0, dmin, dmax)
            x, y = where[tuple(f)]
            f, b = f.astype(np.float64), cands[1 + k]
            rd = 0.5 * (dmax - dmin) * 2.0 ** -k
            d0 = f[0] * x + f[1] * y + f[2]
            d1 = b[0] * x + b[1] * y + b[2]
            assert max(d0 - rd, dmin) - 1e-3 <= d1 <= min(d0 + rd, dmax) + 1e-3, (ci, cj, k, d0, d1)
            at_min += abs(d1 - dmin) < 1e-3
    assert at_min > 0


def test_rho_closed_forms_of_eq_photofunc():
    """Eq. photofunc on constructed pairs, right(u) = left(u + D) + offset + k u (all three
    channels): at the true disparity D the colour term is the L1 norm of the colour difference
    and the gradient term the ramp's slope k (the gray ramp's central difference), each
    truncated by its own threshold (tau_col = 10 on colour, tau_grad = 2 on gradient) and mixed
    (1 - alpha) : alpha = 0.1 : 0.9.  A match outside the right image is clamped to its first
    or last column (reading R6)."""
    rng = np.random.default_rng(21)
    H, W, D = 6, 40, 5
    base = rng.integers(20, 120, size=(H, W + D, 3))
    u_r = np.arange(W)[None, :, None]
    left = np.ascontiguousarray(base[:, :W].astype(np.uint8))

    def rho_at(offset, k):
        right = np.ascontiguousarray((base[:, D:W + D] + np.array(offset) + k * u_r).astype(np.uint8))
        o = oracle.Oracle(left, right, gf_radius=1, disp_max=20.0)
        lab = np.float32([0.0, 0.0, D])
        return [(u, o.rho(lab, u, 3)) for u in range(D + 1, W - 1)], o

    for (u, r) in rho_at((2, -1, 1), 0)[0]:
        assert r == pytest.approx(0.1 * 4.0, abs=1e-12)
    for (u, r) in rho_at((10, 10, 10), 0)[0]:
        assert r == pytest.approx(0.1 * 10.0, abs=1e-12)
    for (u, r) in rho_at((0, 0, 0), 1)[0]:
        assert r == pytest.approx(0.1 * min(3.0 * (u - D), 10.0) + 0.9 * 1.0, abs=1e-12)
    for (u, r) in rho_at((0, 0, 0), 3)[0]:
        assert r == pytest.approx(0.1 * min(9.0 * (u - D), 10.0) + 0.9 * 2.0, abs=1e-12)
    # clamping: a uniform left image; the right image equals it except in the columns next
    # to its first and last ones, so a match clamped anywhere but onto the edge column has
    # another cost
    left = np.full((H, W, 3), 100, np.uint8)
    right = left.copy()
    right[:, 1] = 120
    right[:, W - 2] = 120
    o = oracle.Oracle(left, right, gf_radius=1, disp_max=20.0)
    for u in (2, 17, 39):
        at_first = o.rho(np.float32([0, 0, u]), u, 2)              # u' = 0
        at_last = o.rho(np.float32([0, 0, u - (W - 1)]), u, 2)      # u' = W - 1
        assert at_first != o.rho(np.float32([0, 0, u - 0.5]), u, 2)
        assert at_last != o.rho(np.float32([0, 0, u - (W - 1.5)]), u, 2)
        for extra in (0.5, 7.0):
            assert o.rho(np.float32([0, 0, u + extra]), u, 2) == at_first
            assert o.rho(np.float32([0, 0, u - (W - 1) - extra]), u, 2) == at_last
