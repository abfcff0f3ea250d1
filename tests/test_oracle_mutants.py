"""The oracle's pins catch plausible mistakes.  Each case plants one mistake in a copy of
`oracle/lem_oracle.c` (a wrong sign, a dropped term, transposed operands, a wrong
normalisation, a wrong seed set of the cut, a missing halving, a loose threshold),
compiles it apart, and runs the pins of `tests/test_oracle_pins.py` against that copy in
a child process: some pin must fail.
The oracle itself is not changed; mistakes are only ever planted in these copies."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "lem_oracle.c")

# (name, text in lem_oracle.c, replacement): every occurrence is replaced
MUTANTS = [
    ("warp adds the disparity", "double up = su - d;", "double up = su + d;"),
    ("gradient term dropped from the raw cost",
     "return (1.0 - pa) * fmin(col, c->p.tau_col) + pa * fmin(gd, c->p.tau_grad);",
     "return (1.0 - pa) * fmin(col, c->p.tau_col);"),
    ("plane slopes transposed", "double d = a * su + b * sv + cc;", "double d = a * sv + b * su + cc;"),
    ("interpolation weights swapped", "double rv = (1.0 - t) * r0[ch] + t * r1[ch];",
     "double rv = t * r0[ch] + (1.0 - t) * r1[ch];"),
    ("guided-filter offset b_k with the wrong sign", "bk -= ai * mu[i];", "bk += ai * mu[i];"),
    ("window mean normalised by one pixel too many", "mr /= n;", "mr /= n + 1;"),
    ("smoothness term one-sided",
     "return fabs(disp_at(fp, pu, pv) - disp_at(fq, pu, pv)) + fabs(disp_at(fq, qu, qv) - disp_at(fp, qu, qv));",
     "return fabs(disp_at(fp, pu, pv) - disp_at(fq, pu, pv));"),
    ("smoothness term not truncated", "fmin(lo_psibar(pu, pv, qu, qv, fp, fq), c->p.tau_dis)",
     "lo_psibar(pu, pv, qu, qv, fp, fq)"),
    ("cut side seeded from every node", "if (res_t[i] > 0) {", "if (res_t[i] >= 0) {"),
    ("colour and gradient truncations swapped",
     "return (1.0 - pa) * fmin(col, c->p.tau_col) + pa * fmin(gd, c->p.tau_grad);",
     "return (1.0 - pa) * fmin(col, c->p.tau_grad) + pa * fmin(gd, c->p.tau_col);"),
    ("colour distance L2 instead of L1", "        col += fabs(l[ch] - rv);", "        col += (l[ch] - rv) * (l[ch] - rv);"),
    ("match clamped half a pixel inside the right border", "    if (up > W - 1) up = W - 1;\n",
     "    if (up > W - 1) up = W - 1.5;\n"),
    ("smoothness term evaluated at p on both sides",
     "return fabs(disp_at(fp, pu, pv) - disp_at(fq, pu, pv)) + fabs(disp_at(fq, qu, qv) - disp_at(fp, qu, qv));",
     "return fabs(disp_at(fp, pu, pv) - disp_at(fq, pu, pv)) + fabs(disp_at(fq, pu, pv) - disp_at(fp, pu, pv));"),
    ("contrast weight inside the truncation", "    return wv * fmin(lo_psibar(pu, pv, qu, qv, fp, fq), c->p.tau_dis);",
     "    return fmin(wv * lo_psibar(pu, pv, qu, qv, fp, fq), c->p.tau_dis);"),
    ("contrast weight of the L2 colour distance",
     "double l1 = fabs(lp[0] - lq[0]) + fabs(lp[1] - lq[1]) + fabs(lp[2] - lq[2]);",
     "double l1 = sqrt((lp[0] - lq[0]) * (lp[0] - lq[0]) + (lp[1] - lq[1]) * (lp[1] - lq[1]) + "
     "(lp[2] - lq[2]) * (lp[2] - lq[2]));"),
    ("regulariser on the 0..255 scale", "S[4 * i] += c->p.gf_eps;", "S[4 * i] += c->p.gf_eps * 255.0;"),
    ("sample covariance of the guide", "for (int i = 0; i < 9; i++) S[i] /= n;",
     "for (int i = 0; i < 9; i++) S[i] /= n - 1;"),
    ("regulariser added to a row instead of the diagonal", "S[4 * i] += c->p.gf_eps;", "S[i] += c->p.gf_eps;"),
    ("contrast weight without its floor", "if (w < c->p.eps_w) w = c->p.eps_w;", ""),
    ("LE-BF window of radius r'", "const int H = c->H, W = c->W, R = 2 * c->p.gf_radius;",
     "const int H = c->H, W = c->W, R = c->p.gf_radius;"),
    ("LE-BF weight of the squared colour distance", "exp(-l1 / c->p.bf_gamma)", "exp(-l1 * l1 / c->p.bf_gamma)"),
    ("energy without the diagonal pairs", "if (qx < 0 || qx >= W || qy >= H) continue;",
     "if (qx < 0 || qx >= W || qy >= H || d == 1 || d == 3) continue;"),
    ("energy without lambda", "double ps = lam * lo_psi(", "double ps = lo_psi("),
    ("quantisation truncates", "return (int64_t)nearbyint(S * x);", "return (int64_t)(S * x);"),
    ("pair above B + C not lowered", "if (A > B + C) {", "if (0) {"),
    ("initial plane with the printed sign", "double cc = ((n[0] * u + n[1] * v) + n[2] * z0) / n[2];",
     "double cc = -((n[0] * u + n[1] * v) + n[2] * z0) / n[2];"),
    ("visit draws from the expansion region", "lo_propose(lab, W, stream, C[0], C[1], C[2], C[3], perturb,",
     "lo_propose(lab, W, stream, R[0], R[1], R[2], R[3], perturb,"),
    ("perturbation size not halved within a visit", "            *rd *= 0.5;\n            *rn *= 0.5;\n", ""),
    ("perturbation size not halved per iteration", "double f = ldexp(1.0, -iter);", "double f = 1.0;"),
    ("perturbation with a flipped normal", "double n[3] = {-a / len, -b / len, 1.0 / len};",
     "double n[3] = {a / len, b / len, 1.0 / len};"),
    ("perturbed disparity not clamped to the range", "    if (dp < dmin) dp = dmin;\n    if (dp > dmax) dp = dmax;\n",
     ""),
    ("RANSAC hypothesis slopes swapped", "const double a = (double)na / den, b = (double)nb / den;",
     "const double a = (double)nb / den, b = (double)na / den;"),
    ("RANSAC inlier band of 2 px", "const int ok = fabs(r) <= 1.0;", "const int ok = fabs(r) <= 2.0;"),
    ("RANSAC without the least-squares refinement", "#define RANSAC_LO 2", "#define RANSAC_LO 0"),
    ("groups by (i div 4, j mod 4)", "const int gi = group % 4, gj = group / 4;",
     "const int gi = group / 4, gj = group % 4;"),
    ("region one cell short on the left", "int x0 = imax(0, (ci - 1) * s), x1 = imin(W, (ci + 2) * s);",
     "int x0 = imax(0, ci * s), x1 = imin(W, (ci + 2) * s);"),
    ("switched pixels keep their old cost", "            c->cost[p] = phiA[i];\n", ""),
    ("region scheme without the product of means in the covariance", "cov[ch] = s[1 + ch] / n - mu[ch] * mr;",
     "cov[ch] = s[1 + ch] / n;"),
    ("output window means normalised by the unclipped window", "double n = (double)(kx1 - kx0 + 1) * (ky1 - ky0 + 1);",
     "double n = (double)(2 * r + 1) * (2 * r + 1);"),
    ("Dinic without the reverse residual", "                g.cap[stack_e[k] ^ 1] += b;\n", ""),
    ("graph edge p->q built as q->p", "if (ncap[i * 4 + d] > 0) fg_add(g, i, jy * w + jx, ncap[i * 4 + d]);",
     "if (ncap[i * 4 + d] > 0) fg_add(g, jy * w + jx, i, ncap[i * 4 + d]);"),
    ("initial disparities ignore d_min", "double z0 = dmin + (dmax - dmin) * sm_u01(&st);",
     "double z0 = dmax * sm_u01(&st);"),
    ("perturbed disparity clamped at 0 instead of d_min", "    if (dp < dmin) dp = dmin;\n",
     "    if (dp < 0.0) dp = 0.0;\n"),
    ("outer perturbation size d_max / 2", "*rd = 0.5 * (c->p.disp_max - c->p.disp_min) * f;",
     "*rd = 0.5 * c->p.disp_max * f;"),
    ("x-gradient without the 1/2", "o[3] = 0.5 * (g[xp] - g[xm]);", "o[3] = g[xp] - g[xm];"),
    ("gray weights of R and B swapped", "g[x] = 0.299 * c[0] + 0.587 * c[1] + 0.114 * c[2];",
     "g[x] = 0.114 * c[0] + 0.587 * c[1] + 0.299 * c[2];"),
    ("pair term C - A credited as B - A", "U1[i] += C - A;", "U1[i] += B - A;"),
    ("pair weight read at the wrong node", "int bu = fwd ? pu : qu, bv = fwd ? pv : qv;", "int bu = pu, bv = pv;"),
    ("fixed neighbour folded with alpha on both sides",
     "double pa = lam * wv * fmin(lo_psibar(pu, pv, qu, qv, alpha, fq), c->p.tau_dis);",
     "double pa = lam * wv * fmin(lo_psibar(pu, pv, qu, qv, alpha, alpha), c->p.tau_dis);"),
    ("map candidates drawn before the RANSAC ones",
     "if (t >= kp && t < kp + kr) {\n            lo_propose_ransac",
     "if (t >= kp + kc && t < kp + kc + kr) {\n            lo_propose_ransac"),
]


def _pins_against(so, first_failure):
    """Runs the pins of tests/test_oracle_pins.py in a child process that loads the
    oracle library `so`; returns (exit code, end of its output)."""
    env = dict(os.environ, LEM_ORACLE_LIB=str(so), OMP_NUM_THREADS="2")
    cmd = [sys.executable, "-m", "pytest", os.path.join(ROOT, "tests", "test_oracle_pins.py"), "-q",
           "-p", "no:cacheprovider", "-m", "not gpu"] + (["-x"] if first_failure else [])
    out = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    return out.returncode, out.stdout[-1500:]


def _compile(src_text, d):
    c = os.path.join(d, "lem_oracle_copy.c")
    so = os.path.join(d, "liblem_oracle_copy.so")
    with open(c, "w") as f:
        f.write(src_text)
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fopenmp", c, "-o", so,
                    "-lm"], check=True)
    return so


@pytest.fixture(scope="module")
def c_mutant_runs(tmp_path_factory):
    """Every planted copy (and one unmodified copy, name None) compiled and checked
    against the pins, several at a time."""
    import tempfile
    from concurrent.futures import ThreadPoolExecutor
    src = open(SRC).read()
    # one base directory made here; the workers make theirs with tempfile, which is
    # safe across threads (pytest's factory is not)
    base = str(tmp_path_factory.mktemp("mutants"))

    def run(case):
        name, old, new = case
        d = tempfile.mkdtemp(dir=base)
        if name is None:
            return name, _pins_against(_compile(src, d), first_failure=False)
        if src.count(old) < 1:
            return name, (None, f"mutation site not found: {old}")
        return name, _pins_against(_compile(src.replace(old, new), d), first_failure=True)

    cases = [(None, None, None)] + MUTANTS
    with ThreadPoolExecutor(max_workers=max(1, min(8, (os.cpu_count() or 2) // 2))) as pool:
        return dict(pool.map(run, cases))


@pytest.mark.parametrize("name", [m[0] for m in MUTANTS])
def test_pins_catch_planted_mistake(c_mutant_runs, name):
    rc, tail = c_mutant_runs[name]
    assert rc is not None, tail
    assert rc != 0, f"no pin caught the mistake '{name}':\n{tail}"


def test_unmodified_copy_passes(c_mutant_runs):
    """Control: the same procedure on an unmodified copy passes every pin."""
    rc, tail = c_mutant_runs[None]
    assert rc == 0, tail


# the Python parts of the oracle: (name, module file, text, replacement, pin file)
PY_MUTANTS = [
    ("convolution instead of correlation", "cnn.py", "y += xp[i:i + H, j:j + W] @ w[i, j]",
     "y += xp[i:i + H, j:j + W] @ w[2 - i, 2 - j]", "test_oracle_cnn.py"),
    ("input gradient without the flip", "cnn.py", "dx += dyp[2 - i:2 - i + H, 2 - j:2 - j + W] @ w[i, j].T",
     "dx += dyp[i:i + H, j:j + W] @ w[i, j].T", "test_oracle_cnn.py"),
    ("weight gradient with a flipped window", "cnn.py", "dw[i, j] = xp[i:i + H, j:j + W]",
     "dw[i, j] = xp[2 - i:2 - i + H, 2 - j:2 - j + W]", "test_oracle_cnn.py"),
    ("bfloat16 ties rounded away from zero", "cnn.py",
     "up = (rest > 0x8000) | ((rest == 0x8000) & ((keep & 1) == 1))", "up = rest >= 0x8000", "test_oracle_cnn.py"),
    ("quarter-grid centre off by half a pixel", "cnn.py", "fv = min(max((vv - 1.5) / 4.0, 0.0), H4 - 1.0)",
     "fv = min(max((vv - 2.0) / 4.0, 0.0), H4 - 1.0)", "test_oracle_cnn.py"),
    ("target slopes not clamped", "cnn.py", "t[..., 1:] = np.clip(t[..., 1:], -1.0, 1.0)", "pass",
     "test_oracle_cnn.py"),
    ("Adam without the bias correction of the first moment", "cnn.py", "mh = m / (1.0 - b1 ** step)", "mh = m",
     "test_oracle_cnn.py"),
    ("Adam with eps inside the square root", "cnn.py", "(np.sqrt(vh) + eps)", "np.sqrt(vh + eps)",
     "test_oracle_cnn.py"),
    ("mirrored plane offset with the wrong sign", "postproc.py", "out = np.stack([-a, b, c + a * (W - 1)], axis=-1)",
     "out = np.stack([-a, b, c - a * (W - 1)], axis=-1)", "test_oracle_post.py"),
    ("consistency match on the wrong side", "postproc.py", "q = np.rint(u - dL)", "q = np.rint(u + dL)",
     "test_oracle_post.py"),
    ("filling from the foreground", "postproc.py", "out[y, x] = min(cands)", "out[y, x] = max(cands)",
     "test_oracle_post.py"),
    ("weighted-median window one row short", "postproc.py",
     "y0, y1 = max(0, y - radius), min(H, y + radius + 1)", "y0, y1 = max(0, y - radius), min(H, y + radius)",
     "test_oracle_post.py"),
    ("consistency match rounded down", "postproc.py", "q = np.rint(u - dL)", "q = np.floor(u - dL)",
     "test_oracle_post.py"),
    ("filling searches to the left only", "postproc.py", "for step in (-1, 1):", "for step in (-1,):",
     "test_oracle_post.py"),
    ("L1 loss not averaged over pixels", "cnn.py", "loss = float((np.abs(diff) * scale).sum() / n)",
     "loss = float((np.abs(diff) * scale).sum())", "test_oracle_cnn.py"),
    ("weighted median one element too far", "postproc.py", "k = int(np.searchsorted(cw, 0.5 * cw[-1]))",
     "k = int(np.searchsorted(cw, 0.5 * cw[-1], side='right'))", "test_oracle_post.py"),
    # (a mistake in the band sizes would leave the gloo ranks waiting for each other, so
    # the exchange's content is mutated, not its size)
    ("exchange sends only the centre cells' changes", "stripes.py",
     "changed[R[1]:R[1] + R[3], R[0]:R[0] + R[2]] = True",
     "changed[cj * s:min(H, cj * s + s), ci * s:min(W, ci * s + s)] = True", "test_stripes.py"),
    ("boundary cells owned by two stripes", "stripes.py", "if top <= j * s < bot", "if top <= j * s <= bot",
     "test_stripes.py"),
]


def _python_mutant(d, module, old, new, pins):
    """Copies the oracle package into directory d with one mistake planted in `module` and
    runs the pin file `pins` against the copy in a child process; (exit code, output end),
    or (None, reason) when the mutation site is missing."""
    import shutil
    pkg = os.path.join(d, "oracle")
    shutil.copytree(os.path.join(ROOT, "oracle"), pkg, ignore=shutil.ignore_patterns("*.so", "__pycache__", "*.tmp*"))
    path = os.path.join(pkg, module)
    with open(path) as f:
        text = f.read()
    if text.count(old) != 1:
        return None, f"mutation site not found once: {old}"
    with open(path, "w") as f:
        f.write(text.replace(old, new))
    # the child starts in d, so `import oracle` finds the planted copy first
    env = dict(os.environ, PYTHONPATH=os.pathsep.join([d, ROOT]), OMP_NUM_THREADS="2")
    env.pop("LEM_ORACLE_LIB", None)
    out = subprocess.run([sys.executable, "-m", "pytest", os.path.join(ROOT, "tests", pins), "-x", "-q",
                          "-p", "no:cacheprovider", "-m", "not gpu"], cwd=d, env=env,
                         capture_output=True, text=True, timeout=600)
    return out.returncode, out.stdout[-1500:]


@pytest.fixture(scope="module")
def py_mutant_runs(tmp_path_factory):
    """The planted copies of the network and post-processing references, several at a time
    (the stripe-decomposed driver's start gloo ranks and run one at a time in their test)."""
    import tempfile
    from concurrent.futures import ThreadPoolExecutor
    base = str(tmp_path_factory.mktemp("py_mutants"))
    cases = [m for m in PY_MUTANTS if m[1] != "stripes.py"]

    def run(case):
        name, module, old, new, pins = case
        return name, _python_mutant(tempfile.mkdtemp(dir=base), module, old, new, pins)

    with ThreadPoolExecutor(max_workers=max(1, min(8, (os.cpu_count() or 2) // 2))) as pool:
        return dict(pool.map(run, cases))


@pytest.mark.parametrize("name,module,old,new,pins", PY_MUTANTS, ids=[m[0] for m in PY_MUTANTS])
def test_python_pins_catch_planted_mistake(py_mutant_runs, tmp_path, name, module, old, new, pins):
    if module == "stripes.py":
        rc, tail = _python_mutant(str(tmp_path), module, old, new, pins)
    else:
        rc, tail = py_mutant_runs[name]
    assert rc is not None, tail
    assert rc != 0, f"no pin caught the mistake '{name}':\n{tail}"


def test_python_unmodified_copy_passes(tmp_path):
    """Control for the Python parts: an unmodified copy of the package passes their pins."""
    import shutil
    shutil.copytree(os.path.join(ROOT, "oracle"), tmp_path / "oracle",
                    ignore=shutil.ignore_patterns("*.so", "__pycache__", "*.tmp*"))
    env = dict(os.environ, PYTHONPATH=os.pathsep.join([str(tmp_path), ROOT]))
    env.pop("LEM_ORACLE_LIB", None)
    for pins in ("test_oracle_cnn.py", "test_oracle_post.py"):
        out = subprocess.run([sys.executable, "-m", "pytest", os.path.join(ROOT, "tests", pins), "-q",
                              "-p", "no:cacheprovider", "-m", "not gpu",
                              "-W", "ignore::pytest.PytestAssertRewriteWarning"], cwd=str(tmp_path), env=env,
                             capture_output=True, text=True, timeout=600)
        assert out.returncode == 0, out.stdout[-1500:]
