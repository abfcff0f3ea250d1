"""The oracle's pins catch plausible mistakes.  Each case plants one mistake in a copy of
`oracle/lem_oracle.c` (a wrong sign, a dropped term, transposed operands, a wrong
normalisation, a wrong seed set of the cut), compiles it apart, and runs the pins of
`tests/test_oracle_pins.py` against that copy in a child process: some pin must fail.
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
]


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_planted_mistake(tmp_path, name, old, new):
    src = open(SRC).read()
    assert src.count(old) >= 1, f"mutation site not found: {old}"
    mutant = tmp_path / "lem_oracle_mutant.c"
    mutant.write_text(src.replace(old, new))
    so = tmp_path / "liblem_oracle_mutant.so"
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fopenmp", str(mutant),
                    "-o", str(so), "-lm"], check=True)
    env = dict(os.environ, LEM_ORACLE_LIB=str(so))
    out = subprocess.run([sys.executable, "-m", "pytest", os.path.join(ROOT, "tests", "test_oracle_pins.py"), "-x",
                          "-q", "-p", "no:cacheprovider", "-m", "not gpu"], cwd=ROOT, env=env,
                         capture_output=True, text=True, timeout=600)
    assert out.returncode != 0, f"no pin caught the mistake '{name}':\n{out.stdout[-1500:]}"


def test_unmodified_copy_passes(tmp_path):
    """Control: the same procedure on an unmodified copy passes every pin."""
    so = tmp_path / "liblem_oracle_copy.so"
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fopenmp", SRC, "-o",
                    str(so), "-lm"], check=True)
    env = dict(os.environ, LEM_ORACLE_LIB=str(so))
    out = subprocess.run([sys.executable, "-m", "pytest", os.path.join(ROOT, "tests", "test_oracle_pins.py"), "-q",
                          "-p", "no:cacheprovider", "-m", "not gpu"], cwd=ROOT, env=env, capture_output=True,
                         text=True, timeout=600)
    assert out.returncode == 0, out.stdout[-1500:]


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
    ("mirrored plane offset with the wrong sign", "postproc.py", "out = np.stack([-a, b, c + a * (W - 1)], axis=-1)",
     "out = np.stack([-a, b, c - a * (W - 1)], axis=-1)", "test_oracle_post.py"),
    ("consistency match on the wrong side", "postproc.py", "q = np.rint(u - dL)", "q = np.rint(u + dL)",
     "test_oracle_post.py"),
    ("filling from the foreground", "postproc.py", "out[y, x] = min(cands)", "out[y, x] = max(cands)",
     "test_oracle_post.py"),
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


@pytest.mark.parametrize("name,module,old,new,pins", PY_MUTANTS, ids=[m[0] for m in PY_MUTANTS])
def test_python_pins_catch_planted_mistake(tmp_path, name, module, old, new, pins):
    import shutil
    pkg = tmp_path / "oracle"
    shutil.copytree(os.path.join(ROOT, "oracle"), pkg,
                    ignore=shutil.ignore_patterns("*.so", "__pycache__", "*.tmp*"))
    path = pkg / module
    text = path.read_text()
    assert text.count(old) == 1, f"mutation site not found: {old}"
    path.write_text(text.replace(old, new))
    # the child starts in tmp_path, so `import oracle` finds the planted copy first
    env = dict(os.environ, PYTHONPATH=os.pathsep.join([str(tmp_path), ROOT]))
    env.pop("LEM_ORACLE_LIB", None)
    out = subprocess.run([sys.executable, "-m", "pytest", os.path.join(ROOT, "tests", pins), "-x", "-q",
                          "-p", "no:cacheprovider", "-m", "not gpu"], cwd=str(tmp_path), env=env,
                         capture_output=True, text=True, timeout=600)
    assert out.returncode != 0, f"no pin caught the mistake '{name}':\n{out.stdout[-1500:]}"


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
