"""The C-ABI library builds, loads and exports every symbol include/lem.h declares;
argument checks that need no GPU return the documented status codes."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_1603_08328_gb300 import build as b
    b.build()
    from paper_1603_08328_gb300 import lem
    return lem


def _declared():
    src = open(os.path.join(ROOT, "include", "lem.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lem_[a-z_0-9]+)\s*\(", src)))


def test_header_symbols_are_exported(L):
    names = _declared()
    assert len(names) >= 14
    lib = L.lib()
    for n in names:
        assert hasattr(lib, n), n
        assert hasattr(L, n), f"binding lacks {n}"


def test_struct_sizes_match_header(L):
    # lem_params / lem_stats layouts are mirrored by the binding; a size check
    # against the C compiler's view catches a dropped or reordered field
    import subprocess
    import tempfile
    code = '#include "lem.h"\n#include <stdio.h>\nint main(){printf("%zu %zu %zu %zu\\n", sizeof(lem_params), ' \
           'sizeof(lem_stats), sizeof(lem_image), sizeof(lem_region));return 0;}\n'
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "s.c")
        open(src, "w").write(code)
        exe = os.path.join(d, "s")
        subprocess.run(["gcc", "-I" + os.path.join(ROOT, "include"), src, "-o", exe], check=True)
        sizes = [int(x) for x in subprocess.run([exe], capture_output=True, text=True).stdout.split()]
    assert sizes == [C.sizeof(L.lem_params), C.sizeof(L.lem_stats), C.sizeof(L.lem_image), C.sizeof(L.lem_region)]


def test_default_params_are_the_papers(L):
    p = L.lem_default_params()
    assert (p.gf_radius, p.gf_eps, p.tau_col, p.tau_grad, p.alpha_grad) == (10, 1e-4, 10.0, 2.0, 0.9)
    assert (p.lam, p.tau_dis, p.eps_w, p.gamma) == (1.0, 1.0, 0.01, 10.0)
    assert list(p.cell) == [5, 15, 25] and list(p.k_prop) == [1, 2, 2] and list(p.k_rand) == [7, 0, 0]


def test_create_rejects_bad_arguments_without_touching_the_gpu(L):
    lib = L.lib()
    a = np.zeros((32, 40, 3), np.uint8)
    b = np.zeros((32, 41, 3), np.uint8)
    im_a = L.lem_image(a.ctypes.data, 32, 40, 120, 0)
    im_b = L.lem_image(b.ctypes.data, 32, 41, 123, 0)
    p = L.lem_default_params(gf_radius=2)
    h = C.c_void_p()
    assert lib.lem_create(None, C.byref(im_a), C.byref(p), C.byref(h)) == L.LEM_ERR_ARG
    assert lib.lem_create(C.byref(im_a), C.byref(im_b), C.byref(p), C.byref(h)) == L.LEM_ERR_SHAPE
    assert "differ" in L.lem_last_error(None)
    bad = L.lem_default_params(gf_radius=2, cell=(1025, 15, 25))     # above LEM_MAX_CELL
    assert lib.lem_create(C.byref(im_a), C.byref(im_a), C.byref(bad), C.byref(h)) == L.LEM_ERR_ARG
    bad = L.lem_default_params(gf_radius=2, data_term=2)
    assert lib.lem_create(C.byref(im_a), C.byref(im_a), C.byref(bad), C.byref(h)) == L.LEM_ERR_ARG
    bad = L.lem_default_params(gf_radius=2, data_term=1, bf_gamma=0.0)
    assert lib.lem_create(C.byref(im_a), C.byref(im_a), C.byref(bad), C.byref(h)) == L.LEM_ERR_ARG
    bad = L.lem_default_params(gf_radius=2, threads=100)
    assert lib.lem_create(C.byref(im_a), C.byref(im_a), C.byref(bad), C.byref(h)) == L.LEM_ERR_ARG
    bad = L.lem_default_params(gf_radius=2, disp_min=5.0, disp_max=1.0)
    assert lib.lem_create(C.byref(im_a), C.byref(im_a), C.byref(bad), C.byref(h)) == L.LEM_ERR_ARG
    short = L.lem_image(a.ctypes.data, 32, 40, 100, 0)
    assert lib.lem_create(C.byref(short), C.byref(short), C.byref(p), C.byref(h)) == L.LEM_ERR_SHAPE
    assert not h.value
    im_c = L.lem_image(a.ctypes.data, 32, 40, 120, 0)
    assert lib.lem_create_batch(C.byref(im_c), C.byref(im_c), 0, C.byref(p), C.byref(h)) == L.LEM_ERR_ARG
    assert lib.lem_pair_count(None) == -1
    # NULL handles
    assert lib.lem_expand_iteration(None, 1, None) == L.LEM_ERR_ARG
    assert lib.lem_destroy(None) == L.LEM_OK
    assert lib.lem_evals_per_iteration(None) == -1


def test_v3_settings(L):
    """Sec. 4, Middlebury V3: cells of 1, 3 and 9 % of the image width, lambda = 0.5,
    K_RANS = 1; the other fields stay as they were."""
    p = L.lem_default_params(v3_width=1500)
    assert list(p.cell) == [15, 45, 135] and p.lam == 0.5 and list(p.k_rans) == [1, 1, 1]
    assert p.gf_radius == 10 and list(p.k_prop) == [1, 2, 2] and list(p.k_rand) == [7, 0, 0]
    p = L.lem_default_params(v3_width=2872, disp_max=300.0)
    assert list(p.cell) == [29, 86, 258] and p.disp_max == 300.0
    assert list(L.lem_default_params(v3_width=10).cell) == [1, 1, 1]      # rounded, at least 1 px
    assert L.lib().lem_v3_params(None, 100) == L.LEM_ERR_ARG
    with pytest.raises(L.LemError):
        L.lem_default_params(v3_width=0)


def test_parameter_checks_of_the_later_options(L):
    """Argument checks that run before any GPU work: launch shape, cluster visits,
    candidates per visit, proposer counts and strip rows."""
    lib = L.lib()
    a = np.zeros((32, 40, 3), np.uint8)
    im = L.lem_image(a.ctypes.data, 32, 40, 120, 0)
    h = C.c_void_p()
    bad = [dict(level_threads=(96, 0, 0)), dict(cluster_visits=2), dict(candidates_per_visit=9),
           dict(candidates_per_visit=0), dict(k_cnn=(65, 0, 0)), dict(k_rans=(0, 65, 0)), dict(strip_rows=6),
           dict(level_strip_rows=(0, 68, 0)), dict(level_gr_interval=(-1, 0, 0)), dict(cell=(0, 15, 25)),
           dict(quant_scale=0.0), dict(store_dtype=3), dict(max_rounds=0), dict(threads=1056)]
    for kw in bad:
        p = L.lem_default_params(gf_radius=2, **kw)
        assert lib.lem_create(C.byref(im), C.byref(im), C.byref(p), C.byref(h)) == L.LEM_ERR_ARG, kw
        assert not h.value


def test_image_layout_checks_without_touching_the_gpu(L):
    """lem_image's element type, channel count, pixel stride and alignment are checked
    before any GPU work: an unknown dtype, 2 or 17 channels and a float pointer or stride
    that is not a multiple of 4 bytes are LEM_ERR_ARG; a pixel stride shorter than its
    channels or a row stride shorter than the row is LEM_ERR_SHAPE; dataflow must be 0/1."""
    lib = L.lib()
    a = np.zeros((32, 40, 4), np.float32)
    base = a.ctypes.data
    p = L.lem_default_params(gf_radius=2)
    h = C.c_void_p()

    def rc(im, prm=p):
        return lib.lem_create(C.byref(im), C.byref(im), C.byref(prm), C.byref(h))

    f32 = L.LEM_IMG_F32
    assert rc(L.lem_image(base, 32, 40, 640, 0, 4, 16, 7)) == L.LEM_ERR_ARG           # dtype
    assert rc(L.lem_image(base, 32, 40, 640, 0, 2, 16, f32)) == L.LEM_ERR_ARG         # channels
    assert rc(L.lem_image(base, 32, 40, 640, 0, 17, 16, f32)) == L.LEM_ERR_ARG
    assert rc(L.lem_image(base + 2, 32, 40, 640, 0, 4, 16, f32)) == L.LEM_ERR_ARG     # alignment
    assert rc(L.lem_image(base, 32, 40, 642, 0, 4, 16, f32)) == L.LEM_ERR_ARG
    assert rc(L.lem_image(base, 32, 40, 640, 0, 4, 12, f32)) == L.LEM_ERR_SHAPE       # stride_px < 4 ch
    assert rc(L.lem_image(base, 32, 40, 620, 0, 4, 16, f32)) == L.LEM_ERR_SHAPE       # stride_row < row
    assert "stride_row" in L.lem_last_error(None)
    assert rc(L.lem_image(base, 32, 40, 640, 0, 4, 16, f32), L.lem_default_params(gf_radius=2, dataflow=2)) \
        == L.LEM_ERR_ARG
    # one regression window (2 r' + 1 = 5 pixels) is the smallest image side
    assert rc(L.lem_image(base, 4, 40, 640, 0, 4, 16, f32)) == L.LEM_ERR_SHAPE
    assert rc(L.lem_image(base, 32, 4, 640, 0, 4, 16, f32)) == L.LEM_ERR_SHAPE
    assert not h.value


def test_c_example_compiles_and_links(L):
    """tests/c_example.c (the usage example the README shows) is valid C99 against
    include/lem.h and links with the in-tree liblem.so (compiled and linked only:
    running it needs a GPU)."""
    import subprocess
    import tempfile
    src = os.path.join(ROOT, "tests", "c_example.c")
    libdir = os.path.dirname(L.LIB_PATH)
    with tempfile.TemporaryDirectory() as d:
        out = subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-I" + os.path.join(ROOT, "include"),
                              src, "-o", os.path.join(d, "example"), "-L" + libdir, "-llem",
                              "-Wl,-rpath," + libdir], capture_output=True, text=True)
        assert out.returncode == 0, out.stderr
