"""The C-ABI library without a GPU: it loads, exports every symbol that
include/gf2.h declares, and its host-side checks and planner behave.

No call here launches device work (argument checks run before any CUDA call).
"""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

import paper_0811_1714_gb300 as g

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gf2.h")


@pytest.fixture(scope="module")
def lib():
    g.build()
    return g.lib()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(gf2_[a-z0-9_]+)\s*\(", text)
    return sorted(set(names))


def test_header_and_binding_agree():
    assert sorted(g.EXPORTS) == declared_functions()


CITATION = re.compile(r"Sections? \d|Algorithms? \d|Tables? \d|no counterpart")


def test_every_declaration_cites_its_passage():
    """Each entry point's comment block (the nearest one above it) names the
    passage of the paper it restates -- a Section, Algorithm or Table -- or
    says that the paper has no counterpart."""
    text = open(HEADER).read()
    missing = []
    for mt in re.finditer(r"^[A-Za-z_].*?\b(gf2_[a-z0-9_]+)\s*\(", text, flags=re.M):
        name = mt.group(1)
        before = text[:mt.start()]
        end = before.rfind("*/")
        start = before.rfind("/*", 0, end)
        block = before[start:end] if start >= 0 and end >= 0 else ""
        block = re.sub(r"\s*\n\s*\*?\s*", " ", block)     # one line, comment stars dropped
        if not CITATION.search(block):
            missing.append(name)
    assert not missing, "declarations without a cited passage: %s" % missing
    assert len(set(re.findall(r"^[A-Za-z_].*?\b(gf2_[a-z0-9_]+)\s*\(", text, flags=re.M))) == \
        len(declared_functions())


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", g.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\s[TW]\s+(gf2_[a-z0-9_]+)$", out, flags=re.M))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    for n in declared_functions():
        getattr(lib, n)


def test_strerror_and_defaults(lib):
    for code in range(0, -9, -1):
        assert g.gf2_strerror(code)
    o = g.Opts()
    lib.gf2_default_opts(ctypes.byref(o))
    assert (o.base, o.depth, o.k, o.t, o.accumulate) == (g.GF2_BASE_AUTO, -1, 0, 0, 0)


def host_mat(rows, cols, stride=None):
    w = (cols + 63) // 64
    stride = stride if stride is not None else w + (w & 1)
    arr = np.zeros((rows, max(stride, 1)), np.uint64)
    return arr, g.mat(arr, cols)


def rc_of(fn, *args):
    with pytest.raises(g.GF2Error) as e:
        fn(*args)
    return e.value.status


def test_argument_checks(lib):
    a, A = host_mat(10, 70)
    b, B = host_mat(70, 90)
    c, C = host_mat(10, 90)
    # inner dimensions differ
    b2, B2 = host_mat(71, 90)
    assert rc_of(g.gf2_mul, C, A, B2) == g.GF2_EINVAL
    # C has the wrong shape
    c2, C2 = host_mat(11, 90)
    assert rc_of(g.gf2_mul, C2, A, B) == g.GF2_EINVAL
    # stride below ceil(cols / 64)
    s = np.zeros((10, 1), np.uint64)
    bad = g.mat(s, 70)
    assert rc_of(g.gf2_mul, C, bad, B) == g.GF2_ELAYOUT
    # odd stride
    s3 = np.zeros((10, 3), np.uint64)
    assert rc_of(g.gf2_mul, C, g.mat(s3, 70), B) == g.GF2_ELAYOUT
    # null data with a non-empty shape
    N = g.Mat()
    N.rows, N.cols, N.stride_words, N.device = 10, 70, 2, -1
    assert rc_of(g.gf2_mul, C, N, B) == g.GF2_EINVAL
    # C aliases A
    big = np.zeros((20, 2), np.uint64)
    Aal = g.mat(big, 70)
    Cal = g.mat(big, 90)
    Aal.rows = 10
    Cal.rows = 10
    sq, SQ = host_mat(70, 90)
    assert rc_of(g.gf2_mul, Cal, Aal, SQ) == g.GF2_EALIAS
    # bad options
    assert rc_of(g.gf2_mul, C, A, B, g.opts(base=7)) == g.GF2_EINVAL
    assert rc_of(g.gf2_mul, C, A, B, g.opts(base=g.GF2_BASE_TC_FP4 + 1)) == g.GF2_EINVAL
    assert rc_of(g.gf2_mul, C, A, B, g.opts(depth=-2)) == g.GF2_EINVAL
    assert rc_of(g.gf2_mul, C, A, B, g.opts(k=3, t=3)) == g.GF2_EUNSUPPORTED
    o = g.opts()
    o.reserved[1] = 1
    assert rc_of(g.gf2_mul, C, A, B, o) == g.GF2_EINVAL
    assert rc_of(g.gf2_mul, C, A, B, g.opts(peel=2)) == g.GF2_EINVAL


def test_plan_with_peeling(lib):
    """Peeling (Section 4): the recursion runs on the largest core whose rows
    are a multiple of 2^d and whose columns are multiples of 128 * 2^d."""
    p = g.gf2_describe_plan(20000, 12000, 28000, g.opts(depth=2, base=g.GF2_BASE_M4RM, peel=1))
    assert "peel core=20000x11776x27648" in p and "padded=20000x11776x27648" in p, p
    assert "leftover rows=0 cols=352 k=224" in p, p
    # sizes that already halve evenly: nothing to peel
    q = g.gf2_describe_plan(4096, 4096, 4096, g.opts(depth=2, peel=1))
    assert "peel" not in q and "depth=2" in q
    # no core at this depth: the product runs as requested without peeling
    r = g.gf2_describe_plan(300, 100, 300, g.opts(depth=1, peel=1))
    assert "peel" not in r


def test_plan_padding_and_scratch(lib):
    # Strassen-Winograd pads rows to 2^d and columns to 128 * 2^d (virtual zeros)
    p = g.gf2_describe_plan(20000, 12000, 28000, g.opts(depth=2, base=g.GF2_BASE_M4RM))
    assert "depth=2" in p and "padded=20000x12288x28160" in p and "leaves=49" in p
    p0 = g.gf2_describe_plan(1024, 1024, 1024, g.opts(depth=0))
    assert "depth=0" in p0 and "scratch=0" in p0
    assert g.gf2_scratch_bytes(1024, 1024, 1024, g.opts(depth=0)) == 0
    # scratch of one level: 7 A-operands, 7 B-operands, 7 products, each a quadrant
    q = 7 * (512 * 512 // 64) * 8
    assert g.gf2_scratch_bytes(1024, 1024, 1024, g.opts(depth=1, base=g.GF2_BASE_M4RM)) == 3 * q
    # the automatic depth recurses while the sub-problems stay >= 4096
    assert "depth=3" in g.gf2_describe_plan(32768, 32768, 32768)
    assert "depth=0" in g.gf2_describe_plan(4096, 4096, 4096)


def test_plan_uses_the_cubic_product_for_narrow_right_factors(lib):
    """Section 2.3: at most 64 columns of B take the cubic packed product
    (B's columns as rows, 64 of them, in scratch)."""
    p = g.gf2_describe_plan(5000, 3000, 40, g.opts(base=g.GF2_BASE_M4RM, depth=0))
    assert "cubic=1" in p, p
    assert g.gf2_scratch_bytes(5000, 3000, 40, g.opts(base=g.GF2_BASE_M4RM, depth=0)) == 64 * 48 * 8
    assert "cubic" not in g.gf2_describe_plan(5000, 3000, 65, g.opts(base=g.GF2_BASE_M4RM, depth=0))
    # an explicit table shape keeps the Four Russians
    assert "cubic" not in g.gf2_describe_plan(5000, 3000, 40, g.opts(base=g.GF2_BASE_M4RM, depth=0, k=8, t=4))


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    monkeypatch.setattr(g, "_lib", None)
    monkeypatch.setattr(g, "LIB_PATH", str(tmp_path / "absent.so"))
    with pytest.raises(g.LibraryNotBuilt):
        g.lib()


def test_build_makes_the_peak_probe_program(lib):
    """build() also compiles the throughput probes behind the roofline peaks
    into an executable beside the library (run only by the GPU tests and
    `bench.py --workload peaks`)."""
    from paper_0811_1714_gb300 import buildlib
    exe = buildlib.probe_path("peaks")
    assert os.path.isfile(exe) and os.access(exe, os.X_OK)
