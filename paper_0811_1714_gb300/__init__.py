"""Python binding of libgf2, the GB300 library for dense matrix products over GF(2).

Argument marshalling only: every step of a product runs in the CUDA kernels
of ``libgf2.so`` (built in-tree by :func:`build`).  Importing this package
does not need a GPU; calling into the library does, and there is no CPU
fallback: a missing library raises :class:`LibraryNotBuilt`.

Matrices are passed as :class:`Mat` (the C ``gf2_mat``), made from

* a torch CUDA tensor of dtype int64 and shape ``(rows, stride_words)``
  holding the packed bits (``mat(t, cols)``), or
* a host numpy ``uint64`` array or torch CPU tensor of the same shape
  (device ``GF2_HOST``; pinned memory gives full copy speed).

Entry points keep the C names of every symbol in ``include/gf2.h`` (listed in
:data:`EXPORTS`): the product (``gf2_mul``, ``gf2_mul_batched``,
``gf2_mul_batched_ex``, ``gf2_mul_noalloc``), memory (``gf2_alloc``,
``gf2_free``), the steps of the path callable alone (``gf2_sw_split``,
``gf2_sw_combine``, ``gf2_make_table``), helpers (``gf2_random``,
``gf2_transpose``, ``gf2_freivalds``), scratch control, planning
(``gf2_describe_plan``), device-time accounting (``gf2_profile_*``) and
failure detection (``gf2_device_status``, ``gf2_selftest_wait``).

Base cases (``opts(base=...)``): ``GF2_BASE_AUTO`` (the autotuner's choice),
``GF2_BASE_M4RM`` (packed Method of the Four Russians), ``GF2_BASE_TC_FP8`` and
``GF2_BASE_TC_FP4`` (exact 0/1 FP8 / block-scaled FP4 tcgen05 products on
operands expanded once in HBM), and the warp-level ``GF2_BASE_TC_S8`` (int8)
and ``GF2_BASE_TC_B1`` (1-bit AND + popcount) forms.
"""
from __future__ import annotations

import ctypes
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libgf2.so")

GF2_OK = 0
GF2_EINVAL = -1
GF2_EALIAS = -2
GF2_ELAYOUT = -3
GF2_ENOMEM = -4
GF2_ECUDA = -5
GF2_ETIMEOUT = -6
GF2_EUNSUPPORTED = -7
GF2_EMISMATCH = -8
GF2_ESCRATCH = -9
#: size of the fixed device buffer used by gf2_mul_noalloc
GF2_NOALLOC_SCRATCH_BYTES = 32 << 20
GF2_HOST = -1

GF2_BASE_AUTO = 0
GF2_BASE_M4RM = 1
GF2_BASE_TC_FP8 = 2
GF2_BASE_TC_S8 = 3
GF2_BASE_TC_B1 = 4
GF2_BASE_TC_FP4 = 5

#: every symbol declared in include/gf2.h
EXPORTS = (
    "gf2_default_opts", "gf2_strerror", "gf2_alloc", "gf2_free", "gf2_mul", "gf2_mul_batched",
    "gf2_sw_split", "gf2_sw_combine", "gf2_make_table", "gf2_random", "gf2_transpose",
    "gf2_freivalds", "gf2_scratch_bytes", "gf2_reserve_scratch", "gf2_release_scratch",
    "gf2_launch_count", "gf2_describe_plan", "gf2_profile_enable", "gf2_profile_read",
    "gf2_profile_name", "gf2_mul_noalloc", "gf2_device_status", "gf2_mul_batched_ex",
    "gf2_batched_variant_count", "gf2_batched_variant_name", "gf2_selftest_wait",
)


class LibraryNotBuilt(RuntimeError):
    pass


class GF2Error(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__("%s: %s (%d)" % (where, strerror(status), status))


class Mat(ctypes.Structure):
    """``gf2_mat``: packed matrix (64 entries per word, row-major)."""
    _fields_ = [("data", ctypes.c_void_p), ("rows", ctypes.c_int64), ("cols", ctypes.c_int64),
                ("stride_words", ctypes.c_int64), ("device", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]

    def __repr__(self):
        return "Mat(rows=%d, cols=%d, stride=%d, device=%d)" % (
            self.rows, self.cols, self.stride_words, self.device)


class Opts(ctypes.Structure):
    """``gf2_opts``."""
    _fields_ = [("base", ctypes.c_int32), ("depth", ctypes.c_int32), ("k", ctypes.c_int32),
                ("t", ctypes.c_int32), ("accumulate", ctypes.c_int32), ("peel", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 2)]


def opts(base: int = GF2_BASE_AUTO, depth: int = -1, k: int = 0, t: int = 0,
         accumulate: int = 0, peel: int = -1) -> Opts:
    o = Opts()
    o.base, o.depth, o.k, o.t, o.accumulate, o.peel = base, depth, k, t, accumulate, peel
    return o


_lib = None
_lock = threading.Lock()
_P = ctypes.POINTER


def build(verbose: bool = False) -> str:
    """Compile libgf2.so for sm_103a (nvcc) in-tree."""
    from . import buildlib as _b
    return _b.build(verbose=verbose)


def lib():
    """The loaded ``libgf2.so`` (raises :class:`LibraryNotBuilt` when absent)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise LibraryNotBuilt(
                    "libgf2.so is not built (%s); run paper_0811_1714_gb300.build()" % LIB_PATH)
            L = ctypes.CDLL(LIB_PATH)
            i32, i64, vp, u64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p, ctypes.c_uint64
            sig = {
                "gf2_default_opts": (None, [_P(Opts)]),
                "gf2_strerror": (ctypes.c_char_p, [ctypes.c_int]),
                "gf2_alloc": (ctypes.c_int, [_P(Mat), i64, i64]),
                "gf2_free": (ctypes.c_int, [_P(Mat)]),
                "gf2_mul": (ctypes.c_int, [_P(Mat), _P(Mat), _P(Mat), _P(Opts), vp]),
                "gf2_mul_batched": (ctypes.c_int, [_P(_P(Mat)), _P(_P(Mat)), _P(_P(Mat)), i32,
                                                   _P(Opts), vp]),
                "gf2_sw_split": (ctypes.c_int, [vp, i64, _P(Mat), i32, vp]),
                "gf2_sw_combine": (ctypes.c_int, [_P(Mat), vp, i64, vp]),
                "gf2_make_table": (ctypes.c_int, [_P(Mat), _P(Mat), i64, i32, vp]),
                "gf2_random": (ctypes.c_int, [_P(Mat), u64, ctypes.c_double, vp]),
                "gf2_transpose": (ctypes.c_int, [_P(Mat), _P(Mat), vp]),
                "gf2_freivalds": (ctypes.c_int, [_P(Mat), _P(Mat), _P(Mat), u64, _P(i64), vp]),
                "gf2_scratch_bytes": (i64, [i64, i64, i64, _P(Opts)]),
                "gf2_reserve_scratch": (ctypes.c_int, [i64, vp]),
                "gf2_release_scratch": (ctypes.c_int, []),
                "gf2_launch_count": (i64, []),
                "gf2_describe_plan": (ctypes.c_int, [i64, i64, i64, _P(Opts), ctypes.c_char_p, i32]),
                "gf2_profile_enable": (ctypes.c_int, [i32]),
                "gf2_profile_read": (ctypes.c_int, [i32, _P(ctypes.c_double), _P(i64)]),
                "gf2_profile_name": (ctypes.c_char_p, [i32]),
                "gf2_mul_noalloc": (ctypes.c_int, [_P(Mat), _P(Mat), _P(Mat), _P(Opts), vp]),
                "gf2_device_status": (ctypes.c_int, [vp]),
                "gf2_mul_batched_ex": (ctypes.c_int, [_P(_P(Mat)), _P(_P(Mat)), _P(_P(Mat)), i32,
                                                      _P(Opts), i32, _P(i32), vp]),
                "gf2_batched_variant_count": (i32, []),
                "gf2_batched_variant_name": (ctypes.c_char_p, [i32]),
                "gf2_selftest_wait": (ctypes.c_int, [i64, vp]),
            }
            for name, (res, args) in sig.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def strerror(status: int) -> str:
    try:
        return lib().gf2_strerror(int(status)).decode()
    except LibraryNotBuilt:
        return "status %d" % status


def _check(rc: int, where: str) -> None:
    if rc != GF2_OK:
        raise GF2Error(rc, where)


def _stream(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        except Exception:
            pass
        return ctypes.c_void_p(0)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def mat(x, cols: int) -> Mat:
    """Describe a packed matrix held by a torch tensor or a numpy uint64 array.

    ``x`` has shape ``(rows, stride_words)``; the caller keeps ``x`` alive.
    """
    M = Mat()
    shape = tuple(x.shape)
    if len(shape) != 2:
        raise ValueError("packed matrices are 2-D (rows, stride_words)")
    M.rows, M.stride_words = shape
    M.cols = int(cols)
    if hasattr(x, "data_ptr"):          # torch
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        if x.element_size() != 8:
            raise ValueError("tensor must hold 64-bit words")
        M.data = x.data_ptr() or None
        M.device = x.device.index if x.is_cuda else GF2_HOST
        if x.is_cuda and M.device is None:
            import torch
            M.device = torch.cuda.current_device()
    else:                               # numpy
        if x.dtype.itemsize != 8 or not x.flags.c_contiguous:
            raise ValueError("numpy array must be C-contiguous 64-bit words")
        M.data = x.ctypes.data or None
        M.device = GF2_HOST
    return M


# ---- entry points (same names as the C ABI) -------------------------------

def gf2_alloc(rows: int, cols: int) -> Mat:
    M = Mat()
    _check(lib().gf2_alloc(ctypes.byref(M), rows, cols), "gf2_alloc")
    return M


def gf2_free(M: Mat) -> None:
    _check(lib().gf2_free(ctypes.byref(M)), "gf2_free")


def gf2_mul(C: Mat, A: Mat, B: Mat, options: Opts | None = None, stream=None) -> None:
    o = ctypes.byref(options) if options is not None else None
    _check(lib().gf2_mul(ctypes.byref(C), ctypes.byref(A), ctypes.byref(B), o, _stream(stream)),
           "gf2_mul")


def gf2_mul_noalloc(C: Mat, A: Mat, B: Mat, options: Opts | None = None, stream=None) -> None:
    """gf2_mul without any device allocation: the temporaries come from the
    library's fixed buffer (GF2_NOALLOC_SCRATCH_BYTES).  For callers that
    cannot allocate device memory; calls that overlap on the GPU race."""
    o = ctypes.byref(options) if options is not None else None
    _check(lib().gf2_mul_noalloc(ctypes.byref(C), ctypes.byref(A), ctypes.byref(B), o,
                                 _stream(stream)), "gf2_mul_noalloc")


class MatArrays:
    """Pointer arrays for the batched calls (build once, reuse: the batched
    form caches its plan and CUDA graph per set of operands)."""

    def __init__(self, C: list, A: list, B: list):
        n = len(A)
        if len(B) != n or len(C) != n:
            raise ValueError("C, A, B need the same length")
        self.n = n
        self.keep = (list(C), list(A), list(B))
        self.arrs = []
        for seq in self.keep:
            arr = (_P(Mat) * max(n, 1))()
            for i, M in enumerate(seq):
                arr[i] = ctypes.pointer(M)
            self.arrs.append(arr)


def gf2_mul_batched(C, A=None, B=None, options: Opts | None = None, stream=None) -> None:
    """C[i] = A[i] B[i]; pass three lists, or one MatArrays."""
    arrs = C if isinstance(C, MatArrays) else MatArrays(C, A, B)
    o = ctypes.byref(options) if options is not None else None
    _check(lib().gf2_mul_batched(arrs.arrs[0], arrs.arrs[1], arrs.arrs[2], arrs.n, o, _stream(stream)),
           "gf2_mul_batched")


def gf2_mul_batched_ex(C, A=None, B=None, options: Opts | None = None, variant: int = -1,
                       stream=None) -> int:
    """gf2_mul_batched with a pinned tile variant (or -1: autotuned); returns the variant used."""
    arrs = C if isinstance(C, MatArrays) else MatArrays(C, A, B)
    o = ctypes.byref(options) if options is not None else None
    ch = ctypes.c_int32(-1)
    _check(lib().gf2_mul_batched_ex(arrs.arrs[0], arrs.arrs[1], arrs.arrs[2], arrs.n, o, variant,
                                    ctypes.byref(ch), _stream(stream)), "gf2_mul_batched_ex")
    return ch.value


def gf2_batched_variant_count() -> int:
    return int(lib().gf2_batched_variant_count())


def gf2_batched_variant_name(i: int):
    r = lib().gf2_batched_variant_name(i)
    return r.decode() if r else None


def gf2_sw_split(out_ptr: int, slab_words: int, X: Mat, side: int, stream=None) -> None:
    _check(lib().gf2_sw_split(ctypes.c_void_p(out_ptr), slab_words, ctypes.byref(X), side,
                              _stream(stream)), "gf2_sw_split")


def gf2_sw_combine(C: Mat, P_ptr: int, slab_words: int, stream=None) -> None:
    _check(lib().gf2_sw_combine(ctypes.byref(C), ctypes.c_void_p(P_ptr), slab_words,
                                _stream(stream)), "gf2_sw_combine")


def gf2_make_table(T: Mat, B: Mat, r0: int, k: int, stream=None) -> None:
    _check(lib().gf2_make_table(ctypes.byref(T), ctypes.byref(B), r0, k, _stream(stream)),
           "gf2_make_table")


def gf2_random(M: Mat, seed: int, p: float = 0.5, stream=None) -> None:
    _check(lib().gf2_random(ctypes.byref(M), seed & 0xFFFFFFFFFFFFFFFF, float(p), _stream(stream)),
           "gf2_random")


def gf2_transpose(T: Mat, X: Mat, stream=None) -> None:
    _check(lib().gf2_transpose(ctypes.byref(T), ctypes.byref(X), _stream(stream)), "gf2_transpose")


def gf2_freivalds(C: Mat, A: Mat, B: Mat, seed: int, stream=None) -> int:
    bad = ctypes.c_int64(0)
    _check(lib().gf2_freivalds(ctypes.byref(C), ctypes.byref(A), ctypes.byref(B),
                               seed & 0xFFFFFFFFFFFFFFFF, ctypes.byref(bad), _stream(stream)),
           "gf2_freivalds")
    return bad.value


def gf2_scratch_bytes(m: int, l: int, n: int, options: Opts | None = None) -> int:
    o = ctypes.byref(options) if options is not None else None
    r = lib().gf2_scratch_bytes(m, l, n, o)
    if r < 0:
        raise GF2Error(int(r), "gf2_scratch_bytes")
    return int(r)


def gf2_reserve_scratch(nbytes: int, stream=None) -> None:
    _check(lib().gf2_reserve_scratch(nbytes, _stream(stream)), "gf2_reserve_scratch")


def gf2_release_scratch() -> None:
    _check(lib().gf2_release_scratch(), "gf2_release_scratch")


def gf2_launch_count() -> int:
    return int(lib().gf2_launch_count())


def gf2_describe_plan(m: int, l: int, n: int, options: Opts | None = None) -> str:
    buf = ctypes.create_string_buffer(512)
    o = ctypes.byref(options) if options is not None else None
    _check(lib().gf2_describe_plan(m, l, n, o, buf, 512), "gf2_describe_plan")
    return buf.value.decode()


def gf2_strerror(status: int) -> str:
    return strerror(status)


def gf2_device_status(stream=None) -> None:
    """Raise GF2Error(GF2_ETIMEOUT) when a bounded device wait expired."""
    _check(lib().gf2_device_status(_stream(stream)), "gf2_device_status")


def gf2_selftest_wait(limit_cycles: int, stream=None) -> None:
    """Launch a wait that can only time out (failure-detection self test)."""
    _check(lib().gf2_selftest_wait(limit_cycles, _stream(stream)), "gf2_selftest_wait")


def gf2_profile_enable(on: bool) -> None:
    _check(lib().gf2_profile_enable(1 if on else 0), "gf2_profile_enable")


def gf2_profile_read(family: int):
    """(device ms, launches) summed over the kernel family since profiling was enabled."""
    ms = ctypes.c_double(0)
    n = ctypes.c_int64(0)
    _check(lib().gf2_profile_read(family, ctypes.byref(ms), ctypes.byref(n)), "gf2_profile_read")
    return ms.value, n.value


def gf2_profile_name(family: int):
    r = lib().gf2_profile_name(family)
    return r.decode() if r else None


PROFILE_FAMILIES = ("m4rm", "tc_fp8", "sw_split", "sw_combine", "transpose", "random",
                    "freivalds", "make_table", "batched", "tc_s8", "tc_b1", "tc_fp4", "expand")


# ---- torch conveniences ----------------------------------------------------

def empty(rows: int, cols: int, device=None):
    """Zeroed torch int64 CUDA tensor in the library layout (even stride)."""
    import torch
    w = (cols + 63) // 64
    w += w & 1
    return torch.zeros((rows, w), dtype=torch.int64, device=device or "cuda")


def mul(A, B, l: int, n: int, options: Opts | None = None, out=None, stream=None):
    """C = A B for packed torch CUDA tensors (A: rows x ceil(l/64) words, B: l rows)."""
    m = A.shape[0]
    C = out if out is not None else empty(m, n, device=A.device)
    gf2_mul(mat(C, n), mat(A, l), mat(B, n), options, stream)
    return C
