"""CPU oracle for dense matrix multiplication over GF(2).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  It shares no
code with the CUDA library (``paper_0811_1714_gb300``) and never imports it.

Contents, each citing the passage of Albrecht, Bard and Hart, "Efficient
Multiplication of Dense Matrices over GF(2)" that it restates:

* ``mul`` / ``mul_packed`` -- the definition C[i][j] = XOR_t A[i][t] AND B[t][j]
  (Abstract: + is XOR, * is AND; Section 3 problem statement; Section 2.3),
  computed by the naive cubic loop of ``gf2_oracle.c`` on unpacked bytes.
* ``matvec64`` -- the packed matrix-vector product of Section 2.3 (AND,
  XOR-accumulate, parity), used for Freivalds checks at large sizes.
* ``gray_code`` -- the reflected Gray code built as Section 3.1 describes.
* ``make_table`` / ``m4rm`` -- Algorithm 1 (M4RM) with a Gray-code table
  (Section 3, Section 3.1), plus the t-table variant of Algorithm 3
  (Section 3.3).
* ``strassen_winograd`` / ``sw_operands`` / ``sw_combine`` -- Algorithm 4
  (Section 4), with zero padding of odd sizes (Section 4).

Pins (tests marked ``not gpu``): brute force over all 2x2 and 3x3 operand
pairs, the worked k = 1 example of Section 3, numpy integer products mod 2,
the Gray-code figure of Section 3.1, the 2^k - 1 table-addition count of
Section 3.1, and the algebraic identities A I = A, (AB)C = A(BC),
(AB)^T = B^T A^T and distributivity.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gf2_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "libgf2_oracle.so")
_lib = None
_lock = threading.Lock()

_u64p = ctypes.POINTER(ctypes.c_uint64)
_u8p = ctypes.POINTER(ctypes.c_uint8)
_i64 = ctypes.c_int64


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (OpenMP when available) into oracle/_build."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + ".%d.tmp" % os.getpid()
    base = ["gcc", "-O2", "-std=c11", "-shared", "-fPIC", _SRC, "-o", tmp]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True,
                       capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.gf2o_mul_packed.restype = ctypes.c_int
            lib.gf2o_mul_packed.argtypes = [_u64p, _i64, _u64p, _i64, _u64p, _i64, _i64, _i64, _i64]
            lib.gf2o_mul_unpacked.restype = None
            lib.gf2o_mul_unpacked.argtypes = [_u8p, _u8p, _u8p, _i64, _i64, _i64]
            lib.gf2o_unpack.restype = None
            lib.gf2o_unpack.argtypes = [_u64p, _i64, _i64, _i64, _u8p]
            lib.gf2o_pack.restype = None
            lib.gf2o_pack.argtypes = [_u8p, _i64, _i64, _i64, _u64p]
            lib.gf2o_matvec64.restype = None
            lib.gf2o_matvec64.argtypes = [_u64p, _i64, _i64, _i64, _u64p, _u64p]
            lib.gf2o_num_threads.restype = ctypes.c_int
            lib.gf2o_set_threads.restype = None
            lib.gf2o_set_threads.argtypes = [ctypes.c_int]
            _lib = lib
    return _lib


def num_threads() -> int:
    return _load().gf2o_num_threads()


def set_threads(n: int) -> None:
    _load().gf2o_set_threads(int(n))


def _p64(a):
    return a.ctypes.data_as(_u64p)


def _p8(a):
    return a.ctypes.data_as(_u8p)


# ---------------------------------------------------------------------------
# The definition (Section 2.3, Section 3 problem statement)
# ---------------------------------------------------------------------------

def mul(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """C = A B over GF(2) on unpacked 0/1 arrays (naive cubic, in C)."""
    A = np.ascontiguousarray(A, dtype=np.uint8)
    B = np.ascontiguousarray(B, dtype=np.uint8)
    m, l = A.shape
    l2, n = B.shape
    if l != l2:
        raise ValueError("inner dimensions differ")
    C = np.zeros((m, n), dtype=np.uint8)
    if m and n:
        _load().gf2o_mul_unpacked(_p8(A), _p8(B), _p8(C), m, l, n)
    return C


def unpack(P: np.ndarray, rows: int, cols: int) -> np.ndarray:
    """Packed words (Section 2.1 layout, LSB-first) -> 0/1 bytes (oracle's own code)."""
    P = np.ascontiguousarray(P, dtype=np.uint64)
    out = np.zeros((rows, cols), dtype=np.uint8)
    if rows and cols:
        _load().gf2o_unpack(_p64(P), rows, cols, P.shape[1], _p8(out))
    return out


def pack(bits: np.ndarray, stride: int) -> np.ndarray:
    """0/1 bytes -> packed words with the given stride (oracle's own code)."""
    bits = np.ascontiguousarray(bits, dtype=np.uint8)
    rows, cols = bits.shape
    out = np.zeros((rows, stride), dtype=np.uint64)
    if rows:
        _load().gf2o_pack(_p8(bits), rows, cols, stride, _p64(out))
    return out


def mul_packed(A: np.ndarray, B: np.ndarray, m: int, l: int, n: int,
               stride_c: int | None = None, b_col0: int = 0) -> np.ndarray:
    """C = A B on packed operands (rows of A: l entries, rows of B: n entries).

    ``A`` is ``(m, sa)`` and ``B`` is ``(l, sb)`` uint64.  With ``b_col0``
    (a multiple of 64) the product uses columns ``b_col0 .. b_col0+n-1`` of B.
    Returns ``(m, stride_c)`` packed words, tail bits zero.
    """
    if b_col0 % 64:
        raise ValueError("b_col0 must be a multiple of 64")
    A = np.ascontiguousarray(A, dtype=np.uint64)
    B = np.ascontiguousarray(B, dtype=np.uint64)
    if stride_c is None:
        w = (n + 63) // 64
        stride_c = max(w + (w & 1), 0)
    C = np.zeros((m, max(stride_c, 0)), dtype=np.uint64)
    if m == 0 or n == 0:
        return C
    if l == 0:
        return C
    Bv = B[:, b_col0 // 64:]
    Bv = np.ascontiguousarray(Bv)
    rc = _load().gf2o_mul_packed(_p64(A), A.shape[1], _p64(Bv), Bv.shape[1],
                                 _p64(C), stride_c, m, l, n)
    if rc:
        raise MemoryError("oracle allocation failed")
    return C


def matvec64(M: np.ndarray, r: int, c: int, X: np.ndarray) -> np.ndarray:
    """Y = M X for 64 packed column vectors (Section 2.3 AND / XOR / parity)."""
    M = np.ascontiguousarray(M, dtype=np.uint64)
    X = np.ascontiguousarray(X, dtype=np.uint64).reshape(-1)
    if X.shape[0] < c:
        raise ValueError("X needs one word per column of M")
    Y = np.zeros(r, dtype=np.uint64)
    if r and c:
        _load().gf2o_matvec64(_p64(M), r, c, M.shape[1], _p64(X), _p64(Y))
    return Y


# ---------------------------------------------------------------------------
# Section 3.1: Gray codes
# ---------------------------------------------------------------------------

def gray_code(k: int) -> list[tuple[int, ...]]:
    """Reflected Gray code on k bits, built the way Section 3.1 describes.

    The (k)-bit table is the (k-1)-bit table with 0 prepended, followed by the
    (k-1)-bit table in reverse order with 1 prepended.  Entries are tuples of
    bits, most significant (leftmost in the paper's figure) first.
    """
    if k < 0:
        raise ValueError("k >= 0")
    table: list[tuple[int, ...]] = [()]
    for _ in range(k):
        table = [(0,) + e for e in table] + [(1,) + e for e in reversed(table)]
    return table


def _bits_to_int(bits: tuple[int, ...]) -> int:
    v = 0
    for b in bits:
        v = 2 * v + b
    return v


# ---------------------------------------------------------------------------
# Section 3: Algorithm 1 (M4RM) and Section 3.3: Algorithm 3 (t tables)
# ---------------------------------------------------------------------------

def read_bits(A: np.ndarray, r: int, c: int, k: int) -> int:
    """ReadBits of Algorithm 1: entries c .. c+k-1 of row r, first one most significant."""
    v = 0
    for j in range(k):
        v = 2 * v + int(A[r, c + j])
    return v


def make_table(B: np.ndarray, r: int, c: int, k: int):
    """MakeTable of Algorithm 1 with the Gray-code walk of Section 3.1.

    Returns ``(T, additions)``: ``T[x]`` is the combination of rows
    ``r .. r+k-1`` of B (columns from ``c``) selected by the k-bit value x read
    the way ReadBits reads it (bit k-1-j of x selects row r+j), and
    ``additions`` is the number of row additions performed.  Walking the Gray
    code, each new entry differs from the previous one in exactly one bit, so
    it costs exactly one row addition.
    """
    n = B.shape[1] - c
    T = np.zeros((1 << k, n), dtype=np.uint8)
    codes = gray_code(k)
    additions = 0
    prev_bits = codes[0]
    prev_val = 0
    for bits in codes[1:]:
        diff = [j for j in range(k) if bits[j] != prev_bits[j]]
        assert len(diff) == 1
        j = diff[0]  # position j in the code selects row r + j
        val = _bits_to_int(bits)
        T[val] = T[prev_val] ^ B[r + j, c:]
        additions += 1
        prev_bits, prev_val = bits, val
    return T, additions


def m4rm(A: np.ndarray, B: np.ndarray, k: int) -> np.ndarray:
    """Algorithm 1 (M4RM) on unpacked 0/1 arrays.

    The stripes of k columns of A / k rows of B are taken in order; when k
    does not divide l, the last stripe is narrower (``l mod k`` entries).
    """
    A = np.asarray(A, dtype=np.uint8)
    B = np.asarray(B, dtype=np.uint8)
    m, l = A.shape
    n = B.shape[1]
    C = np.zeros((m, n), dtype=np.uint8)
    for s in range(0, l, k):
        kk = min(k, l - s)
        T, _ = make_table(B, s, 0, kk)
        for j in range(m):
            C[j] ^= T[read_bits(A, j, s, kk)]
    return C


def m4rm_tables(A: np.ndarray, B: np.ndarray, k: int, t: int) -> np.ndarray:
    """Algorithm 3 generalised to t tables (Section 3.3): t tables per pass over
    t*k rows of B; each row of C receives t table rows per pass."""
    A = np.asarray(A, dtype=np.uint8)
    B = np.asarray(B, dtype=np.uint8)
    m, l = A.shape
    n = B.shape[1]
    C = np.zeros((m, n), dtype=np.uint8)
    for s in range(0, l, t * k):
        tabs = []
        for i in range(t):
            r = s + i * k
            if r >= l:
                break
            kk = min(k, l - r)
            tabs.append((r, kk, make_table(B, r, 0, kk)[0]))
        for j in range(m):
            acc = C[j].copy()
            for r, kk, T in tabs:
                acc ^= T[read_bits(A, j, r, kk)]
            C[j] = acc
    return C


# ---------------------------------------------------------------------------
# Section 4: Algorithm 4 (Strassen-Winograd)
# ---------------------------------------------------------------------------

def quadrants(X: np.ndarray):
    """NW, NE, SW, SE quadrants of a matrix with even dimensions."""
    r, c = X.shape
    h, w = r // 2, c // 2
    return X[:h, :w], X[:h, w:], X[h:, :w], X[h:, w:]


def sw_operands(A: np.ndarray, B: np.ndarray):
    """The 8 additions of Algorithm 4 and the operands of its 7 products.

    Over GF(2) subtraction is addition, so every - of the algorithm is XOR.
    Returns ``(lhs, rhs)``: lists of the 7 left and right factors of
    P0 .. P6 in the algorithm's order.
    """
    ANW, ANE, ASW, ASE = quadrants(A)
    BNW, BNE, BSW, BSE = quadrants(B)
    S0 = ASW ^ ASE
    S1 = S0 ^ ANW
    S2 = ANW ^ ASW
    S3 = ANE ^ S1
    T0 = BNE ^ BNW
    T1 = BSE ^ T0
    T2 = BSE ^ BNE
    T3 = T1 ^ BSW
    lhs = [ANW, ANE, S3, ASE, S0, S1, S2]
    rhs = [BNW, BSW, BSE, T3, T0, T1, T2]
    return lhs, rhs


def sw_combine(P: list[np.ndarray]) -> np.ndarray:
    """The 7 final additions of Algorithm 4, then Augment and Stack."""
    P0, P1, P2, P3, P4, P5, P6 = P
    U0 = P0 ^ P1
    U1 = P0 ^ P5
    U2 = U1 ^ P6
    U3 = U1 ^ P4
    U4 = U3 ^ P2
    U5 = U2 ^ P3
    U6 = U2 ^ P4
    CN = np.concatenate([U0, U4], axis=1)   # Augment(U0, U4)
    CS = np.concatenate([U5, U6], axis=1)   # Augment(U5, U6)
    return np.concatenate([CN, CS], axis=0)  # Stack(CN, CS)


def strassen_winograd(A: np.ndarray, B: np.ndarray, depth: int, base=None) -> np.ndarray:
    """Algorithm 4 applied ``depth`` times, then ``base`` (default: the cubic oracle).

    Odd sizes are padded with zero rows / columns to even sizes at each level
    (the "padding" strategy of Section 4); the product is then cut back out.
    """
    A = np.asarray(A, dtype=np.uint8)
    B = np.asarray(B, dtype=np.uint8)
    if base is None:
        base = mul
    m, l = A.shape
    n = B.shape[1]
    if depth <= 0 or min(m, l, n) < 2:
        return base(A, B)
    mp, lp, np_ = m + (m & 1), l + (l & 1), n + (n & 1)
    Ap = np.zeros((mp, lp), dtype=np.uint8)
    Ap[:m, :l] = A
    Bp = np.zeros((lp, np_), dtype=np.uint8)
    Bp[:l, :n] = B
    lhs, rhs = sw_operands(Ap, Bp)
    P = [strassen_winograd(x, y, depth - 1, base) for x, y in zip(lhs, rhs)]
    return sw_combine(P)[:m, :n]
