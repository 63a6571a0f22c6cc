"""Seeded synthetic inputs for GF(2) matrix products.

This module only draws random bits and shapes.  It holds none of the
multiplication arithmetic, so both the CPU oracle and the CUDA path may take
their inputs from it without sharing any of the method.

Generator definition (implemented a second time, independently, by the
device generator of the CUDA library; the two are compared bit for bit):

* SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number
  generators", OOPSLA 2014): the n-th output (n >= 1) of the stream whose
  state starts at ``s0`` is ``mix(s0 + n * GAMMA)`` with
  ``GAMMA = 0x9E3779B97F4A7C15`` and
  ``mix(z) = z3 ^ (z3 >> 31)``, where
  ``z1 = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9``,
  ``z2 = (z1 ^ (z1 >> 27)) * 0x94D049BB133111EB``, ``z3 = z2``
  (all arithmetic modulo 2**64).
* A matrix with ``rows x cols`` entries is drawn from the stream with
  ``s0 = seed``.  Its logical width is ``W = ceil(cols / 64)`` words; the
  word ``w`` of row ``r`` is the output number ``n = r * W + w + 1`` when the
  bit density is 1/2.  Bit ``b`` of a word is the entry in column
  ``64 * w + b`` (least significant bit first).  Columns ``>= cols`` are 0.
* For a density ``p != 1/2`` the word ``(r, w)`` uses the 32 outputs
  ``n = (r * W + w) * 32 + j + 1`` (``j = 0..31``); output ``j`` gives two
  32-bit uniforms, its low half for bit ``2j`` and its high half for bit
  ``2j + 1``; a bit is 1 when its uniform is below ``floor(p * 2**32)``.
* The padded layout has ``stride >= W`` words per row; words ``W..stride-1``
  are 0.  Bits therefore do not depend on the padding.
"""
from __future__ import annotations

import math

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_S30 = np.uint64(30)
_S27 = np.uint64(27)
_S31 = np.uint64(31)

#: seeds used throughout the tests and the benchmark
SEED_A = 1
SEED_B = 2
SEED_C = 3
SEED_FREIVALDS = 1000
SEED_BATCH_DIMS = 42


def _mix(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> _S30)) * _M1
    z = (z ^ (z >> _S27)) * _M2
    return z ^ (z >> _S31)


def splitmix64(seed: int, n: np.ndarray) -> np.ndarray:
    """Outputs number ``n`` (uint64 array, n >= 1) of the stream seeded by ``seed``."""
    with np.errstate(over="ignore"):
        s = np.uint64(int(seed) & 0xFFFFFFFFFFFFFFFF) + np.asarray(n, dtype=np.uint64) * GAMMA
        return _mix(s)


def words_for(cols: int) -> int:
    return (cols + 63) // 64


def padded_stride(cols: int) -> int:
    """Row stride in 64-bit words used by the library: ceil(cols/64) rounded up to even."""
    w = words_for(cols)
    return w + (w & 1)


def tail_mask(cols: int) -> np.uint64:
    r = cols % 64
    return np.uint64(0xFFFFFFFFFFFFFFFF if r == 0 else (1 << r) - 1)


def random_packed(rows: int, cols: int, seed: int, p: float = 0.5,
                  stride: int | None = None, row0: int = 0) -> np.ndarray:
    """Packed bits of rows ``row0 .. row0+rows-1`` of the seeded ``? x cols`` matrix.

    Returns a ``(rows, stride)`` uint64 array (stride defaults to the padded
    library stride).  Drawing a row range gives exactly the rows a full draw
    would give, so large matrices can be sampled without drawing them whole.
    """
    W = words_for(cols)
    if stride is None:
        stride = padded_stride(cols)
    if stride < W:
        raise ValueError("stride below the logical width")
    out = np.zeros((rows, stride), dtype=np.uint64)
    if rows == 0 or W == 0:
        return out
    idx = (np.arange(row0, row0 + rows, dtype=np.uint64)[:, None] * np.uint64(W)
           + np.arange(W, dtype=np.uint64)[None, :])
    if p == 0.5:
        words = splitmix64(seed, idx + np.uint64(1))
    else:
        thr = np.uint64(int(math.floor(p * 2.0 ** 32)))
        words = np.zeros((rows, W), dtype=np.uint64)
        lo_mask = np.uint64(0xFFFFFFFF)
        for j in range(32):
            o = splitmix64(seed, idx * np.uint64(32) + np.uint64(j + 1))
            lo = (o & lo_mask) < thr
            hi = (o >> np.uint64(32)) < thr
            words |= lo.astype(np.uint64) << np.uint64(2 * j)
            words |= hi.astype(np.uint64) << np.uint64(2 * j + 1)
    words[:, W - 1] &= tail_mask(cols)
    out[:, :W] = words
    return out


def random_packed_cols(rows: int, cols: int, seed: int, c0: int, c1: int,
                       p: float = 0.5) -> np.ndarray:
    """Packed bits of columns ``c0 .. c1-1`` (c0 a multiple of 64) of all rows.

    Returns a ``(rows, ceil((c1-c0)/64))`` uint64 array holding those columns
    re-based to column 0, tail bits zero.
    """
    if c0 % 64:
        raise ValueError("c0 must be a multiple of 64")
    W = words_for(cols)
    w0, w1 = c0 // 64, words_for(c1)
    idx = (np.arange(rows, dtype=np.uint64)[:, None] * np.uint64(W)
           + np.arange(w0, w1, dtype=np.uint64)[None, :])
    if p == 0.5:
        words = splitmix64(seed, idx + np.uint64(1))
    else:
        thr = np.uint64(int(math.floor(p * 2.0 ** 32)))
        words = np.zeros(idx.shape, dtype=np.uint64)
        lo_mask = np.uint64(0xFFFFFFFF)
        for j in range(32):
            o = splitmix64(seed, idx * np.uint64(32) + np.uint64(j + 1))
            words |= ((o & lo_mask) < thr).astype(np.uint64) << np.uint64(2 * j)
            words |= ((o >> np.uint64(32)) < thr).astype(np.uint64) << np.uint64(2 * j + 1)
    words[:, -1] &= tail_mask(c1 - c0)
    if cols < c1:
        raise ValueError("column range beyond the matrix")
    return np.ascontiguousarray(words)


def batch_dims(count: int, seed: int = SEED_BATCH_DIMS, lo: int = 64, hi: int = 2048):
    """``count`` triples (m, l, n), each log-uniform in [lo, hi].

    Dimension ``d`` (0, 1, 2) of product ``i`` uses the output
    ``n = 3 * i + d + 1`` of the stream; ``U = (out >> 11) / 2**53`` and the
    size is ``floor(lo * (hi/lo) ** U)`` clamped to [lo, hi].
    """
    n = np.arange(3 * count, dtype=np.uint64) + np.uint64(1)
    u = (splitmix64(seed, n) >> np.uint64(11)).astype(np.float64) / float(2 ** 53)
    v = np.floor(lo * np.exp(u * math.log(hi / lo))).astype(np.int64)
    v = np.clip(v, lo, hi)
    return [tuple(int(x) for x in v[3 * i:3 * i + 3]) for i in range(count)]


def pack_bits(bits: np.ndarray, stride: int | None = None) -> np.ndarray:
    """Pack a 0/1 uint8 ``(rows, cols)`` array into the library layout (LSB-first)."""
    bits = np.asarray(bits, dtype=np.uint8)
    rows, cols = bits.shape
    W = words_for(cols)
    if stride is None:
        stride = padded_stride(cols)
    padded = np.zeros((rows, W * 64), dtype=np.uint8)
    padded[:, :cols] = bits & 1
    b = np.packbits(padded.reshape(rows, W * 8, 8), axis=2, bitorder="little").reshape(rows, W * 8)
    out = np.zeros((rows, stride), dtype=np.uint64)
    out[:, :W] = b.view(np.uint64).reshape(rows, W) if rows else out[:, :W]
    return out


def unpack_bits(packed: np.ndarray, cols: int) -> np.ndarray:
    """Inverse of :func:`pack_bits` (tail bits beyond ``cols`` are dropped)."""
    packed = np.ascontiguousarray(packed, dtype=np.uint64)
    rows = packed.shape[0]
    W = words_for(cols)
    if rows == 0 or cols == 0:
        return np.zeros((rows, cols), dtype=np.uint8)
    b = packed[:, :W].copy().view(np.uint8).reshape(rows, W, 8)
    bits = np.unpackbits(b, axis=2, bitorder="little").reshape(rows, W * 64)
    return np.ascontiguousarray(bits[:, :cols])
