"""Row-block sharding of one product C = A B over the ranks of a process group.

Each row of C depends only on the same row of A and on all of B (the problem
statement of Section 3: C's rows are A's rows times B), so the rows of A and
C are partitioned across the ranks, B is replicated by ONE broadcast, every
rank multiplies its own block of rows with the library's product, and no
reduction is needed.  The blocks of C can be gathered on one rank
(stitching).  A split of the inner dimension K would need an XOR reduction
of partial products, which the collectives do not offer, so it is not used.

The collectives are torch.distributed's (NCCL for CUDA tensors, gloo for CPU
tensors); the arithmetic of every step runs in the library's kernels
(``gf2_mul`` on the rank's GPU) unless the caller hands in another local
product.
"""
from __future__ import annotations


def row_blocks(m: int, world: int, align: int = 64) -> list[tuple[int, int]]:
    """Contiguous blocks [r0, r1) of the m rows, one per rank, as even as
    possible with every boundary a multiple of `align` (the last block takes
    the remainder).  Blocks may be empty when m is small."""
    if world < 1 or m < 0 or align < 1:
        raise ValueError("need world >= 1, m >= 0, align >= 1")
    units = (m + align - 1) // align
    out, start = [], 0
    for r in range(world):
        take = units // world + (1 if r < units % world else 0)
        r0 = min(m, start * align)
        start += take
        r1 = min(m, start * align)
        out.append((r0, r1))
    return out


def gf2_mul_sharded(A_local, B, l: int, n: int, group=None, src: int = 0, gather: bool = True,
                    options=None, local_mul=None):
    """C = A B with the rows of A and C distributed over the ranks of `group`.

    A_local: this rank's block of rows of A (packed, ``(rows, stride_words)``
    int64 tensor; the blocks of the ranks in rank order make up A, e.g. from
    :func:`row_blocks`).  B: a packed ``l x n`` tensor of the same shape on
    every rank; its contents matter on `src` only and are broadcast in place.
    Returns ``(C_local, C)``: this rank's rows of C, and on `src` (with
    `gather`) the whole of C stitched from every rank's rows (None elsewhere).

    local_mul(C, A, B) computes one rank's block; by default the library's
    ``gf2_mul`` on CUDA tensors with `options`.
    """
    import torch
    import torch.distributed as dist
    from . import empty, gf2_mul, mat

    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    if local_mul is None:
        def local_mul(C, A, Bm):
            if A.shape[0]:
                gf2_mul(mat(C, n), mat(A, l), mat(Bm, n), options)
    dist.broadcast(B, src=src, group=group)                   # B replicated: one broadcast
    rows = int(A_local.shape[0])
    W = B.shape[1]
    C_local = torch.zeros((rows, W), dtype=torch.int64, device=A_local.device) \
        if A_local.device.type == "cpu" else empty(rows, n, device=A_local.device)
    local_mul(C_local, A_local, B)
    if not gather:
        return C_local, None
    # stitching: every block padded to the largest, gathered on src in rank order
    counts = torch.tensor([rows], dtype=torch.int64, device=A_local.device)
    all_counts = [torch.zeros_like(counts) for _ in range(world)]
    dist.all_gather(all_counts, counts, group=group)
    sizes = [int(c.item()) for c in all_counts]
    top = max(sizes) if sizes else 0
    padded = torch.zeros((top, W), dtype=torch.int64, device=A_local.device)
    padded[:rows] = C_local
    parts = [torch.zeros_like(padded) for _ in range(world)] if rank == src else None
    dist.gather(padded, gather_list=parts, dst=src, group=group)
    if rank != src:
        return C_local, None
    return C_local, torch.cat([p[:k] for p, k in zip(parts, sizes)], dim=0)
