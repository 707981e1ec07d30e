"""Host logic of a row partition of one large problem over several GPUs (a design for the
multi-GPU case; every run of this build has one GPU, so it is exercised on CPU ranks only).

One SNMPBB block (Alg. 1 over X with X_fix fixed, Eqs. (2.1)-(2.2)) needs, per outer
iteration, B = A X_fix, the r x r Gram G = X_fix^T X_fix, and FP64 inner products; every
other step is row-local.  With the rows of A, W, Ht split into contiguous ranges:

* A X_fix: each rank holds A[rows, :] and needs X_fix in full, so X_fix is all-gathered
  once per product (n x N words); the product of a rank's rows is local.
* G = X_fix^T X_fix = sum over ranks of the local Grams: one all-reduce of r x r per restart.
* the line-search and BB inner products (<g, D>, ||D||^2, <S, Y>, ...): one all-reduce of a
  few FP64 scalars per restart per step; every rank then runs the same scalar control.
* LAI (Sec. 2.3): X^ = U^T X is a sum over row ranges, one all-reduce of l x N.

The compute callables are supplied by the caller (on a GPU the library's kernels); this
module holds the partition and the exchange pattern only and has no arithmetic of its own
beyond the sums the collectives perform.
"""
from __future__ import annotations


def row_ranges(n: int, world: int):
    """Contiguous row ranges [lo, hi) of n rows over `world` ranks, sizes differing by <= 1."""
    base, extra = divmod(n, world)
    out, lo = [], 0
    for k in range(world):
        hi = lo + base + (1 if k < extra else 0)
        out.append((lo, hi))
        lo = hi
    return out


def allgather_rows(X_local, rank: int, world: int, n: int):
    """X in full (n x N) from every rank's row block (torch tensors; gloo or NCCL)."""
    import torch
    import torch.distributed as dist

    ranges = row_ranges(n, world)
    hi_max = max(hi - lo for lo, hi in ranges)
    pad = torch.zeros((hi_max, X_local.shape[1]), dtype=X_local.dtype, device=X_local.device)
    pad[: X_local.shape[0]] = X_local
    parts = [torch.empty_like(pad) for _ in range(world)]
    dist.all_gather(parts, pad)
    return torch.cat([parts[k][: hi - lo] for k, (lo, hi) in enumerate(ranges)], dim=0)


def sharded_product(A_rows, X_local, rank: int, world: int, n: int, product):
    """This rank's rows of A X: X all-gathered, then product(A_rows, X_full) locally."""
    return product(A_rows, allgather_rows(X_local, rank, world, n))


def sharded_gram(X_local, gram):
    """G = sum over ranks of gram(X_local) (one all-reduce of the r x r result)."""
    import torch.distributed as dist

    G = gram(X_local)
    dist.all_reduce(G)
    return G


def sharded_dots(values):
    """FP64 inner-product partials summed over ranks (one all-reduce)."""
    import torch
    import torch.distributed as dist

    t = torch.as_tensor(values, dtype=torch.float64)
    dist.all_reduce(t)
    return t
