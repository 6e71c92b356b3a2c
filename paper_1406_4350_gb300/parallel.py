"""Distribution of one problem, or of a batch of k-points, over the ranks of a job (one GPU
per rank), with torch.distributed for the exchange steps.

Section 5.2 of the paper distributes Psi over a 2-D grid of plane-wave and band groups and
moves it with an all-to-all before Rayleigh-Ritz.  Here the split follows what the method
allows on GPUs that each hold the whole operator:

* bands: Algorithm 2's filter treats every band on its own, so rank r filters the contiguous
  band range ``band_range(nb, world, r)`` with no communication; Rayleigh-Ritz needs every
  band, so ``gather_bands`` assembles the block on every rank (all-gather), each rank runs
  the dense step and keeps its own bands of the rotated block;
* k-points: independent eigenproblems, ``kpoint_range`` gives each rank its share with no
  communication at all;
* ``row_sharded_gram``: the reduction a plane-wave (row) split of Rayleigh-Ritz would use --
  every rank forms X_r^H Y_r on its rows and an all-reduce sums the N_b x N_b partials.

Only argument bookkeeping and collectives live here; all arithmetic on the GPU runs in
libchebfi (the caller passes its local product in).
"""
from __future__ import annotations

__all__ = ["band_range", "kpoint_range", "gather_bands", "row_sharded_gram"]


def band_range(nb: int, world: int, rank: int):
    """Contiguous band range [b0, b1) of rank `rank` when nb bands are split over `world` ranks
    (ceil(nb / world) per rank, the last ranks possibly shorter or empty)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank %d outside a world of %d" % (rank, world))
    per = -(-nb // world)
    b0 = min(nb, rank * per)
    return b0, min(nb, b0 + per)


def kpoint_range(nk: int, world: int, rank: int):
    """k-points [k0, k1) of rank `rank` (the same contiguous split as the bands)."""
    return band_range(nk, world, rank)


def gather_bands(Y_local, nb: int, world: int):
    """Every rank's band range of an (npw, nb) column-major complex block, assembled on every
    rank: returns the full (npw, nb) block, column-major.  Collective over the default group."""
    import torch
    import torch.distributed as dist
    npw = Y_local.shape[0]
    per = -(-nb // world)
    buf = torch.zeros((per, npw), dtype=Y_local.dtype, device=Y_local.device)
    if Y_local.shape[1]:
        buf[: Y_local.shape[1]] = Y_local.T
    parts = [torch.empty_like(buf) for _ in range(world)]
    dist.all_gather([torch.view_as_real(p) for p in parts], torch.view_as_real(buf))
    out = torch.cat(parts, dim=0)[:nb]
    return out.T  # (npw, nb), column-major


def row_sharded_gram(local_product, nb: int):
    """Sum over the ranks of each rank's N_b x N_b partial product (its rows' share of
    X^H Y): `local_product` is this rank's partial; returns the full matrix on every rank."""
    import torch.distributed as dist
    out = local_product.clone()
    dist.all_reduce(out)
    return out
