"""Multi-GPU sharding of the 2D scan (one process per GPU).

The t1 rows of a 2D response are independent once the equilibrium hierarchy is
known: each rank computes a contiguous block of rows (heom_response_2d_rows,
trunk recomputed from rho_eq up to its first row) and the only collective is one
gather of the R arrays at the end.  Spectra are then formed on rank 0
(heom_spectrum_2d).  No data-path collective is needed.
"""
import numpy as np


def row_range(n1, world, rank):
    """Contiguous, balanced block of t1 rows for ``rank`` out of ``world``."""
    base, extra = divmod(n1, world)
    j0 = rank * base + min(rank, extra)
    return j0, j0 + base + (1 if rank < extra else 0)


def gather_rows(local_RI, local_RII, n1, world, rank, dist, group=None):
    """All-gather row blocks (complex, shape (n_t2, rows, n3)) into full arrays.

    Every rank pads its block to the largest block size, so one all_gather of
    equal-sized tensors suffices; returns the full (n_t2, n1, n3) arrays.
    """
    import torch
    n_t2, _, n3 = local_RI.shape
    maxrows = max(row_range(n1, world, r)[1] - row_range(n1, world, r)[0] for r in range(world))
    pad = np.zeros((2, n_t2, maxrows, n3), dtype=np.complex128)
    pad[0, :, :local_RI.shape[1]] = local_RI
    pad[1, :, :local_RII.shape[1]] = local_RII
    t = torch.from_numpy(pad.view(np.float64).copy())
    outs = [torch.empty_like(t) for _ in range(world)]
    dist.all_gather(outs, t, group=group)
    RI = np.zeros((n_t2, n1, n3), dtype=np.complex128)
    RII = np.zeros_like(RI)
    for r, o in enumerate(outs):
        j0, j1 = row_range(n1, world, r)
        blk = o.numpy().view(np.complex128).reshape(2, n_t2, maxrows, n3)
        RI[:, j0:j1] = blk[0, :, :j1 - j0]
        RII[:, j0:j1] = blk[1, :, :j1 - j0]
    return RI, RII


def response_2d_sharded(h, rho_eq, grid, dist=None, rows_fn=None, group=None):
    """R_I, R_II (and S_C on every rank) with the t1 rows split over the ranks.

    ``rows_fn(j0, j1)`` computes a row block; by default the C ABI's
    heom_response_2d_rows on this rank's GPU.
    """
    from . import heom as H
    world = dist.get_world_size(group) if dist is not None and dist.is_initialized() else 1
    rank = dist.get_rank(group) if world > 1 else 0
    j0, j1 = row_range(grid["n1"], world, rank)
    if rows_fn is None:
        def rows_fn(a, b):
            return H.heom_response_2d_rows(h, rho_eq, grid, a, b)
    if j1 > j0:
        RI, RII = rows_fn(j0, j1)
    else:   # more ranks than t1 rows: this rank only takes part in the gather
        RI = np.zeros((len(grid["t2_fs"]), 0, grid["n3"]), dtype=np.complex128)
        RII = np.zeros_like(RI)
    if world > 1:
        RI, RII = gather_rows(RI, RII, grid["n1"], world, rank, dist, group)
    return RI, RII
