"""Resumable 2D scan: t1 row blocks with CRC-checked checkpoint files.

A long scan (the c5 grid takes hours) is split into blocks of t1 rows
(heom_response_2d_rows, the same unit shard.py distributes).  Each finished
block's R_I and R_II are written to ``<directory>/rows_<j0>_<j1>.ckpt`` through
heom_ckpt_write; a later call with the same directory reloads every block whose
file passes its integrity check and computes only the rest.  A block file that
fails the check (truncated, corrupted) is computed again.  Host orchestration
only: the propagation runs in the library.
"""
import os

import numpy as np

from . import heom as H


def _block_path(directory, j0, j1):
    return os.path.join(directory, "rows_%d_%d.ckpt" % (j0, j1))


def response_2d_resumable(h, rho_eq, grid, directory, rows_per_block, stop_after=None):
    """R_I, R_II of shape (n_t2, n1, n3), computed block by block with checkpoints.

    stop_after: compute at most this many new blocks, then raise StopIteration
    (to interrupt a run deliberately; the finished blocks stay on disk).
    Returns (R_I, R_II, computed_blocks, reloaded_blocks).
    """
    os.makedirs(directory, exist_ok=True)
    n1, n3, nt2 = grid["n1"], grid["n3"], len(grid["t2_fs"])
    RI = np.zeros((nt2, n1, n3), dtype=np.complex128)
    RII = np.zeros((nt2, n1, n3), dtype=np.complex128)
    computed = reloaded = 0
    for j0 in range(0, n1, rows_per_block):
        j1 = min(n1, j0 + rows_per_block)
        path = _block_path(directory, j0, j1)
        buf = np.zeros((2, nt2, j1 - j0, n3), dtype=np.complex128)
        if os.path.exists(path):
            try:
                H.heom_ckpt_read(path, buf)
                RI[:, j0:j1], RII[:, j0:j1] = buf[0], buf[1]
                reloaded += 1
                continue
            except H.HeomError:
                pass   # damaged block: compute it again
        if stop_after is not None and computed >= stop_after:
            raise StopIteration("stopped after %d new blocks" % computed)
        bi, bii = H.heom_response_2d_rows(h, rho_eq, grid, j0, j1)
        buf[0], buf[1] = bi, bii
        H.heom_ckpt_write(path, buf)
        RI[:, j0:j1], RII[:, j0:j1] = bi, bii
        computed += 1
    return RI, RII, computed, reloaded
