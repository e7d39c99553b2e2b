"""The row partition of a SAND query in the tensor-core kernel (variant 3), checked on the host.

The kernel's index arithmetic, restated: rows [0, bin_start[1]) (exit layer >= 2) go to the
tensor-core tiles, t = blockIdx + k * grid, rows 128 t + r valid while < bin_start[1]; rows
[bin_start[1], n) (exit layer 1) go to the two CUDA-core warps, each of their 64 threads
taking rows base + 64 j (j < 8) of 512-row steps, base = 512 blockIdx + thread + k * 512 grid,
valid while < n - bin_start[1].  Every row must be taken exactly once and no access may leave
[0, n), for empty, ragged and tile-aligned sizes and for any grid.
"""
import itertools

import numpy as np
import pytest

TILE, CC_THREADS, CC_ROWS = 128, 64, 8


def tensor_core_rows(n_tc, grid):
    n_tiles = (n_tc + TILE - 1) // TILE
    rows = []
    for b in range(grid):
        for t in range(b, n_tiles, grid):
            for r in range(TILE):
                row = t * TILE + r
                if row < n_tc:
                    rows.append(row)
    return rows


def cuda_core_rows(n_tc, n, grid):
    n_cc = n - n_tc
    step = CC_THREADS * CC_ROWS
    stride = grid * step
    rows = []
    for b in range(grid):
        for ct in range(CC_THREADS):
            base = b * step + ct
            while base < n_cc:  # the loop condition tests the step's first row
                for j in range(CC_ROWS):
                    i = base + CC_THREADS * j
                    if i < n_cc:
                        rows.append(n_tc + i)
                base += stride
    return rows


@pytest.mark.parametrize("n,grid", list(itertools.product([0, 1, 63, 64, 127, 128, 129, 511, 512, 513, 4097], [1, 3, 152])))
def test_every_row_once(n, grid):
    for n_tc in sorted({0, n, n // 2, min(n, 127), min(n, 129), max(0, n - 1)}):
        rows = tensor_core_rows(n_tc, grid) + cuda_core_rows(n_tc, n, grid)
        assert all(0 <= r < n for r in rows)
        np.testing.assert_array_equal(np.sort(np.array(rows, np.int64)), np.arange(n))


def test_cuda_core_rows_of_a_step_are_coalesced():
    """In one step a warp's 32 lanes read 32 consecutive rows for every j."""
    step_rows = [[ct + CC_THREADS * j for ct in range(32)] for j in range(CC_ROWS)]
    for r in step_rows:
        assert r == list(range(r[0], r[0] + 32))
