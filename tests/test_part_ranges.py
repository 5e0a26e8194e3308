"""Host-only checks of the one-reduction PCG pass's part table (mqs_part_ranges: no
CUDA call).  The kernel walks each part's plane-tiles column by column and starts a
segment, with one warm-up plane, at the part's first tile, at every column's first
plane and after 32 planes of a column; the table must cover every tile once, in
order, and minimise the largest part cost.  The optimum is checked against an
exhaustive dynamic program over all contiguous splits on small grids, written
here from that cost model alone."""
import functools

import numpy as np
import pytest

MAX_SEG = 32       # planes per segment of the stencil march
TILE_X, TILE_Y = 32, 4


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__ as g
    g.build()
    import paper_1611_06721_gb300 as p
    return p


def n_tiles(n):
    return ((n + TILE_X - 1) // TILE_X) * ((n + TILE_Y - 1) // TILE_Y) * n


def part_cost(u0, u1, n):
    """Tiles plus warm-up planes of the range [u0, u1), walked as the kernel walks it."""
    cost, u = 0, u0
    while u < u1:
        k = u % n
        seg = min(n - k, u1 - u, MAX_SEG)
        cost += seg + 1
        u += seg
    return cost


def best_max_cost(n, parts):
    """The smallest largest part cost over every split of the tiles into `parts`
    contiguous (possibly empty) ranges, by exhaustive dynamic programming."""
    T = n_tiles(n)

    @functools.lru_cache(maxsize=None)
    def f(u, p):
        if u == T:
            return 0
        if p == 0:
            return float("inf")
        return min(max(part_cost(u, v, n), f(v, p - 1)) for v in range(u + 1, T + 1))

    return f(0, parts)


def check_table(t, n, parts):
    T = n_tiles(n)
    assert t.shape == (parts, 2)
    assert t[0, 0] == 0
    assert np.all(t[:, 0] <= t[:, 1])
    assert np.all(t[1:, 0] == t[:-1, 1])          # contiguous, in order
    assert t[-1, 1] == T                          # every tile once
    return max(part_cost(int(a), int(b), n) for a, b in t)


@pytest.mark.parametrize("n,nblk,groups", [(8, 2, 2), (8, 3, 2), (9, 2, 3), (12, 2, 2), (16, 3, 2), (5, 1, 3)])
def test_part_table_is_an_optimal_contiguous_split(pkg, n, nblk, groups):
    from paper_1611_06721_gb300.binding import part_ranges
    t = part_ranges(n, nblk, groups)
    worst = check_table(t, n, nblk * groups)
    assert worst == best_max_cost(n, nblk * groups)


@pytest.mark.parametrize("n,nblk,groups", [(64, 152, 2), (64, 152, 3), (128, 152, 2), (40, 152, 2), (35, 7, 2)])
def test_part_table_beats_the_even_split(pkg, n, nblk, groups):
    # at the benchmark's shape (64^3, one block of two groups per SM) the largest part
    # costs 8 (the even split of 6.74 tiles per part: 9)
    from paper_1611_06721_gb300.binding import part_ranges
    parts = nblk * groups
    t = part_ranges(n, nblk, groups)
    worst = check_table(t, n, parts)
    T = n_tiles(n)
    even = max(part_cost(T * p // parts, T * (p + 1) // parts, n) for p in range(parts))
    assert worst <= even
    # no part can cost less than its share of the tiles plus one warm-up plane
    assert worst >= -(-T // parts) + 1
    if (n, nblk, groups) == (64, 152, 2):
        assert (worst, even) == (8, 9)


def test_part_table_more_parts_than_tiles(pkg):
    # a tiny grid on many parts: the tiles go one per part from the front, the rest are empty
    from paper_1611_06721_gb300.binding import part_ranges
    t = part_ranges(3, 4, 2)                  # 1 x 1 tile columns x 3 planes = 3 tiles, 8 parts
    check_table(t, 3, 8)
    assert [tuple(r) for r in t] == [(0, 1), (1, 2), (2, 3)] + [(3, 3)] * 5


def test_part_table_rejects_bad_arguments(pkg):
    import ctypes as C
    from paper_1611_06721_gb300.binding import part_ranges
    lib = pkg.load()
    buf = (C.c_int * 4)()
    assert lib.mqs_part_ranges(0, 1, 2, buf) == -1          # MQS_ERR_ARG
    assert lib.mqs_part_ranges(8, 0, 2, buf) == -1
    assert lib.mqs_part_ranges(8, 1, 2, None) == -1
    with pytest.raises(ValueError):
        part_ranges(8, 0)
