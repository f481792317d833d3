"""The screens' tile arithmetic, replayed on the host (no GPU).

The kernels cut bond k's superblock (rows I_{<k} x i_k, columns
i_{k+1} x J_{>k+1}) into CTA tiles; with a subtensor grid (the paper's
process grid of Alg. 3, Sec. 3.2) mode k is split into balanced pieces and no
tile crosses one.  Each tile writes one candidate slot per bond, in a buffer
sized at create time from the rank caps.  ``ttcross_check_tiles`` runs the
kernels' own tile geometry on the host; these tests check, for the batch
recipe's 256 Maxwellians and for ragged shapes, that the tiles cover every
superblock entry exactly once, stay inside their piece, and never outnumber
the candidate slots at any ranks up to the caps.
"""
import itertools

import numpy as np
import pytest

from paper_2407_11290_gb300 import ttcross, workloads


def _check(n, ranks, caps, grid, te, stored, stored_ranks=None):
    tiles, cap, bad = ttcross.check_tiles(n, ranks, caps, grid=grid, tile_edge=te, stored=stored,
                                          stored_ranks=stored_ranks)
    assert bad == 0, (n, ranks, stored_ranks, grid, te)
    return tiles, cap


def test_tile_counts_match_the_plain_cut():
    # no grid: ceil(rows / te) x ceil(cols / te)
    tiles, _ = _check([100, 100], [1], [1], None, 64, False)
    assert list(tiles) == [4]
    tiles, _ = _check([100, 100], [1], [1], None, 32, False)
    assert list(tiles) == [16]
    # grid 3 x 3 on n = 100: pieces 34, 33, 33, one 64-wide tile each
    tiles, _ = _check([100, 100], [1], [1], [3, 3], 64, False)
    assert list(tiles) == [9]
    # 32-wide tiles: two per piece
    tiles, _ = _check([100, 100], [1], [1], [3, 3], 32, False)
    assert list(tiles) == [36]
    # three modes at ranks (5, 7): bond 1 is 1*100 x 100*7, bond 2 is 5*100 x 100*1
    tiles, _ = _check([100, 100, 100], [5, 7], [8, 8], None, 64, False)
    assert list(tiles) == [2 * 11, 8 * 2]


def test_batch_recipe_tiles_cover_and_fit_the_slots():
    """The 256 Maxwellians of the batch workload (d = 4..6, n in
    {32, 48, 64, 96, 128}, rank cap 64): library tiles and grids of 2 and 4
    pieces, both tile edges, ranks from 1 to the caps."""
    rng = np.random.default_rng(7)
    for w in workloads.maxwellian_batch(256):
        n = w["n"]
        d = len(n)
        caps = [64] * (d - 1)
        rank_sets = [[1] * (d - 1), [64] * (d - 1), list(rng.integers(1, 65, d - 1))]
        for grid in (None, [2] * d, [4] * d):
            for ranks in rank_sets:
                for te in (32, 64):
                    tiles, cap = _check(n, ranks, caps, grid, te, False)
                    # the stored form, its residual written one pivot (and
                    # all the way) back
                    back = [max(1, int(x) - 1) for x in ranks]
                    _, cap_st = _check(n, ranks, caps, grid, te, True, back)
                    _check(n, ranks, caps, grid, te, True, [1] * (d - 1))
                    if te == 64:
                        # the slots are sized for 64-wide tiles at the caps
                        assert np.all(tiles <= cap) and np.all(4 * tiles <= cap_st)
                    assert np.all(cap_st == 4 * cap)


@pytest.mark.parametrize("seed", range(4))
def test_ragged_shapes_and_pieces(seed):
    """Small ragged modes, pieces that do not divide them (down to pieces of
    one index), every rank up to the caps on three modes."""
    rng = np.random.default_rng(seed)
    for _ in range(40):
        n = [int(v) for v in rng.integers(1, 140, 3)]
        caps = [int(rng.integers(1, 12)), int(rng.integers(1, 12))]
        grid = [int(rng.integers(0, v + 1)) for v in n] if rng.random() < 0.7 else None
        for r0, r1 in itertools.product(range(1, caps[0] + 1), range(1, caps[1] + 1)):
            for te in (32, 64):
                tiles, cap = _check(n, [r0, r1], caps, grid, te, False)
                if te == 64:
                    assert np.all(tiles <= cap)
                _check(n, [r0, r1], caps, grid, te, True,
                       [int(rng.integers(1, r0 + 1)), int(rng.integers(1, r1 + 1))])


def test_carried_rectangle_counts():
    """Stored form, no grid, n = (100, 100, 100), ranks (5, 7) written at
    (3, 7): bond 1's carried rows are the 100 rows of I_<1 (one 64-row tile
    lies inside), its carried columns 100 * 7 (ten 64-column tiles); the
    check passes and the tile counts are those of the plain cut."""
    tiles, _ = _check([100, 100, 100], [5, 7], [8, 8], None, 64, True, [3, 7])
    assert list(tiles) == [2 * 11, 8 * 2]


def test_arguments_checked():
    with pytest.raises(ttcross.TTCError):
        ttcross.check_tiles([10, 10], [3], [2])           # rank above its cap
    with pytest.raises(ttcross.TTCError):
        ttcross.check_tiles([10, 10], [1], [1], tile_edge=48)
    with pytest.raises(ttcross.TTCError):
        ttcross.check_tiles([10, 10], [1], [1], grid=[11, 1])
    with pytest.raises(ttcross.TTCError):
        ttcross.check_tiles([10, 10, 10], [2, 2], [4, 4], stored_ranks=[3, 1])  # above r
