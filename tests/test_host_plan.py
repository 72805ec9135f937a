"""Host logic of the stepping launch, exercised without a GPU: the work
partition of the (unit, level) sequence over the blocks (sfm_plan_pieces)."""
import os

import numpy as np
import pytest


@pytest.fixture(scope="module")
def sfm():
    from paper_1406_6923_gb300 import _build, sfm as mod
    if not os.path.exists(mod.LIB_PATH):
        _build.build()
    mod.load()
    return mod


def _check_partition(ptr, pieces, nunits, k_sub, grid):
    nsub = len(k_sub)
    assert ptr[0] == 0 and ptr[-1] == len(pieces)
    assert np.all(np.diff(ptr) >= 0)
    seen = {}
    for u, j0, j1 in pieces:
        assert 0 <= u < nunits and 0 <= j0 < j1 <= k_sub[u % nsub]
        # never cut at level 1: the piece reading the face levels owns them
        assert j0 != 1
        for j in range(j0, j1):
            seen[(u, j)] = seen.get((u, j), 0) + 1
    want = {(u, j) for u in range(nunits) for j in range(k_sub[u % nsub])}
    assert set(seen) == want and all(v == 1 for v in seen.values())
    # pieces of one block are in unit-major order
    for c in range(grid):
        blk = pieces[ptr[c]:ptr[c + 1]]
        keys = [(int(u), int(j0)) for u, j0, _ in blk]
        assert keys == sorted(keys)


def test_random_partitions_cover_every_level_once(sfm):
    rng = np.random.default_rng(7)
    for _ in range(60):
        nsub = int(rng.integers(1, 30))
        nshots = int(rng.integers(1, 4))
        k = rng.integers(1, 25, size=nsub)
        total = int(k.sum()) * nshots
        grid = int(rng.integers(1, total + 5))
        ptr, pieces = sfm.sfm_plan_pieces(nsub * nshots, k, grid)
        assert len(ptr) == grid + 1
        _check_partition(ptr, pieces, nsub * nshots, k, grid)


def test_uniform_units_with_spare_blocks_are_not_cut(sfm):
    """512 units of 16 levels on 608 blocks: the cost model (extra pieces and
    face work cost about two levels each) keeps every unit whole."""
    ptr, pieces = sfm.sfm_plan_pieces(512, np.full(512, 16), 608)
    assert len(pieces) == 512
    assert np.all(pieces[:, 1] == 0) and np.all(pieces[:, 2] == 16)
    assert np.max(np.diff(ptr)) == 1


def test_plan_is_deterministic_and_rejects_bad_input(sfm):
    k = np.array([3, 1, 7, 2])
    a = sfm.sfm_plan_pieces(8, k, 5)
    b = sfm.sfm_plan_pieces(8, k, 5)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    with pytest.raises(sfm.SfmError):
        sfm.sfm_plan_pieces(7, k, 5)          # not a whole number of shots
    with pytest.raises(sfm.SfmError):
        sfm.sfm_plan_pieces(8, np.array([3, 0, 7, 2]), 5)
