"""Pins of the oracle's neighbour lists (the list of all particles within a
given radius of each sink, Sec. 1 and Sec. 3 of the paper).

Positions on an integer grid make every r.r exact, so the lists must equal the
ones scipy's pairwise distances give, element for element; symmetry, the
strict inequality, self-exclusion and the overflow rule are checked on top."""
import numpy as np
import pytest

scipy_spatial = pytest.importorskip("scipy.spatial")


def _grid_state(n, seed, span=12):
    rng = np.random.default_rng(seed)
    x = rng.integers(-span, span + 1, size=(n, 3)).astype(np.float64)
    ids = rng.permutation(10 * n)[:n].astype(np.int32)
    return ids, x


def _reference(ids_i, xi, h2, ids_j, xj):
    d2 = scipy_spatial.distance.cdist(xi, xj, "sqeuclidean")
    out = []
    for k in range(len(ids_i)):
        sel = (d2[k] < h2[k]) & (ids_j != ids_i[k])
        out.append(np.sort(ids_j[sel]))
    return out


def test_lists_match_pairwise_distances(oracle_mod):
    ids, x = _grid_state(400, 1)
    h2 = np.random.default_rng(2).integers(0, 60, size=400) + 0.5  # no ties with integer r.r
    cnt, lst = oracle_mod.neighbours(ids, x, h2, ids, x, 400)
    ref = _reference(ids, x, h2, ids, x)
    for k in range(400):
        assert cnt[k] == len(ref[k])
        assert np.array_equal(lst[k, :cnt[k]], ref[k])


def test_strict_radius_and_self(oracle_mod):
    ids = np.array([7, 3, 9], np.int32)
    x = np.array([[0.0, 0, 0], [3.0, 4, 0], [0, 0, 1.0]])
    h2 = np.array([25.0, 25.0, 25.0])  # particle 3 sits exactly at r = 5 from 7
    cnt, lst = oracle_mod.neighbours(ids, x, h2, ids, x, 4)
    assert list(cnt) == [1, 0, 1]          # r.r = 25 is not < 25; the self pair never counts
    assert lst[0, 0] == 9 and lst[2, 0] == 7
    cnt, _ = oracle_mod.neighbours(ids, x, np.nextafter(h2, np.inf), ids, x, 4)
    assert list(cnt) == [2, 1, 1]          # 3 and 9 are sqrt(26) apart


def test_symmetric_for_equal_radii(oracle_mod):
    ids, x = _grid_state(300, 3)
    h2 = np.full(300, 40.5)
    cnt, lst = oracle_mod.neighbours(ids, x, h2, ids, x, 300)
    pos = {int(v): k for k, v in enumerate(ids)}
    pairs = {(int(ids[k]), int(v)) for k in range(300) for v in lst[k, :cnt[k]]}
    assert pairs == {(b, a) for a, b in pairs}
    assert all(pos[a] != pos[b] for a, b in pairs)


def test_overflow_keeps_smallest_ids_and_true_count(oracle_mod):
    ids, x = _grid_state(200, 5, span=3)
    h2 = np.full(200, 12.5)
    full_cnt, full = oracle_mod.neighbours(ids, x, h2, ids, x, 200)
    cnt, lst = oracle_mod.neighbours(ids, x, h2, ids, x, 5)
    assert np.array_equal(cnt, full_cnt)
    over = cnt > 5
    assert over.any()
    for k in np.flatnonzero(over):
        assert np.array_equal(lst[k], full[k, :5])


def test_zero_radius_and_separate_source_set(oracle_mod):
    ids, x = _grid_state(50, 7)
    cnt, _ = oracle_mod.neighbours(ids, x, np.zeros(50), ids, x, 8)
    assert not cnt.any()
    # sinks need not be sources: a sink far from every source has no neighbours
    far = np.array([[1e6, 0.0, 0.0]])
    cnt, _ = oracle_mod.neighbours(np.array([-5], np.int32), far, np.array([100.0]), ids, x, 8)
    assert cnt[0] == 0
