"""Shape checks for the seeded input generators (no GPU, no ranking)."""
import numpy as np

import gen


def _heads(succ):
    n = succ.shape[0]
    hp = np.zeros(n, dtype=bool)
    hp[succ[succ != np.arange(n)]] = True
    return np.flatnonzero(~hp)


def test_random_list_is_one_list():
    succ = gen.random_list(1000, 1)
    assert succ.dtype == np.uint32
    assert (succ == np.arange(1000)).sum() == 1
    assert _heads(succ).shape[0] == 1
    assert np.array_equal(gen.random_list(1000, 1), succ)      # seeded
    assert not np.array_equal(gen.random_list(1000, 2), succ)


def test_locality_stays_in_windows():
    n, w = 256 * 10 + 37, 256
    order = gen.locality_order(n, 5, w)
    assert np.array_equal(np.sort(order), np.arange(n))
    assert (order // w == np.arange(n) // w).all()
    assert not np.array_equal(order, np.arange(n))


def test_forest_shape():
    succ, nlists = gen.forest(1 << 15, 2, n_long=4, long_len=1 << 11, mean_short=64)
    assert (succ == np.arange(succ.shape[0])).sum() == nlists
    assert _heads(succ).shape[0] == nlists
    assert nlists > 4 + (1 << 14) // 64 // 2


def test_euler_tour_is_a_list():
    parent = gen.random_recursive_tree(1000, 3)
    assert (parent[1:] < np.arange(1, 1000)).all()
    succ, w = gen.euler_tour(parent)
    assert succ.shape[0] == 2 * 999 and w.sum() == 0
    assert (succ == np.arange(succ.shape[0])).sum() == 1
    assert _heads(succ).tolist() == [0]          # the tour starts with down(first child of 0)


def test_batch_lengths_log_uniform():
    lens = gen.batch_lengths(4096, 7, 8.0, 22.0)
    assert lens.min() >= 256 and lens.max() <= 1 << 22
    # mean of floor(2^U), U ~ U[8,22], is about (2^22 - 2^8) / (14 ln 2)
    expect = ((1 << 22) - 256) / (14 * np.log(2))
    assert abs(lens.mean() / expect - 1) < 0.1
    offsets, succ, w = gen.batch_instances(5, 3, 2.0, 6.0)
    assert offsets[0] == 0 and offsets[-1] == succ.shape[0] == w.shape[0]
    for j in range(5):
        local = succ[offsets[j]:offsets[j + 1]]
        assert local.max() < offsets[j + 1] - offsets[j]


def test_serving_trace():
    t, sizes, kinds, seeds = gen.serving_trace(500, 9, rate_per_s=100.0)
    assert (np.diff(t) >= 0).all() and t[0] == 0
    assert sizes.min() >= 1 << 10 and sizes.max() <= 1 << 26
    assert set(kinds) <= {"random", "locality"}
