"""Pins of the oracle's levels of G/k-normalised expression (state labels
and multistability from levels; Sec. 2.1.3 analysis, Sec. 3.1) against
inputs whose bins, valleys and labels are known by construction.

The reading pinned here: one histogram of v = (x k) / G over all nodes of
all converged solves, n_bins equal bins on [0, 1]; binomial smoothing of
half-width m; modes merged by persistence -- valleys (runs of equal
smoothed counts lower than both neighbours) from the highest down, each
absorbing the group of modes with the lower highest peak, a boundary (the
run's middle) when twice the valley's count is at most that peak and the
peak reaches 1/64 of the highest count; levels = boundaries below a
value's bin; labels pack the levels node by node.
"""
import numpy as np
import pytest

import oracle as O



def states_from_v(v, G, k):
    """x with (x k) / G == v exactly (G and k powers of two)."""
    return v * G[:, None, :] / k[:, None, :]


def pow2_params(S, N, rng):
    G = 2.0 ** rng.integers(0, 7, (S, N)).astype(float)
    k = 2.0 ** -rng.integers(0, 4, (S, N)).astype(float)
    return G, k


def test_bin_edges_and_clamping():
    B = 100
    assert O.gk_bin(0.0, 1.0, 1.0, B) == 0
    assert O.gk_bin(-3.0, 1.0, 1.0, B) == 0
    assert O.gk_bin(0.5, 1.0, 1.0, B) == 50
    assert O.gk_bin(0.015625, 1.0, 1.0, B) == 1          # 1.5625 bins
    assert O.gk_bin(1.0, 1.0, 1.0, B) == B - 1
    assert O.gk_bin(7.0, 1.0, 1.0, B) == B - 1
    assert O.gk_bin(np.nan, 1.0, 1.0, B) == 0
    # (x k) / G: x = 24, k = 0.5, G = 32 -> v = 0.375 -> bin 37 of 100, 3 of 8
    assert O.gk_bin(24.0, 0.5, 32.0, 100) == 37
    assert O.gk_bin(24.0, 0.5, 32.0, 8) == 3


def test_histogram_counts_by_construction():
    rng = np.random.default_rng(0)
    S, I, N, B = 7, 5, 4, 16
    G, k = pow2_params(S, N, rng)
    bins = rng.integers(0, B, (S, I, N))
    v = (bins + 0.5) / B                                  # bin centres, exact
    status = (rng.uniform(size=(S, I)) < 0.3).astype(np.uint8)
    counts = O.gk_histogram(states_from_v(v, G, k), status, G, k, B)
    want = np.zeros(B, dtype=np.uint64)
    for s in range(S):
        for c in range(I):
            if status[s, c] == 0:
                for i in range(N):
                    want[bins[s, c, i]] += 1
    assert np.array_equal(counts, want)
    assert counts.sum() == N * int((status == 0).sum())
    # accumulation into an existing histogram
    again = O.gk_histogram(states_from_v(v, G, k), status, G, k, B, counts=counts.copy())
    assert np.array_equal(again, 2 * want)


def bumps(B, centres, width, height):
    c = np.zeros(B, dtype=np.uint64)
    for ctr, h in zip(centres, height):
        for b in range(ctr - width, ctr + width + 1):
            c[b] += h
    return c


def test_unimodal_and_flat_have_no_boundary():
    assert O.level_boundaries(bumps(100, [50], 8, [1000])).size == 0
    assert O.level_boundaries(np.full(100, 7, dtype=np.uint64)).size == 0
    assert O.level_boundaries(np.zeros(100, dtype=np.uint64)).size == 0


def test_bimodal_gap_middle():
    # modes on bins [5, 15] and [65, 75]; smoothing of half-width 4 spreads
    # them to [1, 19] and [61, 79], so the valley of zeros is [20, 60] and
    # its middle bin is 40
    c = bumps(100, [10, 70], 5, [500, 300])
    assert list(O.level_boundaries(c, m=4)) == [40]
    # without smoothing the zero run is [16, 64]: middle 40 as well
    assert list(O.level_boundaries(c, m=0)) == [40]


def test_trimodal_and_max_boundaries():
    c = bumps(100, [10, 50, 90], 4, [400, 200, 400])
    assert list(O.level_boundaries(c, m=4)) == [30, 70]
    # four modes, the deepest valleys kept first: valleys between modes at
    # 10|35 (zeros), 35|60 (shallower: the modes overlap), 60|85 (zeros)
    c4 = bumps(100, [10, 35, 60, 85], 4, [400, 400, 400, 400])
    c4[40:56] += 150                                      # middle valley: a plateau of 150
    got = O.level_boundaries(c4, m=0, max_b=2)
    assert list(got) == [22, 72]                          # zero runs [15, 30] and [65, 80]
    assert list(O.level_boundaries(c4, m=0, max_b=3)) == [22, 47, 72]


def test_depth_rule_exact_half():
    # no smoothing (m = 0): peaks 100 and 60, valley count 30 = 60 / 2 is a
    # boundary, 31 is not
    c = np.zeros(20, dtype=np.uint64)
    c[4], c[10], c[15] = 100, 30, 60
    c[5:10] = 40; c[11:15] = 40
    assert list(O.level_boundaries(c, m=0)) == [10]
    c[10] = 31
    assert O.level_boundaries(c, m=0).size == 0
    # a valley touching an edge is not a valley
    e = np.zeros(10, dtype=np.uint64); e[5] = 9
    assert O.level_boundaries(e, m=0).size == 0


def test_level_states_labels_by_construction():
    rng = np.random.default_rng(3)
    S, I, N, B = 6, 8, 5, 100
    G, k = pow2_params(S, N, rng)
    bounds = np.array([30, 70], dtype=np.int32)          # three levels, two bits a node
    levels = rng.integers(0, 3, (S, I, N))
    # a bin inside each level: level 0 -> bin 12, 1 -> bin 50, 2 -> bin 88;
    # a value in a boundary's own bin takes the lower level
    rep_bin = np.array([12, 50, 88])
    v = (rep_bin[levels] + 0.25) / B
    v[0, 0, 0] = (30 + 0.5) / B; levels[0, 0, 0] = 0
    v[0, 1, 1] = (31 + 0.5) / B; levels[0, 1, 1] = 1
    status = np.zeros((S, I), dtype=np.uint8)
    status[2, 3] = 1; status[4, :] = 1
    labels, ns, mh = O.level_states(states_from_v(v, G, k), status, G, k, bounds, B)
    for s in range(S):
        want = set()
        for c in range(I):
            if status[s, c]:
                assert labels[s, c] == np.iinfo(np.uint64).max
                continue
            lab = sum(int(levels[s, c, i]) << (2 * i) for i in range(N))
            assert int(labels[s, c]) == lab
            want.add(lab)
        assert ns[s] == len(want)
    assert mh.sum() == S and mh[0] == 1                   # set 4: nothing converged
    assert np.array_equal(mh, np.bincount(ns, minlength=I + 1).astype(np.uint64))


def test_level_states_width_limit_and_no_boundaries():
    rng = np.random.default_rng(4)
    G, k = pow2_params(2, 40, rng)
    v = rng.uniform(0, 1, (2, 3, 40))
    st = np.zeros((2, 3), dtype=np.uint8)
    # 40 nodes x 2 bits > 64: refused
    assert O.level_states(states_from_v(v, G, k), st, G, k, np.array([30, 70], np.int32)) is None
    # 40 nodes x 1 bit fits; with no boundary every label is 0, one state a set
    labels, ns, mh = O.level_states(states_from_v(v, G, k), st, G, k, np.array([], np.int32))
    assert np.all(labels == 0) and np.all(ns == 1) and mh[1] == 2


def test_binomial_smoothing_weights():
    # spikes of 100 at bins 40 and 48, half-width 4 (weights C(8, j)): the
    # smoothed counts are C(8, 4 + 44 - 40) 100 + C(8, 4 + 44 - 48) 100 = 200
    # at bin 44 and C(8, 7) 100 = 800 beside it, so the valley is bin 44;
    # spikes 10 bins apart leave a zero at bin 45, the valley's only bin
    c = np.zeros(100, dtype=np.uint64)
    c[40] = c[48] = 100
    assert list(O.level_boundaries(c, m=4)) == [44]
    c[:] = 0
    c[40] = c[50] = 100
    assert list(O.level_boundaries(c, m=4)) == [45]
    # with m = 1 (weights 1, 2, 1) the spikes 8 apart leave zeros on [42, 46]
    c[:] = 0
    c[40] = c[48] = 100
    assert list(O.level_boundaries(c, m=1)) == [44]


def test_noisy_middle_gives_one_boundary_at_its_lowest_point():
    # modes at bins 5-15 and 80-90; between them a sparse, wiggly region
    # (peaks of 40-60, valleys of 25-35) whose lowest point is bin 51 (10):
    # the wiggles are absorbed at valleys too high for them, the right mode
    # at the lowest valley
    c = np.zeros(100, dtype=np.uint64)
    c[5:16] = 1000
    c[80:91] = 500
    mid = np.arange(20, 76)
    c[20:76] = (45 + 12 * np.sin(mid * 1.3)).astype(np.uint64)
    c[16:20] = [400, 200, 100, 60]                        # the modes' flanks
    c[76:80] = [60, 100, 200, 400]
    c[51] = 10
    assert list(O.level_boundaries(c, m=0)) == [51]
    # the rule with global side maxima alone would also cut at the wiggles
    wiggle_valleys = [b for b in range(21, 75) if c[b] < c[b - 1] and c[b] < c[b + 1]]
    assert len(wiggle_valleys) > 5


def test_minimum_peak_height():
    c = np.zeros(100, dtype=np.uint64)
    c[8:13] = 10000
    c[90] = 3                      # a stray count far in the tail: 3 < 10000 / 64
    assert O.level_boundaries(c, m=0).size == 0
    c[90] = 157                    # 64 * 157 >= 10000: a mode of its own
    assert list(O.level_boundaries(c, m=0)) == [51]


def test_equal_peaks_absorb_the_right_one():
    # equal peaks at 10 and 40, a lower one at 70; valleys at 25 (count 1)
    # and 55 (count 0): the valley at 25 joins the equal peaks (the right one
    # is absorbed), the one at 55 the lower peak
    c = np.zeros(80, dtype=np.uint64)
    c[10] = c[40] = 100
    c[70] = 60
    c[11:40] = 1
    assert list(O.level_boundaries(c, m=0)) == [25, 55]
