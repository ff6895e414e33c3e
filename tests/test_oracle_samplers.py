"""Pins of the oracle's parameter distributions besides Table 1's (the
paper's other samplers, Sec. 2.1.2): log-uniform, normal and log-normal
over a class's range, checked against scipy's distributions, plus the
Box-Muller construction on the draw's two halves."""
import numpy as np
import pytest
from scipy import stats

import oracle as O
from paper_2503_18356_gb300 import workloads as W

NET = O.Network(*W.random_network(3, 3, 4, 2, 0).edges())
S = 20000


def draw(**dist):
    r = O.default_ranges(median_samples=2000, **dist)
    return O.sample_params(NET, 9, S, ranges=r), r


def test_log_uniform():
    p, r = draw(dist_G=1, dist_lam_act=1)
    g = np.log(p.G.ravel())
    assert np.all((p.G >= r.G_min) & (p.G <= r.G_max))
    assert stats.kstest(g, stats.uniform(np.log(r.G_min), np.log(r.G_max) - np.log(r.G_min)).cdf).pvalue > 1e-3
    act = np.tile(NET.sign > 0, (S, 1))
    la = np.log(p.lam[act])
    assert stats.kstest(la, stats.uniform(np.log(r.lam_act_min),
                                          np.log(r.lam_act_max) - np.log(r.lam_act_min)).cdf).pvalue > 1e-3


@pytest.mark.parametrize("field,dist,lo,hi", [("k", 2, 0.1, 1.0), ("G", 3, 1.0, 100.0)])
def test_normal_and_log_normal_clamped_at_three_sd(field, dist, lo, hi):
    p, r = draw(**{"dist_" + field: dist})
    x = getattr(p, field).ravel()
    y = np.log(x) if dist == 3 else x
    a, b = (np.log(lo), np.log(hi)) if dist == 3 else (lo, hi)
    mid, sd = (a + b) / 2, (b - a) / 6
    assert np.all((x >= lo) & (x <= hi))
    inner = y[(y > a) & (y < b)]
    ks = stats.kstest(inner, stats.truncnorm(-3, 3, loc=mid, scale=sd).cdf)
    assert ks.pvalue > 1e-3, ks
    # the clamps hold the tails beyond three standard deviations: 0.135 % a side
    assert abs(np.mean(y <= a) - stats.norm.cdf(-3)) < 0.0015
    assert abs(np.mean(y >= b) - stats.norm.cdf(-3)) < 0.0015


def test_inhibiting_fold_change_distributions():
    p0, r = draw()
    inh = np.tile(NET.sign < 0, (S, 1))
    # Table 1: 1 / U[1, 100] -- its median is 1 / 50.5
    assert abs(np.median(p0.lam[inh]) - 1 / 50.5) < 0.002
    p1, _ = draw(dist_lam_inh=1)
    li = np.log(p1.lam[inh])
    assert stats.kstest(li, stats.uniform(np.log(0.01), -np.log(0.01)).cdf).pvalue > 1e-3


def test_box_muller_halves_are_independent_normals():
    # normal draws of G and k share nothing but come from separate draws;
    # within one draw the two halves make one deviate: check the deviates'
    # moments and that G and k of a set are uncorrelated
    p, r = draw(dist_G=2, dist_k=2)
    zg = (p.G.ravel() - 50.5) / (99 / 6)
    zk = (p.k.ravel() - 0.55) / (0.9 / 6)
    assert abs(zg.mean()) < 0.03 and abs(zg.std() - 0.986) < 0.03
    assert abs(np.corrcoef(zg, zk)[0, 1]) < 0.03


# ---------------------------------------------------------------- Latin hypercube
@pytest.mark.parametrize("S", [1, 2, 3, 5, 17, 64, 100, 1000, 4097])
def test_lhs_stratum_is_a_permutation(S):
    # brute force: for each draw index the map s -> stratum is a bijection
    # of [0, S), whatever S (power of two or not, cycle walking included)
    for d in (0, 1, 7, 123456):
        p = [O.lhs_stratum(2002, d, s, S) for s in range(S)]
        assert sorted(p) == list(range(S)), (S, d)


def test_lhs_strata_differ_between_draws_and_seeds():
    S = 1000
    a = np.array([O.lhs_stratum(1, 0, s, S) for s in range(S)])
    b = np.array([O.lhs_stratum(1, 1, s, S) for s in range(S)])
    c = np.array([O.lhs_stratum(2, 0, s, S) for s in range(S)])
    assert not np.array_equal(a, np.arange(S))
    # independent permutations: rank correlation within a few 1 / sqrt(S)
    for x, y in ((a, b), (a, c)):
        assert abs(np.corrcoef(x, y)[0, 1]) < 4 / np.sqrt(S)


def lhs_draw(S, **dist):
    r = O.default_ranges(median_samples=2000, lhs_sets=S, **dist)
    return O.sample_params(NET, 11, S, ranges=r), r


def order_in_strata(v, lo, hi, S):
    """The i-th smallest of S values lies in the i-th of S equal strata of
    [lo, hi]: one value per stratum, the Latin-hypercube property."""
    z = (np.sort(v) - lo) / (hi - lo) * S
    i = np.arange(S)
    return np.all(z >= i - 1e-9) and np.all(z <= i + 1 + 1e-9)


@pytest.mark.parametrize("S", [1, 7, 500])
def test_lhs_one_value_per_stratum_in_every_dimension(S):
    p, r = lhs_draw(S)
    for i in range(NET.n_nodes):
        assert order_in_strata(p.G[:, i], r.G_min, r.G_max, S)
        assert order_in_strata(p.k[:, i], r.k_min, r.k_max, S)
    for e in range(NET.n_edges):
        if NET.sign[e] > 0:
            assert order_in_strata(p.lam[:, e], r.lam_act_min, r.lam_act_max, S)
        else:
            # Table 1's inhibiting fold change is uniform in the inverse range
            assert order_in_strata(1 / p.lam[:, e], 1 / r.lam_inh_max, 1 / r.lam_inh_min, S)


def test_lhs_log_uniform_strata_and_hill_coefficients():
    S = 600
    p, r = lhs_draw(S, dist_G=1, dist_lam_act=1)
    for i in range(NET.n_nodes):
        assert order_in_strata(np.log(p.G[:, i]), np.log(r.G_min), np.log(r.G_max), S)
    act = NET.sign > 0
    for e in np.flatnonzero(act):
        assert order_in_strata(np.log(p.lam[:, e]), np.log(r.lam_act_min), np.log(r.lam_act_max), S)
    # n is stratified too: S divisible by the n_max - n_min + 1 values, so
    # every value is taken exactly S / 6 times in every edge
    cnt = r.n_max - r.n_min + 1
    for e in range(NET.n_edges):
        assert np.array_equal(np.bincount(p.n[:, e] - r.n_min, minlength=cnt), np.full(cnt, S // cnt))


def test_lhs_thresholds_stratified_before_the_source_median_scale():
    # T = u' M(source), u' over the threshold's range and M the median of
    # the source's in-degree class, the same for every set: T / M is
    # stratified
    S = 300
    p, r = lhs_draw(S)
    for e in range(NET.n_edges):
        j = NET.src[e]
        a = int(np.sum((NET.dst == j) & (NET.sign > 0)))
        b = int(np.sum((NET.dst == j) & (NET.sign < 0)))
        assert order_in_strata(p.T[:, e] / O.median(a, b, r), r.thr_lo, r.thr_hi, S)


def test_lhs_sets_split_across_calls_equal_one_call():
    # counter-based: sets [0, S) drawn in two calls (set0 = 0 and S / 2)
    # equal one call, the permutation depends on S, not on the call
    S = 200
    r = O.default_ranges(median_samples=2000, lhs_sets=S)
    whole = O.sample_params(NET, 5, S, ranges=r)
    a = O.sample_params(NET, 5, S // 2, set0=0, ranges=r)
    b = O.sample_params(NET, 5, S // 2, set0=S // 2, ranges=r)
    for f in ("G", "k", "T", "lam", "n"):
        assert np.array_equal(getattr(whole, f), np.concatenate([getattr(a, f), getattr(b, f)])), f


def test_lhs_off_is_the_plain_sampler():
    r0 = O.default_ranges(median_samples=2000)
    r1 = O.default_ranges(median_samples=2000, lhs_sets=0)
    a, b = O.sample_params(NET, 3, 50, ranges=r0), O.sample_params(NET, 3, 50, ranges=r1)
    for f in ("G", "k", "T", "lam", "n"):
        assert np.array_equal(getattr(a, f), getattr(b, f))


# ---------------------------------------------------------------- Sobol
TAB = None


def sobol_tab():
    global TAB
    if TAB is None:
        TAB = W.sobol_direction_table()
    return TAB


def test_sobol_points_equal_scipy_unscrambled():
    # the plain Sobol sequence from its definition (Bratley-Fox direction
    # integers, Gray-code order) against scipy's generator on the same
    # Joe-Kuo table: every coordinate of 290 dimensions (the 22-node
    # network's 2N + 3E draws) for points 0..511, and from an offset
    qmc = pytest.importorskip("scipy.stats").qmc
    r = O.default_ranges(sobol=1, sobol_table=sobol_tab())
    D, n = 290, 512
    ref = np.rint(qmc.Sobol(D, scramble=False, bits=32).random(n) * 2.0**32).astype(np.uint64)
    mine = np.array([[O.sobol_x(r, 0, d, s) for d in range(D)] for s in range(n)], dtype=np.uint64)
    assert np.array_equal(ref, mine)
    g = qmc.Sobol(40, scramble=False, bits=32)
    g.fast_forward(100_000)
    ref = np.rint(g.random(16) * 2.0**32).astype(np.uint64)
    mine = np.array([[O.sobol_x(r, 0, d, 100_000 + s) for d in range(40)] for s in range(16)], dtype=np.uint64)
    assert np.array_equal(ref, mine)


def elementary_intervals_hold_one_point(u, v, m):
    """(0, m, 2)-net in base 2: every box [a 2^-i, (a+1) 2^-i) x
    [b 2^-(m-i), (b+1) 2^-(m-i)) of area 2^-m holds exactly one point."""
    for i in range(m + 1):
        a = np.floor(u * 2**i).astype(np.int64)
        b = np.floor(v * 2**(m - i)).astype(np.int64)
        cnt = np.bincount(a * 2**(m - i) + b, minlength=2**m)
        if not np.all(cnt == 1):
            return False
    return True


@pytest.mark.parametrize("mode", [1, 2])
def test_sobol_net_and_stratification(mode):
    # the first 2^m points: dimensions 0 and 1 form a (0, m, 2)-net, and
    # every one-dimensional projection holds one point per 2^-m stratum;
    # both survive the linear scramble and the digital shift
    m = 8
    r = O.default_ranges(sobol=mode, sobol_table=sobol_tab())
    X = np.array([[O.sobol_x(r, 77, d, s) for d in range(60)] for s in range(2**m)], dtype=np.float64) * 2.0**-32
    assert elementary_intervals_hold_one_point(X[:, 0], X[:, 1], m)
    for d in range(60):
        assert np.array_equal(np.sort(np.floor(X[:, d] * 2**m)), np.arange(2**m)), d


def test_sobol_scramble_depends_on_the_seed_only_when_scrambled():
    t = sobol_tab()
    plain = O.default_ranges(sobol=1, sobol_table=t)
    scr = O.default_ranges(sobol=2, sobol_table=t)
    pts = lambda r, seed: np.array([[O.sobol_x(r, seed, d, s) for d in range(20)] for s in range(256)])
    assert np.array_equal(pts(plain, 1), pts(plain, 2))
    a, b = pts(scr, 1), pts(scr, 2)
    assert not np.array_equal(a, b) and not np.array_equal(a, pts(plain, 1))
    # a randomised net: coordinates average 1/2 within 1/(2 sqrt(3) 16)-ish
    assert np.all(np.abs(a.mean(axis=0) * 2.0**-32 - 0.5) < 0.01)


def test_sobol_sets_one_value_per_stratum():
    S = 256
    r = O.default_ranges(median_samples=2000, sobol=2, sobol_table=sobol_tab())
    p = O.sample_params(NET, 13, S, ranges=r)
    for i in range(NET.n_nodes):
        assert order_in_strata(p.G[:, i], r.G_min, r.G_max, S)
        assert order_in_strata(p.k[:, i], r.k_min, r.k_max, S)
    cnt = r.n_max - r.n_min + 1
    for e in range(NET.n_edges):
        if NET.sign[e] > 0:
            assert order_in_strata(p.lam[:, e], r.lam_act_min, r.lam_act_max, S)
        else:
            assert order_in_strata(1 / p.lam[:, e], 1 / r.lam_inh_max, 1 / r.lam_inh_min, S)
        # n = n_min + floor(u count): each value S / count sets, within 2
        # for the strata that straddle the value's two boundaries
        c = np.bincount(p.n[:, e] - r.n_min, minlength=cnt)
        assert np.all(np.abs(c - S / cnt) <= 2)
    # sets drawn in two calls equal one call (point index = set index)
    a = O.sample_params(NET, 13, S // 2, set0=0, ranges=r)
    b = O.sample_params(NET, 13, S // 2, set0=S // 2, ranges=r)
    assert np.array_equal(p.G, np.concatenate([a.G, b.G]))


# ---------------------------------------------------------------- per-parameter range table
def class_table(net, r):
    """The per-parameter rows that the class fields of r describe."""
    N, E = net.n_nodes, net.n_edges
    t = np.zeros(2 * N + 3 * E, dtype=O.PARAM_ROW)
    t[:N] = (r.dist_G, 0, r.G_min, r.G_max)
    t[N:2 * N] = (r.dist_k, 0, r.k_min, r.k_max)
    t[2 * N:2 * N + E] = (0, 0, r.thr_lo, r.thr_hi)
    for e in range(E):
        t[2 * N + E + e] = ((r.dist_lam_act, 0, r.lam_act_min, r.lam_act_max) if net.sign[e] > 0
                            else (r.dist_lam_inh, 0, r.lam_inh_min, r.lam_inh_max))
    t[2 * N + 2 * E:] = (0, 0, r.n_min, r.n_max)
    return t


@pytest.mark.parametrize("lhs", [0, 64])
def test_class_equivalent_table_reproduces_the_class_draws(lhs):
    # same draws and units: G, k, lambda, n identical; T differs only by the
    # per-node median replacing the class median
    rc = O.default_ranges(median_samples=2000, lhs_sets=lhs)
    rt = O.default_ranges(median_samples=2000, lhs_sets=lhs, param_ranges=class_table(NET, rc))
    a, b = O.sample_params(NET, 4, 64, ranges=rc), O.sample_params(NET, 4, 64, ranges=rt)
    for f in ("G", "k", "lam", "n"):
        assert np.array_equal(getattr(a, f), getattr(b, f)), f
    Mc, Mt = O.node_medians(NET, rc), O.node_medians(NET, rt)
    ratio = b.T / a.T
    assert np.allclose(ratio, (Mt / Mc)[NET.src][None, :], rtol=1e-14)


def test_degenerate_rows_fix_the_per_node_medians():
    # every row a point: M0_j = G_j / k_j exactly, and a regulated node's
    # median is its level G_j / k_j times the Hill factor of each in-edge
    # (Eq. 1, 2) with the source at G_s / k_s and T = multiplier x M0_s
    net = O.Network(3, np.array([0, 1, 0]), np.array([1, 2, 2]), np.array([1, -1, -1]))
    N, E = 3, 3
    t = np.zeros(2 * N + 3 * E, dtype=O.PARAM_ROW)
    G, k = [10.0, 20.0, 30.0], [0.5, 0.25, 1.0]
    mult, lam, n = [0.5, 1.5, 1.0], [4.0, 0.1, 0.5], [2, 3, 1]
    for i in range(N):
        t[i] = (0, 0, G[i], G[i])
        t[N + i] = (0, 0, k[i], k[i])
    for e in range(E):
        t[2 * N + e] = (0, 0, mult[e], mult[e])
        t[2 * N + E + e] = (0, 0, lam[e], lam[e])
        t[2 * N + 2 * E + e] = (0, 0, n[e], n[e])
    r = O.default_ranges(median_samples=101, param_ranges=t)
    M = O.node_medians(net, r)
    M0 = np.array(G) / np.array(k)

    def factor(e):
        s = net.src[e]
        B, B0 = M0[s], mult[e] * M0[s]
        h = (B0**n[e] + lam[e] * B**n[e]) / (B0**n[e] + B**n[e])
        return h / lam[e] if net.sign[e] > 0 else h
    assert M[0] == M0[0]
    assert np.isclose(M[1], M0[1] * factor(0), rtol=1e-14)
    assert np.isclose(M[2], M0[2] * factor(1) * factor(2), rtol=1e-14)
    # the unregulated mode keeps M0 for every node
    r1 = O.default_ranges(median_samples=101, median_mode=1, param_ranges=t)
    assert np.array_equal(O.node_medians(net, r1), M0)


def test_per_parameter_distributions_mix():
    S = 20000
    r = O.default_ranges(median_samples=2000)
    t = class_table(NET, r)
    N = NET.n_nodes
    t[0] = (1, 0, 5.0, 50.0)          # G_0 log-uniform on [5, 50]
    t[1] = (2, 0, 10.0, 20.0)         # G_1 normal on [10, 20]
    t[N + 2] = (0, 0, 0.5, 0.6)       # k_2 uniform on [0.5, 0.6]
    e_n = 2 * N + 2 * NET.n_edges     # the first edge's Hill coefficient on {2, 3}
    t[e_n] = (0, 0, 2.0, 3.0)
    p = O.sample_params(NET, 6, S, ranges=O.default_ranges(median_samples=2000, param_ranges=t))
    assert stats.kstest(np.log(p.G[:, 0]), stats.uniform(np.log(5), np.log(10)).cdf).pvalue > 1e-3
    inner = p.G[:, 1][(p.G[:, 1] > 10) & (p.G[:, 1] < 20)]
    assert stats.kstest(inner, stats.truncnorm(-3, 3, loc=15, scale=10 / 6).cdf).pvalue > 1e-3
    assert stats.kstest(p.k[:, 2], stats.uniform(0.5, 0.1).cdf).pvalue > 1e-3
    assert set(np.unique(p.n[:, 0])) == {2, 3}
    # the untouched rows keep the class draws
    q = O.sample_params(NET, 6, S, ranges=r)
    assert np.array_equal(p.G[:, 2:], q.G[:, 2:]) and np.array_equal(p.n[:, 1:], q.n[:, 1:])


# ---------------------------------------------------------------- initial-condition ranges
def test_ic_ranges_map_the_same_draws():
    # uniform rows map the default unit draw u to lo + (hi - lo) u; a
    # log-uniform row follows its distribution; rows of [0, 1] reproduce
    # the default
    N, I = 5, 20000
    u = O.sample_ics(N, 3, I)
    rows = np.zeros(N, dtype=O.PARAM_ROW)
    rows[:] = (0, 0, 0.0, 1.0)
    assert np.array_equal(O.sample_ics(N, 3, I, ic_ranges=rows), u)
    rows[1] = (0, 0, 0.25, 0.5)
    rows[2] = (1, 0, 0.01, 1.0)
    rows[3] = (2, 0, 0.2, 0.8)
    v = O.sample_ics(N, 3, I, ic_ranges=rows)
    assert np.array_equal(v[:, [0, 4]], u[:, [0, 4]])
    assert np.array_equal(v[:, 1], 0.25 + (0.5 - 0.25) * u[:, 1])
    assert stats.kstest(np.log(v[:, 2]), stats.uniform(np.log(0.01), -np.log(0.01)).cdf).pvalue > 1e-3
    inner = v[:, 3][(v[:, 3] > 0.2) & (v[:, 3] < 0.8)]
    assert stats.kstest(inner, stats.truncnorm(-3, 3, loc=0.5, scale=0.1).cdf).pvalue > 1e-3
