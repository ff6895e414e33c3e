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
