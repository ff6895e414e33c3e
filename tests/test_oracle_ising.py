"""Pins of the oracle's Boolean Ising formalism (Sec. 2.2, Eq. 3): a toggle
switch worked by hand, the tie rule, the 0/1 encoding, and every fixed point
of small random networks found by brute force over all their states."""
import numpy as np

import oracle as O
from paper_2503_18356_gb300 import workloads as W


def net_of(n, edges):
    src, dst, sign = zip(*edges)
    return O.Network(n, np.array(src), np.array(dst), np.array(sign))


TS = [(0, 1, -1), (1, 0, -1)]        # mutual inhibition; bit 0 = A, bit 1 = B


def test_toggle_switch_synchronous_by_hand():
    net = net_of(2, TS)
    fin, stp, st = O.ising_run(net, mode=0, n_traj=4, init=np.arange(4, dtype=np.uint64), max_steps=7)
    # 01 and 10 are fixed; 00 -> 11 -> 00 ... never settles (7 updates: ends at 11)
    assert list(st) == [2, 0, 0, 2] and list(stp) == [7, 0, 0, 7]
    assert list(fin) == [3, 1, 2, 0]


def test_toggle_switch_asynchronous_reaches_a_fixed_point():
    net = net_of(2, TS)
    fin, stp, st = O.ising_run(net, mode=1, seed=5, n_traj=200, init=np.zeros(200, np.uint64), max_steps=50)
    assert np.all(st == 0) and np.all(stp == 1)           # one flip from 00 settles it
    assert set(fin.tolist()) == {1, 2}                    # both fixed points are reached
    assert 60 < np.sum(fin == 1) < 140


def test_tie_keeps_the_state_and_zero_one_encoding():
    # A and B hold themselves (self-activation); C has A activating, B inhibiting
    net = net_of(3, [(0, 0, 1), (1, 1, 1), (0, 2, 1), (1, 2, -1)])
    init = np.array([0b011, 0b111, 0b000, 0b001], dtype=np.uint64)
    fin, _, st = O.ising_run(net, mode=0, n_traj=4, init=init, max_steps=10)
    # A, B on: field of C is 1 - 1 = 0, C keeps its state; A, B off: -1 + 1 = 0 too
    assert list(fin) == [0b011, 0b111, 0b000, 0b101] and np.all(st == 0)
    # 0/1 encoding: inactive sources count 0 -- the toggle switch's 00 is fixed
    fin01, _, st01 = O.ising_run(net_of(2, TS), mode=0, n_traj=1, init=np.zeros(1, np.uint64),
                                 max_steps=5, enc01=True)
    assert fin01[0] == 0 and st01[0] == 0


def brute_fixed_points(n, src, dst, sign, enc01=False):
    J = np.zeros((n, n), dtype=int)
    for s_, d_, g_ in zip(src, dst, sign):
        J[d_, s_] += g_
    fixed = []
    for code in range(2 ** n):
        bits = np.array([(code >> i) & 1 for i in range(n)])
        s = np.where(bits == 1, 1, 0 if enc01 else -1)
        h = J @ s
        nxt = np.where(h > 0, 1, np.where(h < 0, 0, bits))
        if np.array_equal(nxt, bits):
            fixed.append(code)
    return set(fixed)


def test_fixed_points_by_brute_force():
    for seed, n, e in [(1, 4, 7), (2, 6, 12), (3, 8, 16), (4, 7, 20)]:
        topo = W.random_network(seed, n, e, e // 2, 1)
        N, src, dst, sign = topo.edges()
        net = O.Network(N, src, dst, sign)
        for enc01 in (False, True):
            want = brute_fixed_points(N, src, dst, sign, enc01)
            allc = np.arange(2 ** N, dtype=np.uint64)
            fin, stp, st = O.ising_run(net, mode=0, n_traj=allc.size, init=allc, max_steps=0, enc01=enc01)
            assert set(allc[st == 0].tolist()) == want
            # every settled trajectory, either mode, ends on one of them
            for mode in (0, 1):
                fin, stp, st = O.ising_run(net, mode=mode, seed=seed, n_traj=300, max_steps=400, enc01=enc01)
                assert set(fin[st == 0].tolist()) <= want
                if mode == 1 and want:
                    assert np.mean(st == 0) > 0.5


def test_random_initial_states_from_the_seed():
    net = O.Network(*W.random_network(5, 22, 60, 30, 0).edges())
    a, _, _ = O.ising_run(net, mode=0, seed=11, n_traj=64, max_steps=0)
    b, _, _ = O.ising_run(net, mode=0, seed=11, n_traj=64, max_steps=0)
    c, _, _ = O.ising_run(net, mode=0, seed=12, n_traj=64, max_steps=0)
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    assert np.all(a < (1 << 22))
    bits = np.array([[(int(x) >> i) & 1 for i in range(22)] for x in a])
    assert 0.35 < bits.mean() < 0.65
