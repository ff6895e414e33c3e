"""The library's level-boundary rule (host code, no GPU) against the
oracle's on constructed and random histograms, and its argument checks."""
import numpy as np
import pytest

import oracle as O


def api():
    return pytest.importorskip("paper_2503_18356_gb300.api")


def histograms():
    rng = np.random.default_rng(7)
    out = [np.zeros(100, np.uint64), np.full(100, 5, np.uint64)]
    for _ in range(60):
        B = int(rng.choice([10, 50, 100, 257]))
        x = np.zeros(B)
        for _m in range(int(rng.integers(1, 5))):
            ctr, wid = rng.uniform(0, B), rng.uniform(0.5, B / 6)
            x += rng.uniform(10, 1e4) * np.exp(-0.5 * ((np.arange(B) - ctr) / wid) ** 2)
        if rng.uniform() < 0.5:
            x += rng.poisson(3, B)
        out.append(np.floor(x).astype(np.uint64))
    return out


@pytest.mark.parametrize("m", [0, 1, 4, 8])
@pytest.mark.parametrize("max_b", [1, 3, 16])
def test_library_boundaries_match_oracle(m, max_b):
    A = api()
    for c in histograms():
        assert list(A.level_boundaries(c, half_width=m, max_boundaries=max_b)) == \
            list(O.level_boundaries(c, m=m, max_b=max_b))


def test_library_boundaries_argument_checks():
    A = api()
    c = np.ones(10, np.uint64)
    for kw in (dict(half_width=9), dict(half_width=-1), dict(max_boundaries=0), dict(max_boundaries=17)):
        with pytest.raises(A.GrinsError):
            A.level_boundaries(c, **kw)
    with pytest.raises(A.GrinsError):
        A.level_boundaries(np.ones(1, np.uint64))
