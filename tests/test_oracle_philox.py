"""Pins of oracle/philox.py: the generator against the published known-answer vectors of
Philox4x32-10, the Box-Muller normals and the accept uniforms against their distributions,
and the step-size rule of App. B on cases worked by hand."""
import math
import os

import numpy as np
import pytest

from oracle import philox

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat():
    rows = []
    with open(GOLDEN) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            w = [int(x, 16) for x in line.split()]
            rows.append((w[0:4], w[4:6], w[6:10]))
    return rows


def test_known_answer_vectors():
    rows = _kat()
    assert len(rows) == 3
    for ctr, key, want in rows:
        got = [int(x) for x in philox.philox4x32_10(ctr, key)]
        assert got == want


def test_vectorised_counters_match_scalar_calls():
    ctr = (np.arange(5, dtype=np.uint64), 7, 0, 0)
    out = philox.philox4x32_10(ctr, (11, 13))
    for i in range(5):
        one = philox.philox4x32_10((i, 7, 0, 0), (11, 13))
        assert all(int(out[j][i]) == int(one[j]) for j in range(4))


def test_normals_are_standard_normal():
    from scipy import stats
    z = philox.normals(20250430, 3, 200_003)
    assert z.shape == (200_003,)
    assert abs(z.mean()) < 5.0 / math.sqrt(z.size)
    assert abs(z.var() - 1.0) < 5.0 * math.sqrt(2.0 / z.size)
    assert stats.kstest(z, "norm").pvalue > 1e-3
    # the two members of a Box-Muller pair are uncorrelated
    zz = philox.normals(20250430, 3, 200_000).reshape(-1, 2)
    assert abs(np.corrcoef(zz[:, 0], zz[:, 1])[0, 1]) < 5.0 / math.sqrt(zz.shape[0])


def test_normals_depend_on_seed_and_iteration_only():
    a = philox.normals(5, 9, 1001)
    assert np.array_equal(a[:400], philox.normals(5, 9, 400))          # a prefix is the same draw
    b = philox.normals(5, 10, 1001)
    c = philox.normals(6, 9, 1001)
    assert abs(np.corrcoef(a, b)[0, 1]) < 0.15 and abs(np.corrcoef(a, c)[0, 1]) < 0.15
    # iteration words above 2^32 take the high counter word
    assert not np.array_equal(philox.normals(5, 1 << 32, 64), philox.normals(5, 0, 64))


def test_uniforms_are_uniform_and_inside_the_open_interval():
    from scipy import stats
    u = philox.uniforms24(1, 2, 100_000)
    assert u.min() > 0.0 and u.max() < 1.0
    assert stats.kstest(u, "uniform").pvalue > 1e-3
    ua = np.array([philox.accept_uniform(77, k) for k in range(4000)])
    assert ua.min() > 0.0 and ua.max() < 1.0
    assert stats.kstest(ua, "uniform").pvalue > 1e-3
    # the accept uniform is output word 0 of counter (0, it, 0, 1), scaled by 2^-32
    w = philox.philox4x32_10((0, 12, 0, 1), (77, 0))
    assert philox.accept_uniform(77, 12) == (int(w[0]) + 0.5) / 2.0 ** 32


def test_step_rule_worked_cases():
    # below the threshold: shrink by 1.2 and keep shrinking
    assert philox.adapt_step(0.12, 0.12, 0.1, 0.2) == 0.12 / 1.2
    assert philox.adapt_step(0.1, 0.12, 0.0, 0.2) == 0.1 / 1.2
    # at or above the threshold: grow by 1.2, capped at the original step
    assert philox.adapt_step(0.1, 0.2, 0.5, 0.2) == 1.2 * 0.1
    assert philox.adapt_step(0.11, 0.12, 0.2, 0.2) == 0.12
    assert philox.adapt_step(0.12, 0.12, 1.0, 0.2) == 0.12
    # a sequence: two rejections then recovery to eps0
    eps, seq = 0.3, []
    for a in (0.05, 0.1, 0.9, 0.9, 0.9):
        eps = philox.adapt_step(eps, 0.3, a, 0.2)
        seq.append(eps)
    assert seq == pytest.approx([0.25, 0.3 / 1.44, 0.25, 0.3, 0.3], rel=1e-15)


def test_acceptance_probability():
    assert philox.acceptance_probability(1.0, 0.5) == 1.0
    assert philox.acceptance_probability(1.0, 1.0) == 1.0
    assert philox.acceptance_probability(1.0, 3.0) == math.exp(-2.0)
    assert philox.acceptance_probability(1.0, float("inf")) == 0.0
    assert philox.acceptance_probability(float("nan"), 1.0) == 0.0
