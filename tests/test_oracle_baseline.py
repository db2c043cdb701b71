"""The arithmetic of the timed CPU baseline's model (oracle/baseline.py, no
GPU): power-law fits recover an exact power law, and the model charges each
sparse level one worker start-up and one factorisation plus, per subspace
iteration, two q-column solves, the rest of the iteration and the q x q
eigensolve, then the coarsest level's dense eigensolve."""
import math

import pytest

from oracle import baseline


def test_power_law_fit_recovers_the_law():
    ns = [10_000, 20_000, 40_000, 90_000]
    f, b = baseline._fit(ns, [3e-6 * n ** 1.5 for n in ns])
    assert b == pytest.approx(1.5, rel=1e-12)
    assert f(10 ** 6) == pytest.approx(3e-6 * 1e9, rel=1e-10)


def test_predict_charges_each_level_and_iteration():
    model = {"fits": {"factor": (lambda n: 2.0e-3 * n, 1.0), "solve": (lambda n: 0.5, 0.0),
                      "gram": (lambda n: 0.25, 0.0)}, "pool": 1.0, "ritz": 0.1}
    sizes, iters, coarse = [1000, 100, 3], [2, 3, 0], 0.7
    per_iter = 2 * 0.5 + 0.25 + 0.1
    want = (1.0 + 2.0 + 2 * per_iter) + (1.0 + 0.2 + 3 * per_iter) + coarse
    assert baseline.predict(model, sizes, iters, coarse) == pytest.approx(want, rel=1e-15)
    # no sparse level: only the dense eigensolve
    assert baseline.predict(model, [50], [0], coarse) == coarse
    assert math.isfinite(baseline.predict(model, sizes, [100, 100, 0], coarse))
