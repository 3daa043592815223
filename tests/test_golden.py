"""The FP64 oracle against the stored values under tests/golden/ (written by
tests/golden/make_golden.py from the oracle itself): a change to the
oracle's arithmetic shows up here and must be justified by the passage of
the paper it follows.  Independent pins of the oracle live in
test_oracle_pins.py."""
import numpy as np
import pytest

from tests.golden import make_golden as G

CASES = list(G.cases())


@pytest.mark.parametrize("prob", CASES, ids=[p.name for p in CASES])
def test_oracle_matches_stored_values(prob):
    stored = G.read(prob.name)
    now = G.compute(prob)
    assert set(stored) == set(now)
    for key in stored:
        np.testing.assert_allclose(now[key], stored[key], rtol=1e-13, atol=1e-15, err_msg=key)


def test_stored_values_obey_the_invariants():
    """Histogram rows sum to 1, M_1 equals the central c_1, and uniform axes
    carry no sensitivity (Sec. 5.3 hard truncation)."""
    for prob in CASES:
        v = G.read(prob.name)
        np.testing.assert_allclose(v["hist"].sum(axis=1), 1.0, atol=1e-14)
        np.testing.assert_allclose(v["raw"][:, 0], v["central"][:, 0], atol=1e-15)
        for k in range(prob.K):
            for d in range(prob.ndim):
                if prob.dens.kind[k, d] == 1:
                    assert np.all(v["dmu"][k, d] == 0) and np.all(v["dsigma"][k, d] == 0)
