"""Host logic of the long-run driver: extended-self-similarity exponents
(SI section 3) recovered from synthetic power laws."""
import numpy as np
import pytest

pytest.importorskip("torch")
from paper_2403_18466_gb300 import les  # noqa: E402


def test_ess_recovers_power_law_ratios():
    r = np.arange(1, 40, dtype=float)
    zeta = np.array([0.37, 0.71, 1.0, 1.26, 1.49, 1.70])   # any exponents
    S = np.array([(p + 2.0) * r ** (zeta[p] * 0.9) for p in range(6)])
    xi = les.ess_exponents(S)
    assert np.allclose(xi, zeta / zeta[2], rtol=1e-10)


def test_ess_uses_absolute_values_and_range():
    r = np.arange(1, 30, dtype=float)
    S = np.array([(-1) ** p * r ** ((p + 1) / 3) for p in range(6)])   # odd orders negative
    assert np.allclose(les.ess_exponents(S), np.arange(1, 7) / 3, rtol=1e-10)
    # outside the chosen S^3 range the data may break the law without effect
    S2 = S.copy()
    S2[:, -5:] *= 7.0
    rng = (1.0, float(np.abs(S[2, -6])))
    assert np.allclose(les.ess_exponents(S2, rng), np.arange(1, 7) / 3, rtol=1e-10)
    assert np.all(np.isnan(les.ess_exponents(S2, (1e9, 1e10))))
