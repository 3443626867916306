"""Host helpers of the batched magnetisation curve (paper_1212_2934_gb300.magnetisation).

L(alpha) against the oracle's Langevin function (Sec. 5, Eq. Langevin) and its limits, and
the pooled integrated autocorrelation time against the closed form of an AR(1) series,
tau = (1 + rho) / (1 - rho)."""
import numpy as np

from paper_1212_2934_gb300 import magnetisation as mg


def test_langevin_matches_the_oracle_and_its_limits(ora):
    a = np.array([0.0, 1e-6, 1e-3, 0.5, 1.0, 3.0, 5.0, 50.0])
    np.testing.assert_allclose(mg.langevin(a), ora.langevin(a), rtol=1e-12, atol=1e-15)
    assert mg.langevin(0.0) == 0.0
    assert abs(mg.langevin(1e-4) - (1e-4 / 3 - 1e-12 / 45)) < 1e-20
    assert abs(mg.langevin(50.0) - (1 - 1 / 50.0)) < 1e-12


def test_pooled_tau_of_ar1_series():
    rng = np.random.default_rng(3)
    rho, systems, w = 0.6, 400, 400
    x = np.zeros((systems, w))
    e = rng.standard_normal((systems, w))
    x[:, 0] = e[:, 0] / np.sqrt(1 - rho ** 2)
    for t in range(1, w):
        x[:, t] = rho * x[:, t - 1] + e[:, t]
    tau, lags = mg.pooled_tau(x)
    assert abs(tau - (1 + rho) / (1 - rho)) < 0.15 * (1 + rho) / (1 - rho)
    white, _ = mg.pooled_tau(rng.standard_normal((systems, w)))
    assert abs(white - 1.0) < 0.05
