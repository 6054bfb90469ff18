"""Host-side pins of the experiment analysis: the a -> 0 fit of the paper's
benzene footnote (E0 + k1 a^2 + k2 a^4) and the power-law exponent of
Fig. 2, on synthetic data with known answers (no GPU)."""
import numpy as np
import pytest

from paper_1909_01589_gb300 import experiments as X


def test_fit_a0_recovers_exact_polynomial():
    """Noise-free E(a) = E0 + k1 a^2 + k2 a^4: the fit returns E0, k1, k2
    to rounding and chi^2 = 0."""
    a = np.array([0.4, 0.3, 0.2, 0.15, 0.1])
    E0, k1, k2 = -2.903724, 0.35, -1.7
    E = E0 + k1 * a ** 2 + k2 * a ** 4
    fit = X.fit_a0(a, E, np.full(len(a), 1e-4))
    assert abs(fit["E0"] - E0) < 1e-12
    assert abs(fit["k1"] - k1) < 1e-9 and abs(fit["k2"] - k2) < 1e-8
    assert fit["chi2_per_dof"] < 1e-12


def test_fit_a0_error_is_calibrated():
    """With Gaussian noise of the stated errors, (E0_fit - E0) / E0_error is
    standard normal over many synthetic data sets and chi^2 per degree of
    freedom averages 1: the reported error bar means what it says."""
    rng = np.random.default_rng(7)
    a = np.array([0.4, 0.3, 0.2, 0.15, 0.1])
    err = np.array([2e-4, 2.5e-4, 3e-4, 3.5e-4, 4e-4])
    E0, k1, k2 = -128.9, 0.9, 2.0
    z, chi = [], []
    for _ in range(4000):
        E = E0 + k1 * a ** 2 + k2 * a ** 4 + err * rng.normal(size=len(a))
        fit = X.fit_a0(a, E, err)
        z.append((fit["E0"] - E0) / fit["E0_error"])
        chi.append(fit["chi2_per_dof"])
    z = np.array(z)
    assert abs(np.mean(z)) < 0.06 and abs(np.std(z) - 1.0) < 0.05
    assert abs(np.mean(chi) - 1.0) < 0.06


def test_fit_a0_rejects_too_few_points():
    with pytest.raises(ValueError):
        X.fit_a0([0.2, 0.1], [1.0, 1.0], [0.1, 0.1])


def test_z_exponent_and_fixed_error_cost():
    """cost = c Z^x is fitted exactly; summarize() reports the exponent of
    the cost per unit projection time and of the cost at fixed error
    (1/efficiency), and their ratio single/double as the acceleration."""
    Z = np.array([2.0, 10.0, 18.0, 36.0])
    assert abs(X.z_exponent(Z, 3.0 * Z ** 5.55) - 5.55) < 1e-12
    rows = []
    for z in Z:
        row = {"system": f"Z{int(z)}", "Z": z, "walkers": 100, "tau": 0.01,
               "double_this_work_acceleration_jumps": 2.0}
        for k, xt, xe in (("single", 4.0, 5.55), ("double_this_work", 3.6, 5.06), ("double_previous", 3.8, 5.3)):
            row[k] = {"seconds": 1e-3 * z ** xt * 100 * 50 * 0.01, "intervals": 50, "tau": 0.01,
                      "efficiency": 1.0 / (7.0 * z ** xe)}
        rows.append(row)
    derived, fit = X.summarize(rows)
    assert abs(fit["single"] - 4.0) < 1e-9 and abs(fit["double_this_work"] - 3.6) < 1e-9
    assert abs(fit["single_fixed_error"] - 5.55) < 1e-9 and abs(fit["double_this_work_fixed_error"] - 5.06) < 1e-9
    for z, d in zip(Z, derived):
        assert abs(d["acceleration_fixed_error"] - z ** (5.55 - 5.06)) < 1e-9 * z
