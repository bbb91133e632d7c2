"""Host arithmetic of the degree/scale tuner: iteration predictions from two
residual probes, on closed cases (an exactly geometric residual history)."""
import math

import pytest

from paper_2008_01440_gb300.tune import predict_iterations


@pytest.mark.parametrize("rho", [0.5, 0.9, 0.99])
def test_geometric_history_is_extrapolated_exactly(rho):
    # ||r_i|| / ||b|| = rho^i: tol is reached at i = log(tol) / log(rho)
    ia, ib, tol = 3, 12, 1e-8
    got_rho, it = predict_iterations(ia, rho ** ia, ib, rho ** ib, tol)
    assert got_rho == pytest.approx(rho, rel=1e-12)
    assert it == pytest.approx(math.log(tol) / math.log(rho), rel=1e-9)


def test_converged_within_the_probes():
    rho = 0.05
    # the short probe already below tol: interpolate from its start
    _, it = predict_iterations(8, rho ** 8, 16, rho ** 16, 1e-8)
    assert it == pytest.approx(math.log(1e-8) / math.log(rho), rel=1e-9)
    # crossed between the probes
    _, it2 = predict_iterations(2, rho ** 2, 12, rho ** 12, 1e-8)
    assert 2 < it2 < 12 and it2 == pytest.approx(math.log(1e-8) / math.log(rho), rel=1e-9)


def test_stagnation_predicts_no_convergence():
    rho, it = predict_iterations(3, 0.5, 12, 0.5, 1e-8)
    assert rho == pytest.approx(1.0) and math.isinf(it)
