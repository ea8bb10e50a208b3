"""Host-side pieces of the bow-shock validation tool: the reference values it prints and
its shock locator (no GPU)."""
import math

import numpy as np
import pytest

from paper_2506_16076_gb300 import bow_shock as B


@pytest.mark.parametrize("M", [1.5, 3.0, 3.5, 25.0])
def test_pitot_pressure_matches_the_normal_shock_relations(M):
    g = 1.4
    p2 = 1.0 + 2 * g / (g + 1) * (M * M - 1)                      # static pressure jump
    M2sq = (1 + 0.5 * (g - 1) * M * M) / (g * M * M - 0.5 * (g - 1))  # post-shock Mach^2
    p02 = p2 * (1 + 0.5 * (g - 1) * M2sq) ** (g / (g - 1))         # isentropic to rest
    assert abs(B.pitot_pressure(M) - p02) <= 1e-12 * p02


def test_billig_fit_reproduces_the_printed_table_values():
    # Sec. 7, table bow: the fit gives 0.283 at M = 3.5 and 0.194 at M = 25 (lambda_1 = 0.193)
    assert round(B.billig_standoff(3.5), 3) == 0.283
    assert round(B.billig_standoff(25.0), 3) == 0.194
    # and 0.293 / 0.201 with the approximated lambda_1 = 0.2
    assert round(B.billig_standoff(3.5, lam1=0.2), 3) == 0.293
    assert round(B.billig_standoff(25.0, lam1=0.2), 3) == 0.201


def test_shock_radius_on_a_smeared_jump():
    r = np.linspace(0.5, 1.5, 401)
    rho = 1.4 + 0.5 * (5.4 - 1.4) * (1 - np.tanh((r - 0.83) / 0.01)) + 0.3 * np.exp(-(r - 0.5) / 0.05)
    assert abs(B.shock_radius(r, rho, 1.4) - 0.83) < 0.01
    assert math.isnan(B.shock_radius(r, np.full_like(r, 1.4) - 1.0, 1.4))
