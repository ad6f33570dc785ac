"""Host-side helpers of the learned-tolerance controller (no GPU): the half-decade tau
grid and the relative energy error used to judge an SP2 run."""
import math

import pytest

C = pytest.importorskip("paper_1011_3534_gb300.controller")


def test_half_decade_grid():
    g = C.half_decades(1e-8, 1e-4)
    assert len(g) == 9
    assert g[0] == pytest.approx(1e-8, rel=1e-12) and g[-1] == pytest.approx(1e-4, rel=1e-12)
    for a, b in zip(g, g[1:]):
        assert b / a == pytest.approx(math.sqrt(10.0), rel=1e-12)


def test_half_decade_grid_single_point():
    assert C.half_decades(1e-6, 1e-6) == [pytest.approx(1e-6, rel=1e-12)]


def test_energy_error_is_relative():
    assert C.energy_error({"energy": -101.0}, -100.0) == pytest.approx(0.01)
    assert C.energy_error({"energy": 3.0}, 3.0) == 0.0
