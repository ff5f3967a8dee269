"""Energy watchdog of dgh_step (DGH_EUNSTABLE).  The failures are made on the
host: an energy bound set below the run's energy, and a corrupted input state
(one NaN in the fields).  No GPU fault is involved; NaN arithmetic is
ordinary floating point."""
import numpy as np
import pytest

import paper_1610_05023_b300 as dgh
from paper_1610_05023_b300 import workloads as W


def _solver(seed=60):
    VX, EToV = W.kuhn_mesh(3, 1.0, 0.02, seed=seed)
    g = dgh.Solver(VX, EToV, 3, 2)
    g.init_gaussian([0.2, -0.1, 0.1], 0.3)
    return g


@pytest.mark.gpu
def test_watchdog_that_never_trips_changes_nothing():
    a, b = _solver(), _solver()
    b.set_watchdog(5, energy_limit=1e9)
    a.step(20)
    b.step(20)
    for lv in (3, 2, 1):
        assert np.array_equal(a.get_state(lv), b.get_state(lv))


@pytest.mark.gpu
def test_watchdog_trips_on_a_host_set_energy_bound():
    g = _solver()
    E0 = g.energy()
    g.set_watchdog(4, energy_limit=0.5 * E0)    # below the energy of the run: a forced trip
    with pytest.raises(dgh.DghError) as ei:
        g.step(20)
    assert ei.value.code == dgh.DGH_EUNSTABLE
    assert "watchdog" in str(ei.value)
    assert g.info["step_count"] == 4            # stopped at the first check
    g.set_watchdog(4, energy_limit=2.0 * E0)    # a sound bound: the run goes on
    g.step(8)
    assert g.info["step_count"] == 12
    g.set_watchdog(0)
    g.step(3)
    assert np.isfinite(g.energy())


@pytest.mark.gpu
def test_watchdog_catches_a_non_finite_state():
    g = _solver()
    q = g.get_state(3)
    q[5, 0, 3] = np.nan                          # corrupted input array
    g.set_state(3, q)
    g.set_watchdog(1)
    with pytest.raises(dgh.DghError) as ei:
        g.step(3)
    assert ei.value.code == dgh.DGH_EUNSTABLE
    assert g.info["step_count"] == 1
