"""Pins of the oracle's drift calibration (step 11) by synthetic closure: a
timeframe generated with the drift velocity scaled by (1 + eps) gives back eps,
and one generated with another collision time gives back that time."""
import pytest

import oracle
import tpcgen


@pytest.mark.parametrize("eps", [0.01, -0.02])
def test_drift_velocity_closure(eps):
    tf = tpcgen.generate(tpcgen.full_tpc(3, n_tracks=4000, bin_cm=0.5 * (1 + eps)))
    r = oracle.reconstruct(tf)
    tv, e, t0, n = oracle.calibrate_drift(r, 250.0)
    assert n > 1000
    assert tv == pytest.approx(250.0 + 500.0 / (1 + eps), abs=0.1)
    assert e == pytest.approx(eps, abs=2e-4)


def test_collision_time_closure():
    tf = tpcgen.generate(tpcgen.full_tpc(4, n_tracks=4000, coll_t0=[180.0]))
    r = oracle.reconstruct(tf)
    tv, e, t0, n = oracle.calibrate_drift(r, 180.0)
    assert n > 1000 and t0 == pytest.approx(180.0, abs=0.1) and abs(e) < 2e-4
