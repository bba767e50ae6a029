"""The 2D ray tracer on the device (moc_track_params.trace_on_device) gives
the host tracer's 2D segments bit for bit, and both match the oracle's."""
import numpy as np
import pytest

import oracle
import synth
from paper_2503_17743_gb300 import Geometry, Tracks, track_params

pytestmark = pytest.mark.gpu


def _lat3_rings():
    p = synth.lattice(5, n=3, G=3, height=4.0, n_layers=4, n_azim=8, n_polar=4,
                      radial_spacing=0.15, axial_spacing=0.5, bc=(1, 0, 1, 1, 0, 1), n_gt=2)
    return p.with_tracks(fuel_rings=2, moderator_rings=1, sectors=8, name="lat3_rings")


CASES = {
    "pin_cell": lambda: synth.workload("pin_cell"),
    "pin_cell_rings": lambda: synth.workload("pin_cell_rings"),
    "lat3_rings": _lat3_rings,
    "lattice5_rings": lambda: synth.workload("lattice5_rings"),
    "lattice17": lambda: synth.workload("lattice17"),
    "asm3x3": lambda: synth.workload("asm3x3"),
}


@pytest.mark.parametrize("name", list(CASES))
def test_device_tracer_is_the_host_tracer(name):
    p = CASES[name]()
    g = Geometry(p)
    host = Tracks(g, track_params(p, trace_on_device=0, preload_budget_bytes=0))
    dev = Tracks(g, track_params(p, trace_on_device=1, preload_budget_bytes=0))
    assert dev.info["tracks2d"] == host.info["tracks2d"]
    assert dev.info["segments3d"] == host.info["segments3d"]
    nt = host.info["tracks2d"]
    ts = range(nt) if nt <= 20000 else np.random.default_rng(3).integers(0, nt, 20000)
    for t in ts:
        hr, hl, hp = host.segments2d(int(t))
        dr, dl, dp = dev.segments2d(int(t))
        np.testing.assert_array_equal(dr, hr)
        np.testing.assert_array_equal(dl, hl)  # bit for bit
        np.testing.assert_array_equal(dp, hp)
    # volumes sum FP64 contributions with atomics: equal up to the order of the adds
    np.testing.assert_allclose(dev.volumes(), host.volumes(), rtol=1e-12)
    host.close()
    dev.close()


@pytest.mark.parametrize("name", ["pin_cell_rings", "lat3_rings"])
def test_device_tracer_against_oracle(name):
    p = CASES[name]()
    o = oracle.Oracle(p)
    dev = Tracks(Geometry(p), track_params(p, trace_on_device=1))
    for t in range(o.n_tracks2d):
        oreg, oln, opos = o.segments2d(t)
        dreg, dln, dpos = dev.segments2d(t)
        np.testing.assert_array_equal(dreg, oreg)
        np.testing.assert_allclose(dln, oln, rtol=0, atol=1e-12)
        np.testing.assert_allclose(dpos, opos, rtol=0, atol=1e-12)
    dev.close()
