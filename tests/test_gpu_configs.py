"""Parity on the large configurations, on outputs the oracle can produce one
by one:

* 3x3 assemblies + reflector (64 cm, 32 layers, 64 azimuths x 6 polar,
  0.05 / 0.25 cm), with a preload budget below the full template set so part
  of the stacks is generated on the fly;
* the 7x7-assembly core with a reflector ring (200 cm, 100 layers,
  128 azimuths x 6 polar, all faces vacuum).

For each: sampled z-stacks bit-exact (10^4 on the assemblies, 500 on the
core), and one sweep of a sample of 2D tracks
(every polar angle, both senses, zero incoming flux) from a seeded source,
tallies element by element against the FP64 oracle (FP32 tolerance 2e-5 of
the largest).  The oracle runs in its light mode (tracks and segments only).
"""
import os

import numpy as np
import pytest

import oracle
import synth
from paper_2503_17743_gb300 import MOC_FP32, Geometry, Tracks, track_params

pytestmark = pytest.mark.gpu

NTH = os.cpu_count() or 4


@pytest.mark.parametrize("name,budget,n_stacks", [("asm3x3", 1 << 30, 10000), ("core7x7", -1, 500)])
def test_large_configuration_samples(name, budget, n_stacks):
    p = synth.workload(name)
    o = oracle.Oracle(p, n_threads=NTH, light=True)
    tr = Tracks(Geometry(p), track_params(p, precision=MOC_FP32, preload_budget_bytes=budget))
    info = tr.info
    assert info["tracks3d"] == o.n_tracks3d
    if budget > 0:
        # part stored, part generated on the fly (Sec. 4.2)
        assert 0 < info["preloaded_stacks"] < info["stacks"] // 2
    rng = np.random.default_rng(31)
    for _ in range(n_stacks):
        t = int(rng.integers(o.n_tracks2d))
        pp = int(rng.integers(p.n_polar))
        oi, on, of, ol = o.stack(t, pp)
        gi, gn, gf, gl = tr.stack_segments(t, pp)
        np.testing.assert_array_equal(gi, oi)
        np.testing.assert_array_equal(gn, on)
        np.testing.assert_array_equal(gf, of)
        assert np.all(np.abs(gl - ol) <= 1e-6 * ol + 1e-6)
    Q = rng.uniform(0.2, 1.0, size=(o.n_fsr, p.num_groups))
    # a sample from the middle of the laydown and one from its end (the
    # largest and the smallest work units of an azimuth)
    for t0 in (o.n_tracks2d // 3, o.n_tracks2d - 24):
        n, ot = o.sweep_sample(Q, t0, t0 + 24)
        gt, _ = tr.sweep_units_from_source(Q, t0, t0 + 24)
        scale = np.abs(ot).max()
        assert n > 0 and scale > 0
        assert np.abs(gt - ot).max() <= 2e-5 * scale, np.abs(gt - ot).max() / scale
    tr.close()
