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
tallies element by element against the FP64 oracle (1e-4 relative above
1e-3 of the largest, 2e-5 of the largest below), from a uniform source and
from one peaked at the centre of the core.  The oracle runs in its light mode (tracks and segments only).
"""
import os

import numpy as np
import pytest

import oracle
import synth
from paper_2503_17743_gb300 import MOC_FP32, Geometry, Tracks, track_params

from tests.parity import check_tally, shaped_source

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
    # both sweep in radial chunks; the core's records carry their material
    # (one material per radial region), the assemblies' rows carry Sigma_t
    # (the absorber changes a guide tube's material with the layer)
    assert info["chunk_segments"] > 0
    assert info["material_keys"] == (1 if name == "core7x7" else 0)
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
    Qu = rng.uniform(0.2, 1.0, size=(o.n_fsr, p.num_groups))
    # a source peaked at the centre, 1e-3 of the peak at the edges: low-flux
    # regions share their 2D tracks (and fixed-point tally scale) with the
    # peak's
    Qs = shaped_source(p, p.num_groups, seed=37)
    # a sample from the middle of the laydown and one from its end (the
    # largest and the smallest work units of an azimuth)
    for label, Q in (("uniform", Qu), ("shaped", Qs)):
        for t0 in (o.n_tracks2d // 3, o.n_tracks2d - 24):
            n, ot = o.sweep_sample(Q, t0, t0 + 24)
            gt, _ = tr.sweep_units_from_source(Q, t0, t0 + 24)
            assert n > 0
            check_tally(gt, ot, what=f"{name} {label} tracks {t0}-{t0 + 24}")
    tr.close()
