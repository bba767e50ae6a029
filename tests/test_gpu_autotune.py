"""The schedule autotuner: it times every candidate, returns the fastest, and
the schedule it picks sweeps like any other (the schedule changes where work
runs, not what is computed)."""
import numpy as np
import pytest

import synth
from paper_2503_17743_gb300 import MOC_TALLY_GLOBAL, Geometry, Tracks, autotune, track_params

pytestmark = pytest.mark.gpu


def test_autotune_picks_the_fastest_candidate():
    p = synth.workload("lattice5")
    g = Geometry(p)
    base = track_params(p, preload_budget_bytes=200000)
    best, sec, table = autotune(g, base, iterations=3)
    assert table.shape[0] >= 6  # 3 lane shapes x at least 2 tally / budget choices
    assert sec == pytest.approx(table[:, 4].min())
    row = table[np.argmin(table[:, 4])]
    assert best.groups_per_lane == int(row[0]) and best.tally_mode == int(row[1])
    assert best.preload_budget_bytes == int(row[2]) and best.sync_block == int(row[5])
    assert set(table[:, 0].astype(int)) == {1, 2, 4}
    # two groups per lane with stored templates: every warp schedule is timed
    two = table[(table[:, 0] == 2) & (table[:, 2] != 0)]
    assert {1, 4, 8} <= set(two[:, 5].astype(int))
    assert MOC_TALLY_GLOBAL in set(table[:, 1].astype(int))
    # same sweep under the tuned and the default schedule
    Q = np.random.default_rng(1).uniform(0.2, 1.0, size=(Tracks(g, base).n_fsr, p.num_groups))
    a = Tracks(g, best).sweep_from_source(Q)[0]
    b = Tracks(g, track_params(p)).sweep_from_source(Q)[0]
    np.testing.assert_allclose(a, b, rtol=1e-5, atol=1e-6 * np.abs(b).max())
