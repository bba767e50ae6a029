"""The load-balancing and preload ablations (Sec. 4.2 stored vs regenerated
segments, Fig. 6; Sec. 4.3 load balancing, Fig. 7) sweep like the oracle:
every MOC_SCHED_* schedule and every stored share of the segment templates
(0, 1/4, 1/2, 3/4, all) gives the oracle's tallies element by element, from
the same seeded source, and the same tallies as the default schedule up to
FP32 rounding (the orders of the sweep change, the arithmetic does not)."""
import os

import numpy as np
import pytest

import oracle
import synth
from paper_2503_17743_gb300 import (MOC_FP32, MOC_SCHED_TRACKS_NATURAL, MOC_SCHED_UNITS_NATURAL,
                                    Geometry, Tracks, track_params)
from tests.parity import check_flux, check_tally

pytestmark = pytest.mark.gpu

NTH = os.cpu_count() or 4


@pytest.fixture(scope="module")
def problem():
    p = synth.workload("lattice17_small")
    o = oracle.Oracle(p, n_threads=NTH)
    g = Geometry(p)
    Q = np.random.default_rng(41).uniform(0.2, 1.0, size=(o.n_fsr, p.num_groups))
    o.reset()
    ot, ol = o.sweep_once(Q)
    full = Tracks(g, track_params(p, precision=MOC_FP32, preload_budget_bytes=-1))
    tpl_bytes = full.info["stored_segments"] * 8
    base, _ = full.sweep_from_source(Q)
    full.close()
    return p, o, g, Q, ot, ol, tpl_bytes, base


CASES = [("EXP share", f, 0) for f in (0.0, 0.25, 0.5, 0.75, 1.0)] + [
    ("schedule", 1.0, MOC_SCHED_UNITS_NATURAL | MOC_SCHED_TRACKS_NATURAL),
    ("schedule", 1.0, MOC_SCHED_TRACKS_NATURAL),
    ("schedule", 1.0, MOC_SCHED_UNITS_NATURAL),
    ("schedule", 0.5, MOC_SCHED_UNITS_NATURAL | MOC_SCHED_TRACKS_NATURAL),
]


@pytest.mark.parametrize("kind,frac,sched", CASES)
def test_ablation_case_sweeps_like_the_oracle(problem, kind, frac, sched):
    p, o, g, Q, ot, ol, tpl_bytes, base = problem
    budget = -1 if frac >= 1.0 else int(frac * tpl_bytes)
    tr = Tracks(g, track_params(p, precision=MOC_FP32, preload_budget_bytes=budget, schedule=sched))
    info = tr.info
    if frac == 0.0:
        assert info["stored_segments"] == 0
    elif frac < 1.0:
        assert 0 < info["stored_segments"] * 8 <= budget
        assert 0 < info["preloaded_stacks"] < info["stacks"] // 2
    gt, gl = tr.sweep_from_source(Q)
    what = f"{kind} {frac} schedule {sched}"
    check_flux(gt, ot, Q, o.volumes(), p.sigma_t[o.fsr_materials()], what=what)
    check_tally(gt, ot, what=what)
    assert abs(gl - ol) <= 2e-5 * abs(ol)
    # against the default schedule's sweep: rounding-level differences only
    assert np.abs(gt - base).max() <= 1e-5 * np.abs(base).max()
    tr.close()
