"""FP32 solves with the shared tally are deterministic: the units' tallies
are summed in exact fixed point and every reduction has a fixed order, so the
same sweep or solve repeated gives the same bits (the order in which work
units finish on the device changes from run to run)."""
import numpy as np
import pytest

import synth
from paper_2503_17743_gb300 import MOC_FP32, Geometry, Tracks, track_params

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name", ["lattice5", "lattice5_rings", "asm1_absorber"])
def test_sweep_repeats_bit_for_bit(name):
    p = synth.workload(name)
    tr = Tracks(Geometry(p), track_params(p, precision=MOC_FP32))
    Q = np.random.default_rng(3).uniform(0.2, 1.0, size=(tr.n_fsr, p.num_groups))
    outs = []
    for _ in range(3):
        tr.reset()
        outs.append(tr.sweep_from_source(Q)[0])
    np.testing.assert_array_equal(outs[0], outs[1])
    np.testing.assert_array_equal(outs[0], outs[2])
    tr.close()


@pytest.mark.parametrize("name", ["lattice5", "lattice17_small"])
def test_solve_repeats_bit_for_bit(name):
    p = synth.workload(name)
    g = Geometry(p)
    res = []
    for _ in range(2):
        tr = Tracks(g, track_params(p, precision=MOC_FP32))
        r = tr.solve_eigen(tol_k=1e-7, tol_src=1e-6, max_iter=4000)
        phi, k = tr.flux()
        res.append((r["iterations"], k, phi))
        tr.close()
    assert res[0][0] == res[1][0]
    assert res[0][1] == res[1][1]
    np.testing.assert_array_equal(res[0][2], res[1][2])
