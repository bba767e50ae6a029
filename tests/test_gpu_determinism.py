"""FP32 solves with the shared tally are deterministic: the units' tallies
are summed in exact fixed point and every reduction has a fixed order, so the
same sweep or solve repeated gives the same bits (the order in which work
units finish on the device changes from run to run)."""
import numpy as np
import pytest

import synth
from paper_2503_17743_gb300 import MOC_FP32, MOC_SCHED_ROWS_WITH_SIGMA, Geometry, Tracks, track_params

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


@pytest.mark.parametrize("name,chunk", [("lattice5", 0), ("lattice5_rings", 0), ("lattice17_small", 0),
                                        ("lattice5", 3), ("lattice17_small", 7)])
def test_material_keyed_rows_give_the_same_bits(name, chunk):
    """Where every radial region has one material in all layers, the stored
    segments carry it and the shared rows hold Qr only, Sigma_t coming from
    the material table: the same values enter Eq. 3, so a sweep's tallies and
    an iterated solve's k and flux are the same bits as with rows that carry
    Sigma_t; so too for units swept in radial chunks of a given size."""
    p = synth.workload(name)
    g = Geometry(p)
    Q = np.random.default_rng(5).uniform(0.2, 1.0, size=(p.n_fsr, p.num_groups))
    outs = []
    for sched, keyed in ((0, 1), (MOC_SCHED_ROWS_WITH_SIGMA, 0)):
        tr = Tracks(g, track_params(p, precision=MOC_FP32, groups_per_lane=2, schedule=sched,
                                    chunk_segments=chunk))
        assert tr.info["material_keys"] == keyed
        assert tr.info["chunk_segments"] == chunk
        t, lk = tr.sweep_from_source(Q)
        tr.reset()
        tr.iterate(12)
        phi, k = tr.flux()
        outs.append((t, lk, k, phi))
        tr.close()
    np.testing.assert_array_equal(outs[0][0], outs[1][0])
    # (the leakage is summed in FP32 per lane, in the order a lane takes its
    # tracks, which changes from run to run: equal to FP32 rounding)
    assert outs[0][1] == pytest.approx(outs[1][1], rel=1e-6)
    assert outs[0][2] == outs[1][2]
    np.testing.assert_array_equal(outs[0][3], outs[1][3])


def test_material_keys_need_one_material_per_region():
    """asm1_absorber puts an absorber in the top layer of some guide tubes: a
    region whose material changes with the layer keeps Sigma_t in the rows."""
    p = synth.workload("asm1_absorber")
    tr = Tracks(Geometry(p), track_params(p, precision=MOC_FP32, groups_per_lane=2))
    assert tr.info["material_keys"] == 0
    tr.close()
