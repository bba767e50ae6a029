"""Solve states sharing one layout (moc_state_create) and the batched outer
iteration (moc_batch_step: the sweeps of several solves in one persistent
launch), against independent solves and the FP64 oracle."""
import dataclasses

import numpy as np
import pytest

import oracle
import synth
from paper_2503_17743_gb300 import (MOC_FP32, MOC_FP64, MOC_TALLY_GLOBAL, Geometry, MocError, Tracks,
                                    batch_step, track_params)

pytestmark = pytest.mark.gpu


def _fixed(seed=3):
    return synth.lattice(seed, n=3, G=3, height=4.0, n_layers=4, n_azim=8, n_polar=4,
                         radial_spacing=0.15, axial_spacing=0.5, bc=(1, 0, 1, 1, 0, 1), n_gt=2,
                         fixed_source=True, name="lat3_fixed")


@pytest.mark.parametrize("prec,tol", [(MOC_FP64, 1e-11), (MOC_FP32, 1e-5)])
def test_state_is_an_independent_solve(prec, tol):
    p = synth.workload("lattice5")
    g = Geometry(p)
    base = Tracks(g, track_params(p, precision=prec))
    st = base.state()
    # the state shares the stored templates and tables: far less memory
    assert st.info["device_bytes"] < base.info["device_bytes"]
    assert st.info["stored_segments"] == base.info["stored_segments"]
    r1 = base.iterate(12)
    r2 = st.iterate(12)
    o = oracle.Oracle(p)
    o.reset()
    ref = o.iterate(12)
    for r, t in ((r1, base), (r2, st)):
        phi, k = t.flux()
        assert r["iterations"] == 12
        assert abs(k - ref["k"]) < tol
        np.testing.assert_allclose(phi, o.flux(), rtol=10 * tol)
    # the layout outlives its owner's handle while a state uses it, but takes
    # no new states once the owner is closed
    base.close()
    with pytest.raises(MocError):
        st.state()
    r3 = st.iterate(3)
    assert r3["iterations"] == 3
    st.close()


def test_state_with_its_own_external_source():
    """A fixed-source state with twice the source: the problem is linear, so
    its flux is twice the layout owner's, and it matches the oracle on the
    problem with that source."""
    p = _fixed()
    g = Geometry(p)
    base = Tracks(g, track_params(p, precision=MOC_FP64))
    st = base.state(ext_source=2.0 * p.ext_source)
    base.solve_fixed_source(tol_src=1e-11, max_iter=3000)
    st.solve_fixed_source(tol_src=1e-11, max_iter=3000)
    phi1, _ = base.flux()
    phi2, _ = st.flux()
    np.testing.assert_allclose(phi2, 2.0 * phi1, rtol=1e-9)
    o = oracle.Oracle(dataclasses.replace(p, ext_source=2.0 * p.ext_source))
    o.reset()
    o.iterate(40)
    st2 = base.state(ext_source=2.0 * p.ext_source)
    st2.iterate(40)
    np.testing.assert_allclose(st2.flux()[0], o.flux(), rtol=1e-10)
    for t in (st2, st, base):
        t.close()


@pytest.mark.parametrize("prec,rtol", [(MOC_FP64, 1e-11), (MOC_FP32, 2e-5)])
@pytest.mark.parametrize("name", ["lattice5", "lat3_fixed"])
def test_batch_step_matches_each_solve_alone(name, prec, rtol):
    """Three solves of one layout (the owner and two states; for the fixed
    source problem with three different sources) advanced by batched
    iterations equal the same solves iterated one by one, and the oracle."""
    p = synth.workload("lattice5") if name == "lattice5" else _fixed()
    g = Geometry(p)
    srcs = [None, None, None] if p.ext_source is None else [None, 0.5 * p.ext_source, 3.0 * p.ext_source]
    owner = Tracks(g, track_params(p, precision=prec))
    batch = [owner] + [owner.state(ext_source=s) for s in srcs[1:]]
    alone_owner = Tracks(g, track_params(p, precision=prec))
    alone = [alone_owner] + [alone_owner.state(ext_source=s) for s in srcs[1:]]
    n = 10
    for _ in range(n):
        batch_step(batch)
    for t in alone:
        t.iterate(n)
    for i, (a, b) in enumerate(zip(batch, alone)):
        pa, ka = a.flux()
        pb, kb = b.flux()
        assert abs(ka - kb) < (1e-12 if prec == MOC_FP64 else 1e-6), i
        np.testing.assert_allclose(pa, pb, rtol=rtol, err_msg=f"solve {i}")
    # the first solve against the oracle
    o = oracle.Oracle(p)
    o.reset()
    ref = o.iterate(n)
    phi, k = batch[0].flux()
    assert abs(k - ref["k"]) < (1e-11 if prec == MOC_FP64 else 1e-5)
    np.testing.assert_allclose(phi, o.flux(), rtol=1e-10 if prec == MOC_FP64 else 1e-4)
    for t in batch[1:] + alone[1:] + [owner, alone_owner]:
        t.close()


def test_batch_step_global_tally_runs_per_solve():
    p = synth.workload("lattice5")
    g = Geometry(p)
    owner = Tracks(g, track_params(p, tally_mode=MOC_TALLY_GLOBAL))
    st = owner.state()
    for _ in range(5):
        batch_step([owner, st])
    ref = Tracks(g, track_params(p, tally_mode=MOC_TALLY_GLOBAL))
    ref.iterate(5)
    np.testing.assert_allclose(st.flux()[0], ref.flux()[0], rtol=1e-5)
    for t in (st, owner, ref):
        t.close()


def test_batch_step_rejects_mixed_layouts():
    p = synth.workload("lattice5")
    a = Tracks(Geometry(p), track_params(p))
    b = Tracks(Geometry(p), track_params(p))
    with pytest.raises(MocError):
        batch_step([a, b])
    with pytest.raises(MocError):
        batch_step([a, a])
    a.close()
    b.close()


def test_states_and_batch_step_off_the_lattice():
    """A layout with layer planes off the axial lattice: its solve states
    share the off-lattice tables, and batched steps (one iteration per solve:
    the off-lattice sweep tallies globally) equal the solves iterated alone
    and the oracle."""
    p = synth.workload("lattice5_offaxial")
    g = Geometry(p)
    owner = Tracks(g, track_params(p))
    assert owner.info["off_lattice"] == 1
    st = owner.state()
    for _ in range(8):
        batch_step([owner, st])
    o = oracle.Oracle(p)
    o.reset()
    ref = o.iterate(8)
    for t in (owner, st):
        phi, k = t.flux()
        assert abs(k - ref["k"]) < 1e-5
        np.testing.assert_allclose(phi, o.flux(), rtol=1e-4)
    st.close()
    owner.close()
