"""The serving engine (moc_server_*): every solve gives the same answer alone
and in a mix of resident solves, admission respects the memory budget,
requests submitted while others run are served (continuous batching), and a
request that fails (not converged, over the memory budget, an unsupported
mesh) gets its own error status without disturbing its neighbours."""
import numpy as np
import pytest

import synth
from paper_2503_17743_gb300 import Geometry, Server, Tracks, track_params
from paper_2503_17743_gb300 import _moc

pytestmark = pytest.mark.gpu

TOL = dict(tol_k=1e-7, tol_src=1e-6, max_iter=4000)


def requests(n, seed=5):
    return [synth.serving_request(seed, i) for i in range(n)]


def alone(p):
    tr = Tracks(Geometry(p), track_params(p))
    if p.ext_source is None:
        r = tr.solve_eigen(**TOL)
    else:
        r = tr.solve_fixed_source(tol_src=TOL["tol_src"], max_iter=TOL["max_iter"])
    phi, _ = tr.flux()
    tr.close()
    return r, phi


def check_same(r_mix, phi_mix, r_alone, phi_alone):
    """The same iterations on the same data give the same numbers: the FP32
    sweep's FSR tallies are summed in exact fixed point (three 64-bit words
    per FSR-group; integer adds, so the order
    in which work units finish does not matter) and every reduction has a
    fixed order, so a solve in a mix repeats its solve alone bit for bit."""
    assert r_mix["iterations"] == r_alone["iterations"]
    assert r_mix["iterations"] < TOL["max_iter"]
    assert r_mix["k"] == r_alone["k"], (r_mix["k"], r_alone["k"])
    np.testing.assert_array_equal(phi_mix, phi_alone)


def drain(srv, tickets, limit=100000):
    out = {}
    for _ in range(limit):
        srv.step()
        for t in tickets:
            if t not in out:
                r = srv.result(t)
                if r is not None:
                    out[t] = r
        if len(out) == len(tickets):
            return out
    raise AssertionError("server did not finish")


def test_mix_matches_alone():
    probs = requests(8)
    ref = [alone(p) for p in probs]
    srv = Server(max_active=4, iterations_per_poll=8)
    geoms = [Geometry(p) for p in probs]
    tickets = [srv.submit(g, track_params(p), **TOL) for g, p in zip(geoms, probs)]
    out = drain(srv, tickets)
    for t, (r0, phi0) in zip(tickets, ref):
        r, phi, queued, latency, rc = out[t]
        assert rc == 0 and latency >= queued >= 0.0
        check_same(r, phi, r0, phi0)
    st = srv.stats()
    assert st["retired"] == len(probs) and st["resident"] == 0 and st["queued"] == 0
    assert 1 < st["max_resident"] <= 4
    srv.close()


def test_quantum_does_not_change_results():
    probs = requests(3, seed=9)
    res = []
    for q in (1, 13):
        srv = Server(max_active=3, iterations_per_poll=q)
        geoms = [Geometry(p) for p in probs]
        tickets = [srv.submit(g, track_params(p), **TOL) for g, p in zip(geoms, probs)]
        out = drain(srv, tickets)
        res.append([out[t] for t in tickets])
        srv.close()
    for a, b in zip(*res):
        check_same(a[0], a[1], b[0], b[1])


def test_memory_budget_limits_residency():
    probs = requests(6, seed=11)
    geoms = [Geometry(p) for p in probs]
    params = [track_params(p) for p in probs]
    foot = [sum(g.footprint(tp)) for g, tp in zip(geoms, params)]
    budget = max(foot) + min(foot) // 2  # never room for the two largest together
    srv = Server(max_active=6, memory_budget_bytes=budget)
    tickets = [srv.submit(g, tp, **TOL) for g, tp in zip(geoms, params)]
    peak = 0
    out = {}
    while len(out) < len(tickets):
        srv.step()
        st = srv.stats()
        assert st["bytes_resident"] <= budget or st["resident"] == 1
        peak = max(peak, st["resident"])
        for t in tickets:
            if t not in out:
                r = srv.result(t)
                if r is not None:
                    out[t] = r
    assert all(out[t][4] == 0 for t in tickets)
    srv.close()


def test_requests_arriving_while_others_run():
    probs = requests(6, seed=13)
    ref = [alone(p) for p in probs]
    srv = Server(max_active=4)
    geoms = [Geometry(p) for p in probs]
    tickets = []
    out = {}
    for i, (g, p) in enumerate(zip(geoms, probs)):
        tickets.append(srv.submit(g, track_params(p), **TOL))
        for _ in range(2):  # a couple of steps before the next arrival
            srv.step()
            for t in tickets:
                if t not in out:
                    r = srv.result(t)
                    if r is not None:
                        out[t] = r
    out.update({t: r for t, r in drain(srv, [t for t in tickets if t not in out]).items()})
    for t, (r0, phi0) in zip(tickets, ref):
        check_same(out[t][0], out[t][1], r0, phi0)
    srv.close()


def test_failing_requests_do_not_disturb_neighbours():
    good = requests(3, seed=17)
    ref = [alone(p) for p in good]
    # a ringed, sectored lattice: its flux array is larger than 2 regions a pin
    rings = synth.workload("lattice5_rings")
    ref_rings = alone(rings)
    # an axial mesh off the lattice (a plane at 0.6 cm with 0.5 cm spacing):
    # served like the others
    off = synth.pin_cell(1, n_layers=3).with_tracks(layer_z=np.array([0.0, 0.6, 1.5, 2.0]))
    ref_off = alone(off)
    # more than 32 polar angles: refused at track generation
    bad = synth.pin_cell(1).with_tracks(n_polar=34)
    srv = Server(max_active=4, iterations_per_poll=8)
    geoms = {}
    tickets = {}
    for i, p in enumerate(good):
        geoms[f"good{i}"] = Geometry(p)
        tickets[f"good{i}"] = srv.submit(geoms[f"good{i}"], track_params(p), **TOL)
    geoms["few"] = Geometry(good[0])
    tickets["few"] = srv.submit(geoms["few"], track_params(good[0]), tol_k=1e-12, tol_src=1e-12,
                                max_iter=3)
    geoms["off"] = Geometry(off)
    tickets["off"] = srv.submit(geoms["off"], track_params(off), **TOL)
    geoms["bad"] = Geometry(bad)
    tickets["bad"] = srv.submit(geoms["bad"], track_params(bad), **TOL)
    geoms["rings"] = Geometry(rings)
    tickets["rings"] = srv.submit(geoms["rings"], track_params(rings), **TOL)
    out = {}
    order = list(tickets)
    for _ in range(100000):
        srv.step()
        for name in order:
            if name not in out:
                r = srv.result(tickets[name], check=False)
                if r is not None:
                    out[name] = r
        if len(out) == len(order):
            break
    assert len(out) == len(order)
    # max_iter reached first: NOT_CONVERGED with the last k of 3 iterations
    r, phi, _, _, rc = out["few"]
    assert rc == _moc.MOC_ERR_NOT_CONVERGED and r["iterations"] == 3 and np.isfinite(r["k"])
    tr = Tracks(Geometry(good[0]), track_params(good[0]))
    r3 = tr.iterate(3)
    assert abs(r["k"] - r3["k"]) < 1e-5
    tr.close()
    assert out["rings"][4] == 0 and out["rings"][1].shape == (rings.n_fsr, rings.num_groups)
    check_same(out["rings"][0], out["rings"][1], *ref_rings)
    # the off-lattice solve: its FSR tally is summed with FP64 atomics, so
    # alone and in the mix agree to rounding rather than bit for bit
    r, phi, _, _, rc = out["off"]
    assert rc == 0 and abs(r["iterations"] - ref_off[0]["iterations"]) <= 1
    assert abs(r["k"] - ref_off[0]["k"]) < 1e-9
    np.testing.assert_allclose(phi, ref_off[1], rtol=1e-6)
    assert out["bad"][4] == _moc.MOC_ERR_UNSUPPORTED
    for i in range(len(good)):
        r, phi, _, _, rc = out[f"good{i}"]
        assert rc == 0
        check_same(r, phi, *ref[i])
    srv.close()


def test_request_over_the_budget_is_rejected():
    probs = requests(3, seed=19)
    geoms = [Geometry(p) for p in probs]
    params = [track_params(p) for p in probs]
    foot = [sum(g.footprint(tp)) for g, tp in zip(geoms, params)]
    big = int(np.argmax(foot))
    budget = max(f for i, f in enumerate(foot) if i != big) if foot.count(max(foot)) == 1 else None
    if budget is None or budget >= foot[big]:
        pytest.skip("no request is larger than the others")
    ref = {i: alone(p) for i, p in enumerate(probs) if i != big}
    srv = Server(max_active=3, memory_budget_bytes=budget)
    tickets = [srv.submit(g, tp, **TOL) for g, tp in zip(geoms, params)]
    out = {}
    for _ in range(100000):
        srv.step()
        for i, t in enumerate(tickets):
            if i not in out:
                r = srv.result(t, check=False)
                if r is not None:
                    out[i] = r
        if len(out) == len(tickets):
            break
    assert out[big][4] == _moc.MOC_ERR_OUT_OF_MEMORY
    for i, (r0, phi0) in ref.items():
        assert out[i][4] == 0
        check_same(out[i][0], out[i][1], r0, phi0)
    assert srv.stats()["retired"] == len(tickets)
    srv.close()
