"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Bars: FSR-id sequences and segment counts bit-exact; FP32 segment lengths
within 1e-6 (relative) + 1e-6 cm; tallies, fluxes and k within the stated
tolerances (FP64 sweeps ~1e-10, FP32 sweeps: flux 1e-4 max relative, k 1e-5
absolute).
"""
import os

import numpy as np
import pytest

import oracle
import synth
from paper_2503_17743_gb300 import (MOC_FP32, MOC_FP64, MOC_TALLY_GLOBAL, MOC_TALLY_SHARED,
                                    Geometry, Tracks, track_params)

from tests.parity import check_flux, check_tally

pytestmark = pytest.mark.gpu

NTH = os.cpu_count() or 4


def _lat3(bc=(1, 1, 1, 1, 1, 1), seed=3):
    return synth.lattice(seed, n=3, G=3, height=4.0, n_layers=4, n_azim=8, n_polar=4,
                         radial_spacing=0.15, axial_spacing=0.5, bc=bc, n_gt=2, name="lat3")


PROBLEMS = {
    "pin": lambda: synth.pin_cell(1),
    "lat3": lambda: _lat3(),
    "lat3_mixed": lambda: _lat3(bc=(1, 0, 1, 1, 0, 1), seed=4),
    "lattice5": lambda: synth.workload("lattice5"),
    "l17_small": lambda: synth.workload("lattice17_small"),
    # finer pin-cell regions: rings and angular sectors
    "lat3_rings": lambda: _lat3(bc=(1, 0, 1, 1, 0, 1), seed=5).with_tracks(
        fuel_rings=2, moderator_rings=1, sectors=8, name="lat3_rings"),
    "lattice5_rings": lambda: synth.workload("lattice5_rings"),
}

_cache = {}


def get(name):
    if name not in _cache:
        p = PROBLEMS[name]()
        _cache[name] = (p, oracle.Oracle(p, n_threads=NTH), Geometry(p))
    return _cache[name]


def make(name, **kw):
    p, o, g = get(name)
    return p, o, Tracks(g, track_params(p, **kw))


@pytest.mark.parametrize("name", list(PROBLEMS))
def test_segments_bit_exact(name):
    p, o, tr = make(name)
    step = max(1, o.n_tracks2d // 60)
    for t in range(0, o.n_tracks2d, step):
        for pp in range(p.n_polar):
            oi, on, of, ol = o.stack(t, pp)
            gi, gn, gf, gl = tr.stack_segments(t, pp)
            np.testing.assert_array_equal(gi, oi, err_msg=f"track indices t={t} p={pp}")
            np.testing.assert_array_equal(gn, on, err_msg=f"segment counts t={t} p={pp}")
            np.testing.assert_array_equal(gf, of, err_msg=f"fsr ids t={t} p={pp}")
            assert np.all(np.abs(gl - ol) <= 1e-6 * ol + 1e-6), (t, pp, np.abs(gl - ol).max())
    tr.close()


@pytest.mark.parametrize("name", list(PROBLEMS))
def test_volumes(name):
    p, o, tr = make(name)
    np.testing.assert_allclose(tr.volumes(), o.volumes(), rtol=1e-6)
    info = tr.info
    assert info["tracks3d"] == o.n_tracks3d
    tr.close()


def sweep_bars(prec, name=""):
    """(relative bar above the floor, absolute bar over the largest tally,
    flux bar) of one sweep's tallies in each precision.  FP32 pins split into
    rings and sectors have optically thin regions (chords of a few hundredths
    of a cm): their contributions are small against the unit's fixed-point
    grid and against the absolute error of the FP32 escape fraction
    1 - 2^-x (about 2^-22, reading of Eq. 3 in FP32), so their tallies carry
    a few 1e-4 relative; the flux they give stays within 1e-5 (the bar below
    is the metric's 1e-4)."""
    if prec == MOC_FP64:
        return 1e-9, 1e-11, 1e-10
    return (5e-4 if "rings" in name else 1e-4), 2e-5, 1e-4


@pytest.mark.parametrize("prec", [MOC_FP64, MOC_FP32])
@pytest.mark.parametrize("name", ["pin", "lat3", "lat3_mixed", "l17_small", "lat3_rings"])
def test_two_sweeps_from_source(name, prec):
    """Seeded source, zero incoming fluxes, two sweeps: the second one runs on
    the boundary fluxes the first one passed through the links.  Tallies
    element by element (relative above a floor of 1e-3 of the largest,
    absolute below it) and the flux they give on every FSR-group."""
    p, o, tr = make(name, precision=prec)
    rel, absb, frel = sweep_bars(prec, name)
    rng = np.random.default_rng(11)
    Q = rng.uniform(0.2, 1.0, size=(o.n_fsr, p.num_groups))
    sigt = p.sigma_t[o.fsr_materials()]
    o.reset()
    for sweep in range(2):
        ot, ol = o.sweep_once(Q)
        gt, gl = tr.sweep_from_source(Q)
        check_flux(gt, ot, Q, o.volumes(), sigt, rel=frel, what=f"{name} sweep {sweep}")
        check_tally(gt, ot, rel=rel, abs_frac=absb, what=f"{name} sweep {sweep}")
        assert abs(gl - ol) <= absb * max(abs(ol), 1e-300) + 1e-300
    o.reset()
    tr.close()


def _asm1():
    """One assembly with the reflector on two sides and an absorber in the top
    layer of a seeded half of its guide tubes: regions whose material changes
    with the layer (Sigma_t per row, not per 2D segment)."""
    return synth.assemblies(seed=2, n_asm=1, height=8.0, n_layers=4, absorber_height=2.0,
                            n_azim=8, n_polar=4, radial_spacing=0.1, axial_spacing=0.5)


PROBLEMS["asm1_absorber"] = _asm1


@pytest.mark.parametrize("sync", [1, 4, 8])
@pytest.mark.parametrize("name", ["lat3_mixed", "l17_small", "lattice5_rings", "asm1_absorber"])
def test_sync_blocks_sweep_and_iterate_like_the_oracle(name, sync):
    """Every warp schedule of the stored stacks (each track on its own
    records, or synchronous blocks of 4 or 8 tracks of one template) gives
    the oracle's sweep element by element and its power iterations."""
    p, o, tr = make(name, precision=MOC_FP32, sync_block=sync)
    info = tr.info
    if info["groups_per_lane"] == 2 and info["chunk_segments"] == 0 and info["tally_mode"] == MOC_TALLY_SHARED:
        assert info["sync_block"] == min(sync, 32 // info["lanes_per_track"]) or sync == 1
    rng = np.random.default_rng(13)
    Q = rng.uniform(0.2, 1.0, size=(o.n_fsr, p.num_groups))
    o.reset()
    ot, ol = o.sweep_once(Q)
    gt, gl = tr.sweep_from_source(Q)
    check_flux(gt, ot, Q, o.volumes(), p.sigma_t[o.fsr_materials()], what=f"{name} sync {sync}")
    assert np.abs(gt - ot).max() <= 2e-5 * np.abs(ot).max()
    assert abs(gl - ol) <= 2e-5 * abs(ol)
    o.reset()
    tr.reset()
    ref = o.iterate(15)
    res = tr.iterate(15)
    phi, k = tr.flux()
    assert abs(k - ref["k"]) < 1e-5, (k, ref["k"])
    np.testing.assert_allclose(phi, o.flux(), rtol=1e-4)
    o.reset()
    tr.close()


@pytest.mark.parametrize("name", ["lat3", "lat3_mixed"])
def test_single_track_links(name):
    """Q = 0 and one incoming flux: the flux arrives attenuated at exactly the
    track direction the oracle's geometric link names."""
    p, o, tr = make(name, precision=MOC_FP64)
    rng = np.random.default_rng(5)
    G = p.num_groups
    zero = np.zeros((o.n_fsr, G))
    for _ in range(12):
        t = int(rng.integers(o.n_tracks2d))
        pp = int(rng.integers(p.n_polar))
        imin, n = o.stack_range(t, pp)
        i = imin + int(rng.integers(n))
        s = int(rng.integers(2))
        val = rng.uniform(0.5, 2.0, size=G)
        o.reset(); o.clear_psi()
        tr.reset()
        o.psi(t, pp, i, s, val)
        tr.psi(t, pp, i, s, val)
        ot, _ = o.sweep_once(zero)
        gt, _ = tr.sweep_from_source(zero)
        np.testing.assert_allclose(gt, ot, rtol=1e-12, atol=1e-14)
        d = o.link(t, pp, i, s)
        if d[0] >= 0:
            np.testing.assert_allclose(tr.psi(*d), o.psi(*d), rtol=1e-12)
            assert np.all(o.psi(*d) > 0)
    o.reset()
    tr.close()


@pytest.mark.parametrize("prec,ktol,ftol", [(MOC_FP64, 1e-11, 1e-10), (MOC_FP32, 1e-5, 1e-4)])
@pytest.mark.parametrize("name", ["pin", "lat3_mixed", "lattice5", "l17_small", "lattice5_rings"])
def test_power_iterations(name, prec, ktol, ftol):
    p, o, tr = make(name, precision=prec)
    n = 15
    o.reset()
    ref = o.iterate(n)
    res = tr.iterate(n, use_graph=True)
    phi, k = tr.flux()
    assert res["iterations"] == n
    assert abs(k - ref["k"]) < ktol, (k, ref["k"])
    np.testing.assert_allclose(phi, o.flux(), rtol=ftol)
    tr.close()


def test_converged_pin_cell_fp64():
    p, o, tr = make("pin", precision=MOC_FP64)
    ref = o.solve(tol_k=1e-10, tol_src=1e-9, max_iter=5000)
    res = tr.solve_eigen(tol_k=1e-10, tol_src=1e-9, max_iter=5000)
    assert ref["converged"] and res["converged"]
    assert abs(res["k"] - ref["k"]) < 1e-10
    assert abs(res["iterations"] - ref["iterations"]) <= 1
    phi, _ = tr.flux()
    np.testing.assert_allclose(phi, o.flux(), rtol=1e-9)
    # balance: production / k = absorption (all faces reflective), to the
    # convergence level of the solve
    assert abs(1.0 / res["k"] - res["absorption"]) < 1e-7
    tr.close()


@pytest.mark.parametrize("prec,tol", [(MOC_FP64, 1e-9), (MOC_FP32, 1e-5)])
def test_infinite_medium_closed_form(prec, tol):
    p = synth.pin_cell(1, homogeneous=True)
    tr = Tracks(Geometry(p), track_params(p, precision=prec))
    res = tr.solve_eigen(tol_k=1e-12 if prec == MOC_FP64 else 1e-8,
                         tol_src=1e-11 if prec == MOC_FP64 else 1e-6, max_iter=20000)
    st, ss, nsf, chi = p.sigma_t[0], p.sigma_s[0], p.nu_sigma_f[0], p.chi[0]
    kinf = nsf @ np.linalg.solve(np.diag(st) - ss.T, chi)
    assert abs(res["k"] - kinf) < tol
    tr.close()


@pytest.mark.parametrize("prec,tol", [(MOC_FP64, 1e-9), (MOC_FP32, 1e-5)])
def test_fixed_source(prec, tol):
    p = synth.pin_cell(5, G=3, homogeneous=True)
    p = p.with_tracks(nu_sigma_f=np.zeros_like(p.nu_sigma_f),
                      ext_source=np.tile([[1.0, 0.4, 0.2]], (p.num_materials, 1)))
    tr = Tracks(Geometry(p), track_params(p, precision=prec))
    res = tr.solve_fixed_source(tol_src=1e-11 if prec == MOC_FP64 else 1e-6, max_iter=20000)
    ref = np.linalg.solve(np.diag(p.sigma_t[0]) - p.sigma_s[0].T, p.ext_source[0])
    phi, _ = tr.flux()
    np.testing.assert_allclose(phi, np.tile(ref, (phi.shape[0], 1)), rtol=tol)
    tr.close()
    # heterogeneous fixed-source lattice vs the oracle after n iterations
    q = synth.lattice(8, n=3, G=4, height=4.0, n_layers=2, n_azim=8, n_polar=4,
                      radial_spacing=0.2, axial_spacing=0.5, fixed_source=True)
    o = oracle.Oracle(q, n_threads=NTH)
    o.reset()
    o.iterate(12)
    tr = Tracks(Geometry(q), track_params(q, precision=prec))
    tr.iterate(12)
    phi, _ = tr.flux()
    np.testing.assert_allclose(phi, o.flux(), rtol=1e-9 if prec == MOC_FP64 else 1e-4)
    tr.close()


@pytest.mark.parametrize("name", ["lat3_mixed", "l17_small"])
def test_stored_and_generated_segments_agree(name):
    """Preload budgets: everything stored (EXP), nothing stored (OTF), and a
    partial budget give the same sweep (Sec. 4.2)."""
    p, o, _ = get(name)
    Q = np.random.default_rng(2).uniform(0.2, 1.0, size=(o.n_fsr, p.num_groups))
    outs, infos = [], []
    full = Tracks(get(name)[2], track_params(p, preload_budget_bytes=-1))
    half_budget = full.info["stored_segments"] * 8 // 2
    full.close()
    for budget in (-1, 0, half_budget):
        tr = Tracks(get(name)[2], track_params(p, preload_budget_bytes=budget))
        infos.append(tr.info)
        outs.append([tr.sweep_from_source(Q)[0], tr.sweep_from_source(Q)[0]])
        tr.close()
    # stored templates: one per class of each stack, far fewer pieces than segments
    assert 0 < infos[0]["stored_segments"] * 2 < infos[0]["segments3d"]
    assert infos[0]["preloaded_stacks"] == infos[0]["stacks"] // 2
    assert infos[1]["stored_segments"] == 0
    assert 0 < infos[2]["preloaded_stacks"] < infos[0]["preloaded_stacks"]
    for run in outs[1:]:
        for a, b in zip(run, outs[0]):
            # FP32 sweeps: the same contributions summed in a different order
            np.testing.assert_allclose(a, b, rtol=1e-5, atol=1e-6 * np.abs(b).max())


def test_tally_modes_agree():
    p, o, g = get("l17_small")
    Q = np.random.default_rng(4).uniform(0.2, 1.0, size=(o.n_fsr, p.num_groups))
    res = []
    for mode in (MOC_TALLY_SHARED, MOC_TALLY_GLOBAL):
        tr = Tracks(g, track_params(p, tally_mode=mode))
        assert tr.info["tally_mode"] == mode
        res.append(tr.sweep_from_source(Q)[0])
        tr.close()
    np.testing.assert_allclose(res[0], res[1], rtol=1e-5, atol=1e-6 * np.abs(res[0]).max())


def test_graph_and_stream_agree():
    p, o, g = get("lattice5")
    a = Tracks(g, track_params(p))
    b = Tracks(g, track_params(p))
    ra = a.iterate(10, use_graph=True)
    rb = b.iterate(10, use_graph=False)
    assert abs(ra["k"] - rb["k"]) < 1e-6
    np.testing.assert_allclose(a.flux()[0], b.flux()[0], rtol=1e-5)
    a.close()
    b.close()


@pytest.mark.parametrize("gpl", [1, 2, 4])
@pytest.mark.parametrize("name", ["lat3_mixed", "l17_small"])
def test_groups_per_lane_against_oracle(name, gpl):
    """Every lane shape (1, 2 or 4 groups per lane) sweeps like the oracle."""
    p, o, g = get(name)
    tr = Tracks(g, track_params(p, groups_per_lane=gpl))
    assert tr.info["groups_per_lane"] == gpl
    Q = np.random.default_rng(6).uniform(0.2, 1.0, size=(o.n_fsr, p.num_groups))
    o.reset()
    for sweep in range(2):
        ot, ol = o.sweep_once(Q)
        gt, gl = tr.sweep_from_source(Q)
        scale = np.abs(ot).max()
        assert np.abs(gt - ot).max() <= 2e-5 * scale, (sweep, np.abs(gt - ot).max() / scale)
        assert abs(gl - ol) <= 2e-5 * max(abs(ol), 1e-300) + 1e-300
    o.reset()
    tr.close()


# --------------------------------------------------------------- radial chunks

def _half_budget(name):
    p, o, g = get(name)
    full = Tracks(g, track_params(p, preload_budget_bytes=-1))
    b = full.info["stored_segments"] * 8 // 2
    full.close()
    return b


@pytest.mark.parametrize("budget", ["all", "none", "half"])
@pytest.mark.parametrize("prec,rtol", [(MOC_FP64, 1e-11), (MOC_FP32, 2e-5)])
@pytest.mark.parametrize("name", ["lat3_mixed", "l17_small", "lat3_rings"])
def test_radial_chunks_against_oracle(name, prec, rtol, budget):
    """Units swept in radial chunks of 2 2D segments (psi handed from chunk to
    chunk, sense 0 outwards then sense 1 back): two sweeps from a seeded
    source match the oracle like the whole-unit sweep, with stored, generated
    and mixed segments."""
    p, o, g = get(name)
    b = {"all": -1, "none": 0, "half": _half_budget(name)}[budget]
    tr = Tracks(g, track_params(p, precision=prec, tally_mode=MOC_TALLY_SHARED,
                                preload_budget_bytes=b, chunk_segments=2))
    assert tr.info["chunk_segments"] == 2 and tr.info["tally_mode"] == MOC_TALLY_SHARED
    rng = np.random.default_rng(11)
    Q = rng.uniform(0.2, 1.0, size=(o.n_fsr, p.num_groups))
    o.reset()
    for sweep in range(2):
        ot, ol = o.sweep_once(Q)
        gt, gl = tr.sweep_from_source(Q)
        scale = np.abs(ot).max()
        assert np.abs(gt - ot).max() <= rtol * scale, (sweep, np.abs(gt - ot).max() / scale)
        assert abs(gl - ol) <= rtol * max(abs(ol), 1e-300) + 1e-300
    o.reset()
    tr.close()


@pytest.mark.parametrize("prec,ktol,ftol", [(MOC_FP64, 1e-11, 1e-10), (MOC_FP32, 1e-5, 1e-4)])
@pytest.mark.parametrize("name", ["lattice5", "lattice5_rings"])
def test_radial_chunks_power_iterations(name, prec, ktol, ftol):
    p, o, g = get(name)
    tr = Tracks(g, track_params(p, precision=prec, tally_mode=MOC_TALLY_SHARED, chunk_segments=3))
    assert tr.info["chunk_segments"] == 3
    n = 15
    o.reset()
    ref = o.iterate(n)
    res = tr.iterate(n, use_graph=True)
    phi, k = tr.flux()
    assert res["iterations"] == n
    assert abs(k - ref["k"]) < ktol, (k, ref["k"])
    np.testing.assert_allclose(phi, o.flux(), rtol=ftol)
    tr.close()


@pytest.mark.parametrize("prec,rtol", [(MOC_FP64, 1e-12), (MOC_FP32, 1e-5)])
@pytest.mark.parametrize("k", [2, 3])
def test_virtual_shards_sum_to_the_sweep(k, prec, rtol):
    """Angular decomposition on one GPU: k disjoint ranges of 2D tracks
    (whole azimuths in laydown order) swept separately from one source with
    zero incoming flux; their tallies and leakages sum to the sweep of all
    tracks, which is the all-reduce a sharded sweep would do."""
    p, o, g = get("lat3_mixed")
    tr = Tracks(g, track_params(p, precision=prec))
    Q = np.random.default_rng(5).uniform(0.2, 1.0, size=(o.n_fsr, p.num_groups))
    full, lf = tr.sweep_units_from_source(Q, 0, o.n_tracks2d)
    edges = np.linspace(0, o.n_tracks2d, k + 1).astype(int)
    parts = [tr.sweep_units_from_source(Q, int(a), int(b)) for a, b in zip(edges[:-1], edges[1:])]
    total = sum(t for t, _ in parts)
    np.testing.assert_allclose(total, full, rtol=rtol, atol=rtol * np.abs(full).max())
    assert abs(sum(lk for _, lk in parts) - lf) <= rtol * abs(lf) + 1e-300
    # and the shards partition the work: each one alone misses the others' part
    assert all(np.abs(t).sum() < np.abs(full).sum() for t, _ in parts)
    tr.close()


# --------------------------------------------------------------- unequal layers

def _lat3z(seed=6):
    """Unequal layers on the 0.5 cm axial lattice (0.5, 1.0, 1.5, 1.0 cm),
    mixed faces; the sweep runs on 0.5 cm layers mapped to these four."""
    p = synth.lattice(seed, n=3, G=3, height=4.0, n_layers=4, n_azim=8, n_polar=4,
                      radial_spacing=0.15, axial_spacing=0.5, bc=(1, 0, 1, 1, 0, 1), n_gt=2,
                      name="lat3z")
    return p.with_tracks(layer_z=np.array([0.0, 0.5, 1.5, 3.0, 4.0]))


def _merge_runs(fsr, ln):
    """Consecutive pieces in one FSR as one segment (the sweep's layers split
    a segment where the geometry's do not)."""
    if len(fsr) == 0:
        return fsr, ln
    keep = np.concatenate([[True], fsr[1:] != fsr[:-1]])
    idx = np.cumsum(keep) - 1
    return fsr[keep], np.bincount(idx, weights=ln)


UNEQUAL = {"lat3z": _lat3z, "lattice5_axial": lambda: synth.workload("lattice5_axial")}


@pytest.mark.parametrize("name", list(UNEQUAL))
def test_unequal_layers_segments_and_volumes(name):
    p = UNEQUAL[name]()
    o = oracle.Oracle(p, n_threads=NTH)
    tr = Tracks(Geometry(p), track_params(p))
    assert tr.info["n_fsr"] == o.n_fsr
    np.testing.assert_allclose(tr.volumes(), o.volumes(), rtol=1e-6)
    for t in range(0, o.n_tracks2d, max(1, o.n_tracks2d // 30)):
        for pp in range(p.n_polar):
            oi, on, of, ol = o.stack(t, pp)
            gi, gn, gf, gl = tr.stack_segments(t, pp)
            np.testing.assert_array_equal(gi, oi)
            go = np.concatenate([[0], np.cumsum(gn)])
            oo = np.concatenate([[0], np.cumsum(on)])
            for k in range(len(oi)):
                f, l = _merge_runs(gf[go[k]:go[k + 1]], gl[go[k]:go[k + 1]])
                np.testing.assert_array_equal(f, of[oo[k]:oo[k + 1]], err_msg=f"t={t} p={pp} k={k}")
                np.testing.assert_allclose(l, ol[oo[k]:oo[k + 1]], rtol=2e-6, atol=2e-6)
    tr.close()


@pytest.mark.parametrize("prec,ktol,ftol", [(MOC_FP64, 1e-11, 1e-10), (MOC_FP32, 1e-5, 1e-4)])
@pytest.mark.parametrize("name", list(UNEQUAL))
def test_unequal_layers_power_iterations(name, prec, ktol, ftol):
    p = UNEQUAL[name]()
    o = oracle.Oracle(p, n_threads=NTH)
    tr = Tracks(Geometry(p), track_params(p, precision=prec))
    o.reset()
    ref = o.iterate(15)
    tr.iterate(15)
    phi, k = tr.flux()
    assert abs(k - ref["k"]) < ktol, (k, ref["k"])
    np.testing.assert_allclose(phi, o.flux(), rtol=ftol)
    tr.close()


# ------------------------------------------- layer planes off the axial lattice

def _lat3o():
    """Planes 0.6, 1.7 and 3.1 cm with 0.5 cm spacing (fractions 0.2, 0.4 and
    0.2 of a spacing; the mirrored frame's 0.8 and 0.6), mixed faces."""
    return _lat3(bc=(1, 0, 1, 1, 0, 1), seed=7).with_tracks(layer_z=np.array([0.0, 0.6, 1.7, 3.1, 4.0]),
                                                            name="lat3o")


def _lat3_eq3():
    """Three equal layers of 4/3 cm with 0.5 cm spacing: planes 8/3 and 16/3
    spacings up (equal layers that are not whole spacings)."""
    return synth.lattice(8, n=3, G=3, height=4.0, n_layers=3, n_azim=8, n_polar=4,
                         radial_spacing=0.15, axial_spacing=0.5, bc=(1, 1, 1, 1, 1, 1), n_gt=2,
                         name="lat3_eq3")


def _pin_ties():
    """The pin cell with one plane where an upward track of a stack starts
    and one where a downward track starts: tracks that touch a plane at
    their first boundary (exact ties, decided from the FP64 layout)."""
    base = synth.pin_cell(1, n_layers=3)
    o0 = oracle.Oracle(base.with_tracks(layer_z=np.array([0.0, 0.6, 1.3, 2.0])), n_threads=1)

    def start_frac(p_idx):
        for t in range(o0.n_tracks2d):
            z = o0.stack_zeta(t, p_idx)[0]
            f = z - np.floor(z)
            if 0.05 < f < 0.95:
                return f
        raise AssertionError("no track start off the lattice")

    fu, fd = start_frac(0), start_frac(base.n_polar // 2)
    mesh = np.array([0.0, (1.0 + fu) * 0.5, (2.0 + fd) * 0.5, 2.0])
    return base.with_tracks(layer_z=mesh, name="pin_ties")


OFFLAT = {"lat3o": _lat3o, "lat3_eq3": _lat3_eq3, "pin_ties": _pin_ties,
          "lattice5_offaxial": lambda: synth.workload("lattice5_offaxial")}
_offlat_cache = {}


def get_offlat(name):
    if name not in _offlat_cache:
        p = OFFLAT[name]()
        _offlat_cache[name] = (p, oracle.Oracle(p, n_threads=NTH), Geometry(p))
    return _offlat_cache[name]


@pytest.mark.parametrize("prec", [MOC_FP32, MOC_FP64])
@pytest.mark.parametrize("name", list(OFFLAT))
def test_off_lattice_segments_bit_exact_and_volumes(name, prec):
    """Layer planes off the axial lattice (Sec. 2.2's local axial mesh):
    every listed stack's track indices, segment counts and FSR-id sequences
    equal the oracle's exactly, in both frames (upward and downward polar
    stacks); lengths within 1e-6 (FP32) or 1e-12 (FP64); tracked volumes."""
    p, o, g = get_offlat(name)
    tr = Tracks(g, track_params(p, precision=prec))
    assert tr.info["n_fsr"] == o.n_fsr and tr.info["tracks3d"] == o.n_tracks3d
    lrel = 1e-6 if prec == MOC_FP32 else 1e-12
    for t in range(0, o.n_tracks2d, max(1, o.n_tracks2d // 40)):
        for pp in range(p.n_polar):
            oi, on, of, ol = o.stack(t, pp)
            gi, gn, gf, gl = tr.stack_segments(t, pp)
            np.testing.assert_array_equal(gi, oi, err_msg=f"track indices t={t} p={pp}")
            np.testing.assert_array_equal(gn, on, err_msg=f"segment counts t={t} p={pp}")
            np.testing.assert_array_equal(gf, of, err_msg=f"fsr ids t={t} p={pp}")
            assert np.all(np.abs(gl - ol) <= lrel * ol + lrel), (t, pp, np.abs(gl - ol).max())
    np.testing.assert_allclose(tr.volumes(), o.volumes(), rtol=1e-6 if prec == MOC_FP32 else 1e-11)
    tr.close()


@pytest.mark.parametrize("prec", [MOC_FP64, MOC_FP32])
@pytest.mark.parametrize("name", list(OFFLAT))
def test_off_lattice_two_sweeps_from_source(name, prec):
    """Two sweeps from a seeded source through the off-lattice sweep: tallies
    element by element and the flux they give, as for the lattice meshes."""
    p, o, g = get_offlat(name)
    tr = Tracks(g, track_params(p, precision=prec))
    rel, absb, frel = sweep_bars(prec, name)
    Q = np.random.default_rng(13).uniform(0.2, 1.0, size=(o.n_fsr, p.num_groups))
    sigt = p.sigma_t[o.fsr_materials()]
    o.reset()
    for sweep in range(2):
        ot, ol = o.sweep_once(Q)
        gt, gl = tr.sweep_from_source(Q)
        check_flux(gt, ot, Q, o.volumes(), sigt, rel=frel, what=f"{name} sweep {sweep}")
        check_tally(gt, ot, rel=rel, abs_frac=absb, what=f"{name} sweep {sweep}")
        assert abs(gl - ol) <= absb * max(abs(ol), 1e-300) + 1e-300
    o.reset()
    tr.close()


@pytest.mark.parametrize("prec,ktol,ftol", [(MOC_FP64, 1e-11, 1e-10), (MOC_FP32, 1e-5, 1e-4)])
@pytest.mark.parametrize("name", list(OFFLAT))
def test_off_lattice_power_iterations(name, prec, ktol, ftol):
    p, o, g = get_offlat(name)
    tr = Tracks(g, track_params(p, precision=prec))
    o.reset()
    ref = o.iterate(15)
    res = tr.iterate(15, use_graph=True)
    phi, k = tr.flux()
    assert res["iterations"] == 15
    assert abs(k - ref["k"]) < ktol, (k, ref["k"])
    np.testing.assert_allclose(phi, o.flux(), rtol=ftol)
    o.reset()
    tr.close()


# --------------------------------------------------------------- group counts

def _lat2(G):
    return synth.lattice(6, n=2, G=G, height=2.0, n_layers=2, n_azim=8, n_polar=4,
                         radial_spacing=0.2, axial_spacing=0.5, bc=(1, 0, 1, 1, 0, 1),
                         n_gt=1, name=f"lat2_g{G}")


@pytest.mark.parametrize("prec,rtol,ktol,ftol", [(MOC_FP64, 1e-11, 1e-11, 1e-10),
                                                 (MOC_FP32, 2e-5, 1e-5, 1e-4)])
@pytest.mark.parametrize("G", [1, 12, 40])
def test_group_counts_against_oracle(G, prec, rtol, ktol, ftol):
    """One group, and more groups than the usual lane shape holds (12: eight
    lanes per track in FP32; 40: two chunks of 32 groups): two sweeps from a
    seeded source, then power iterations, like the oracle."""
    p = _lat2(G)
    o = oracle.Oracle(p, n_threads=NTH)
    tr = Tracks(Geometry(p), track_params(p, precision=prec))
    Q = np.random.default_rng(G).uniform(0.2, 1.0, size=(o.n_fsr, G))
    o.reset()
    for sweep in range(2):
        ot, ol = o.sweep_once(Q)
        gt, gl = tr.sweep_from_source(Q)
        scale = np.abs(ot).max()
        assert np.abs(gt - ot).max() <= rtol * scale, (sweep, np.abs(gt - ot).max() / scale)
        assert abs(gl - ol) <= rtol * max(abs(ol), 1e-300) + 1e-300
    o.reset()
    tr.reset()
    n = 10
    ref = o.iterate(n)
    res = tr.iterate(n, use_graph=True)
    phi, k = tr.flux()
    assert res["iterations"] == n
    assert abs(k - ref["k"]) < ktol, (k, ref["k"])
    np.testing.assert_allclose(phi, o.flux(), rtol=ftol)
    tr.close()


@pytest.mark.parametrize("prec,rtol,ktol,ftol", [(MOC_FP64, 1e-11, 1e-11, 1e-10),
                                                 (MOC_FP32, 2e-5, 1e-5, 1e-4)])
def test_all_vacuum_against_oracle(prec, rtol, ktol, ftol):
    """Vacuum on all six faces (no boundary flux is stored or read: the
    fixed-point bound comes from the source alone): sweeps and power
    iterations like the oracle, and every track leaks."""
    p = _lat3(bc=(0, 0, 0, 0, 0, 0), seed=9)
    o = oracle.Oracle(p, n_threads=NTH)
    tr = Tracks(Geometry(p), track_params(p, precision=prec))
    Q = np.random.default_rng(9).uniform(0.2, 1.0, size=(o.n_fsr, p.num_groups))
    o.reset()
    for sweep in range(2):
        ot, ol = o.sweep_once(Q)
        gt, gl = tr.sweep_from_source(Q)
        scale = np.abs(ot).max()
        assert np.abs(gt - ot).max() <= rtol * scale, (sweep, np.abs(gt - ot).max() / scale)
        assert ol > 0.0 and abs(gl - ol) <= rtol * abs(ol)
    # an empty range of 2D tracks sweeps nothing
    et, el = tr.sweep_units_from_source(Q, 3, 3)
    assert not et.any() and el == 0.0
    o.reset()
    tr.reset()
    ref = o.iterate(12)
    res = tr.iterate(12, use_graph=True)
    phi, k = tr.flux()
    assert abs(k - ref["k"]) < ktol, (k, ref["k"])
    np.testing.assert_allclose(phi, o.flux(), rtol=ftol)
    tr.close()


# ------------------------------------------- optically thin regions

def _lat3_thin(factor):
    """lat3 with its moderator (material 1) made optically thin: Sigma_t and
    the scattering matrix scaled by `factor` (the scattering ratio kept), so
    that the moderator's segments have tau = Sigma_t l of 1e-4 to 1e-3 (the
    void-like reflector cells of the large configurations)."""
    p = _lat3(bc=(1, 0, 1, 1, 0, 1), seed=9)
    st, ss = p.sigma_t.copy(), p.sigma_s.copy()
    st[1] *= factor
    ss[1] *= factor
    return p.with_tracks(sigma_t=st, sigma_s=ss, name=f"lat3_thin{factor:g}")


@pytest.mark.parametrize("prec,factor,srel,frel,ktol", [(MOC_FP32, 1e-2, 1e-2, 1e-4, 1e-5),
                                                         (MOC_FP32, 1e-3, None, 1e-4, 1e-5),
                                                         (MOC_FP64, 1e-2, 1e-9, 1e-9, 1e-11),
                                                         (MOC_FP64, 1e-3, 1e-9, 1e-9, 1e-11)])
def test_optically_thin_regions(prec, factor, srel, frel, ktol):
    """A bound on optically thin regions (the moderator of this lattice with
    Sigma_t and scattering scaled by 1e-2 or 1e-3: tau = Sigma_t l about
    1e-3 to 1e-2, or 1e-4 to 1e-3).

    A sweep from a uniform source Q in every FSR is the hard case: Eq. 4's
    flux (4 pi Q + tally / V) / Sigma_t cancels two nearly equal terms where
    tau is small (the tally is about -4 pi Q V; their difference is of
    relative size tau / 2), so the FP32 sweep's relative error (the escape
    fraction's absolute error near 2^-24, the fixed-point grid of the unit's
    largest |W Qr|) is amplified by about 2 / tau: 2.4e-3 at 1e-2 (bound
    1e-2 here), 18% at 1e-3.  In a power iteration the source of a thin
    region is its own scattering and fission, proportional to the scaled
    cross sections, so Qr = Q / Sigma_t stays of the order of the flux and
    nothing cancels: 15 FP32 iterations meet the 1e-5 / 1e-4 bars at both
    scales.  FP64 meets 1e-9 everywhere."""
    p = _lat3_thin(factor)
    o = oracle.Oracle(p, n_threads=NTH)
    g = Geometry(p)
    tr = Tracks(g, track_params(p, precision=prec))
    Q = np.random.default_rng(17).uniform(0.2, 1.0, size=(o.n_fsr, p.num_groups))
    sigt = p.sigma_t[o.fsr_materials()]
    o.reset()
    ot, _ = o.sweep_once(Q)
    gt, _ = tr.sweep_from_source(Q)
    V = np.asarray(o.volumes())[:, None]
    r_sweep = float(np.abs((4 * np.pi * Q + gt / V) / (4 * np.pi * Q + ot / V) - 1).max())
    print(f"thin {factor:g} precision {prec}: uniform-source sweep flux max relative error {r_sweep:.3g}")
    if srel is not None:
        check_flux(gt, ot, Q, o.volumes(), sigt, rel=srel, what=f"thin {factor:g} precision {prec}")
    o.reset()
    tr.reset()
    ref = o.iterate(15)
    tr.iterate(15)
    phi, k = tr.flux()
    r = float(np.abs(phi / o.flux() - 1).max())
    print(f"thin {factor:g} precision {prec}: k error {abs(k - ref['k']):.3g}, flux max relative error {r:.3g}")
    assert abs(k - ref["k"]) < ktol
    assert r <= frel
    tr.close()
