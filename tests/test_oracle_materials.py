"""Pins of the oracle's FSR -> material map (the cross sections every FSR
sweeps with, Eq. 3), against things other than the oracle's own map:

* direct point location: at random points (x, y, z) the material the problem
  puts there (the cell's mat_in inside its fuel circle, mat_out elsewhere,
  per layer) equals the material of the FSR whose number the brute-force
  point classifier gives (region by region, FSR = region * n_layers + layer);
* the same map rebuilt from the documented numbering alone;
* analytic volumes per material and layer: the tracked volume of every
  material in every layer equals pi r^2 h per pin (mat_in) and the rest of
  the cell (mat_out), within the tracking error of the layout.

A swap of mat_in and mat_out, a ring inside the fuel circle given the
moderator, or the top-of-core absorber placed in the wrong layers fails each.
"""
import math

import numpy as np
import pytest

import synth
from tests import bruteforce as bf


def _reduced_assemblies():
    """One 17x17 assembly with the moderator reflector on two sides and an
    absorber in the top quarter of a seeded half of its guide tubes (the
    3x3-assembly workload's structure at a size the oracle builds quickly)."""
    return synth.assemblies(seed=2, n_asm=1, height=8.0, n_layers=4, absorber_height=2.0,
                            n_azim=8, n_polar=4, radial_spacing=0.1, axial_spacing=0.5)


CASES = {
    "pin_cell": lambda: synth.workload("pin_cell"),
    "lattice5_rings": lambda: synth.workload("lattice5_rings"),
    "lattice5_axial": lambda: synth.workload("lattice5_axial"),
    "asm1_absorber": _reduced_assemblies,
}


@pytest.fixture(scope="module", params=sorted(CASES))
def case(request, oracle_mod):
    p = CASES[request.param]()
    return p, oracle_mod.Oracle(p, n_threads=4)


def test_reduced_assembly_has_absorber_in_top_layers_only():
    p = _reduced_assemblies()
    mi = np.asarray(p.mat_in).reshape(-1, p.n_layers)
    has_abs = (mi == synth.MAT_ABS)
    assert has_abs.any()
    # absorber_height 2 cm of 8 cm in 4 layers: the top layer only
    assert not has_abs[:, :-1].any() and has_abs[:, -1].any()


def test_fsr_material_at_random_points(case):
    p, o = case
    fm = o.fsr_materials()
    rng = np.random.default_rng(5)
    n = 40000
    x = rng.uniform(0, p.ncx * p.pitch, n)
    y = rng.uniform(0, p.ncy * p.pitch, n)
    z = rng.uniform(0, p.height, n)
    fsr = bf.region_ids(p, x, y) * p.n_layers + bf.layer_of(p, z)
    np.testing.assert_array_equal(fm[fsr], bf.point_material(p, x, y, z))


def test_fsr_materials_match_documented_numbering(case):
    p, o = case
    np.testing.assert_array_equal(o.fsr_materials(), bf.fsr_materials(p))


def test_volume_per_material_and_layer_matches_analytic(case):
    p, o = case
    fm = o.fsr_materials()
    V = o.volumes()
    NL = p.n_layers
    h = np.diff(p.layer_z) if p.layer_z is not None else np.full(NL, p.height / NL)
    layer = np.arange(o.n_fsr) % NL
    circle = math.pi * p.fuel_radius ** 2
    cell = p.pitch ** 2
    mi = np.asarray(p.mat_in).reshape(-1, NL)
    mo = np.asarray(p.mat_out).reshape(-1, NL)
    pin = np.asarray(p.has_pin) != 0
    for m in range(p.num_materials):
        for L in range(NL):
            expect = (np.sum(pin & (mi[:, L] == m)) * circle
                      + np.sum(pin & (mo[:, L] == m)) * (cell - circle)
                      + np.sum(~pin & (mo[:, L] == m)) * cell) * h[L]
            got = V[(fm == m) & (layer == L)].sum()
            # chord sums of the layout: within 1% of the analytic volume
            assert abs(got - expect) <= 0.01 * max(expect, circle * h[L]), (m, L, got, expect)
