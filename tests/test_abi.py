"""CPU checks of the C ABI: the library loads, exports every symbol the
header declares, and its host-only entry points validate their inputs."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import synth
from paper_2503_17743_gb300 import _moc
from paper_2503_17743_gb300 import build as libbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    txt = open(os.path.join(ROOT, "include", "moc.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(moc_[a-z0-9_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    libbuild.build()
    return _moc.load()


def test_library_exports_every_header_symbol(lib):
    names = header_functions()
    assert len(names) >= 18
    for n in names:
        assert hasattr(lib, n), n
        assert n in _moc.SIGNATURES, n


def test_build_targets_sm103a_only():
    assert libbuild.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_geometry_validation_rejects_bad_inputs(lib):
    p = synth.pin_cell(1)
    g = _moc.Geometry(p)
    assert g._h
    bad = p.with_tracks(sigma_t=-p.sigma_t)
    with pytest.raises(_moc.MocError) as e:
        _moc.Geometry(bad)
    assert e.value.code == _moc.MOC_ERR_INVALID_ARG
    nan = p.sigma_t.copy()
    nan[0, 0] = np.nan
    with pytest.raises(_moc.MocError):
        _moc.Geometry(p.with_tracks(sigma_t=nan))
    ss = p.sigma_s.copy()
    ss[0, 0, :] = p.sigma_t[0, 0]  # row sum above sigma_t
    with pytest.raises(_moc.MocError):
        _moc.Geometry(p.with_tracks(sigma_s=ss))
    mat = p.mat_in.copy()
    mat[0] = 99
    with pytest.raises(_moc.MocError):
        _moc.Geometry(p.with_tracks(mat_in=mat))
    with pytest.raises(_moc.MocError):
        _moc.Geometry(p.with_tracks(fuel_radius=0.7))


def test_footprint_host_only(lib):
    p = synth.workload("lattice17")
    g = _moc.Geometry(p)
    res, pre = g.footprint(_moc.track_params(p))
    # 2 x 4 variants x G x 4 B per stored track dominate: ~ 2.3e6/2 tracks
    assert 50e6 < res < 2e9
    # stored segments: 9.0e8 integrations / (2 senses x 7 groups) / 2 frames x 8 B ~ 0.26 GB
    assert 1e8 < pre < 2e9


def test_axial_mesh_off_the_lattice_host(lib):
    """Equal layers that are not whole axial spacings are planes off the
    lattice: the layout is built (host query) and stores no segments."""
    p = synth.pin_cell(1, axial_spacing=0.3)  # 0.5 cm layers are not whole spacings
    g = _moc.Geometry(p)
    res, pre = g.footprint(_moc.track_params(p))
    assert res > 0 and pre == 0


def test_bad_track_params(lib):
    p = synth.pin_cell(1)
    g = _moc.Geometry(p)
    with pytest.raises(_moc.MocError):
        g.footprint(_moc.track_params(p.with_tracks(n_azim=6)))
    with pytest.raises(_moc.MocError):
        g.footprint(_moc.track_params(p.with_tracks(n_polar=3)))


def test_unequal_layers_host_checks(lib):
    """Layer planes: rising from 0 to the height (geometry); on or off the
    axial lattice (layout); the footprint query runs the layout on the host."""
    p = synth.pin_cell(1, n_layers=3)
    ok = p.with_tracks(layer_z=np.array([0.0, 0.5, 1.5, 2.0]))
    g = _moc.Geometry(ok)
    res, _ = g.footprint(_moc.track_params(ok))
    assert res > 0
    with pytest.raises(_moc.MocError) as e:
        _moc.Geometry(p.with_tracks(layer_z=np.array([0.0, 1.5, 0.5, 2.0])))
    assert e.value.code == _moc.MOC_ERR_INVALID_ARG
    with pytest.raises(_moc.MocError):
        _moc.Geometry(p.with_tracks(layer_z=np.array([0.0, 0.5, 1.5, 2.5])))  # not the height
    off = p.with_tracks(layer_z=np.array([0.0, 0.6, 1.5, 2.0]))  # 0.6 is off the 0.5 cm lattice
    res, pre = _moc.Geometry(off).footprint(_moc.track_params(off))
    assert res > 0 and pre == 0  # planes off the lattice: nothing is stored


def test_ring_and_sector_counts_host(lib):
    """Rings and sectors multiply a pin cell's regions; out-of-range counts
    are rejected."""
    p = synth.workload("lattice5_rings")
    g = _moc.Geometry(p)
    assert g._h
    with pytest.raises(_moc.MocError):
        _moc.Geometry(p.with_tracks(sectors=65))
    with pytest.raises(_moc.MocError):
        _moc.Geometry(p.with_tracks(fuel_rings=-1))


def test_negative_chunk_segments_rejected(lib):
    p = synth.pin_cell(1)
    g = _moc.Geometry(p)
    with pytest.raises(_moc.MocError) as e:
        _moc.Tracks(g, _moc.track_params(p, chunk_segments=-1))
    assert e.value.code == _moc.MOC_ERR_INVALID_ARG  # checked before any device work
