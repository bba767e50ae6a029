"""The allocation-free entry point moc_group_rates_static against the
existing entry points (moc_iterate / moc_read_result totals, moc_get_flux and
moc_get_volumes for the per-group values), two calls in a row.

This file is named to be collected last, so that it runs both alone and after
every other GPU test in the same process (the scratch address is resolved on
the first call and reused).
"""
import numpy as np
import pytest

import synth
from paper_2503_17743_gb300 import Geometry, Tracks, track_params
from tests import bruteforce as bf

pytestmark = pytest.mark.gpu


def _expected(p, fsr_mat, vol, phi):
    sig_a = p.sigma_t - p.sigma_s.sum(axis=2)                 # [M, G]
    prod = (vol[:, None] * p.nu_sigma_f[fsr_mat] * phi).sum(axis=0)
    absn = (vol[:, None] * sig_a[fsr_mat] * phi).sum(axis=0)
    return prod, absn


@pytest.mark.parametrize("fixed", [False, True])
def test_group_rates_static_two_calls_in_a_row(fixed):
    if fixed:
        p = synth.lattice(8, n=3, G=4, height=4.0, n_layers=2, n_azim=8, n_polar=4,
                          radial_spacing=0.2, axial_spacing=0.5, fixed_source=True)
    else:
        p = synth.workload("lattice5")
    # the FSR -> material map from the problem's documented numbering
    fsr_mat = bf.fsr_materials(p)
    tr = Tracks(Geometry(p), track_params(p))
    vol = tr.volumes()
    for _ in range(2):
        res = tr.iterate(4)
        phi, _ = tr.flux()
        ep, ea = _expected(p, fsr_mat, vol, phi)
        first = tr.group_rates_static()
        second = tr.group_rates_static()
        for prod, absn in (first, second):
            np.testing.assert_allclose(prod, ep, rtol=1e-12, atol=1e-300)
            np.testing.assert_allclose(absn, ea, rtol=1e-12, atol=1e-300)
            assert abs(prod.sum() - res["production"]) <= 1e-12 * max(1.0, abs(res["production"]))
            assert abs(absn.sum() - res["absorption"]) <= 1e-12 * max(1.0, abs(res["absorption"]))
        # fixed block order in the final pass: the two calls agree bit for bit
        np.testing.assert_array_equal(first[0], second[0])
        np.testing.assert_array_equal(first[1], second[1])
    tr.close()


def test_group_rates_static_rejects_too_many_groups():
    p = synth.pin_cell(3, G=33, homogeneous=True, n_layers=1, height=0.5)
    tr = Tracks(Geometry(p), track_params(p))
    with pytest.raises(RuntimeError, match="at most 32 energy groups"):
        tr.group_rates_static()
    tr.close()
