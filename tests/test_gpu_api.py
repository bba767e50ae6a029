"""Entry points around the solve, through the C ABI on the GPU:

* moc_get_flux_device: the flux where it lives on the device, viewed by
  PyTorch without a copy, equals moc_get_flux (which copies to the host);
* a solve that reaches max_iter before its stopping rule holds returns
  MOC_ERR_NOT_CONVERGED with its last k, which is the oracle's k after the
  same number of iterations (eigenvalue and fixed-source problems).
"""
import numpy as np
import pytest

import oracle
import synth
from paper_2503_17743_gb300 import MOC_FP32, MOC_FP64, Geometry, MocError, Tracks, track_params
from paper_2503_17743_gb300 import _moc

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", [MOC_FP32, MOC_FP64])
def test_flux_device_pointer_is_the_flux(prec):
    torch = pytest.importorskip("torch")
    p = synth.workload("lattice5")
    tr = Tracks(Geometry(p), track_params(p, precision=prec))
    tr.iterate(6)
    phi_dev, scale_dev = tr.flux_device()
    assert phi_dev.shape == (tr.n_fsr, tr.G) and scale_dev.shape == (1,)
    t_phi = torch.as_tensor(phi_dev, device="cuda")
    t_scale = torch.as_tensor(scale_dev, device="cuda")
    assert t_phi.dtype == torch.float64 and t_phi.data_ptr() == phi_dev.ptr
    host, _ = tr.flux()
    # the same FP64 product as the host copy: bit for bit
    np.testing.assert_array_equal((t_phi * t_scale).cpu().numpy(), host)
    # the view follows the iterations (same memory, new values)
    tr.iterate(2)
    host2, _ = tr.flux()
    assert not np.array_equal(host2, host)
    np.testing.assert_array_equal((t_phi * t_scale).cpu().numpy(), host2)
    assert tr.flux_device()[0].ptr == phi_dev.ptr
    tr.close()


def test_flux_device_rejects_null():
    lib = _moc.load()
    import ctypes as C
    p = C.c_void_p()
    assert lib.moc_get_flux_device(None, C.byref(p), None, None, None) == _moc.MOC_ERR_INVALID_ARG


@pytest.mark.parametrize("name", ["pin_cell", "lattice5"])
def test_solve_eigen_not_converged_returns_last_k(name):
    p = synth.workload(name)
    o = oracle.Oracle(p, n_threads=4)
    o.reset()
    ref = o.iterate(3)
    tr = Tracks(Geometry(p), track_params(p, precision=MOC_FP64))
    with pytest.raises(MocError) as e:
        tr.solve_eigen(tol_k=1e-12, tol_src=1e-12, max_iter=3)
    assert e.value.code == _moc.MOC_ERR_NOT_CONVERGED
    r = tr.solve_eigen(tol_k=1e-12, tol_src=1e-12, max_iter=3, check=False)
    assert r["iterations"] == 3 and not r["converged"]
    assert abs(r["k"] - ref["k"]) < 1e-11, (r["k"], ref["k"])
    tr.close()


def test_solve_fixed_source_not_converged():
    p = synth.lattice(4, n=3, G=3, height=4.0, n_layers=2, n_azim=8, n_polar=4,
                      radial_spacing=0.2, axial_spacing=0.5, fixed_source=True)
    tr = Tracks(Geometry(p), track_params(p))
    with pytest.raises(MocError) as e:
        tr.solve_fixed_source(tol_src=1e-12, max_iter=2)
    assert e.value.code == _moc.MOC_ERR_NOT_CONVERGED
    r = tr.solve_fixed_source(tol_src=1e-12, max_iter=2, check=False)
    assert r["iterations"] == 2 and not r["converged"] and r["k"] == 1.0
    tr.close()


def test_negative_or_nonfinite_inputs_are_refused():
    """Sources, fluxes and boundary fluxes handed to the library must be
    finite and non-negative (physical values; the FP32 tally's fixed-point
    bound relies on it): each entry point that takes them refuses others."""
    p = synth.workload("lattice5")
    tr = Tracks(Geometry(p), track_params(p))
    n, G = tr.n_fsr, tr.G
    bad_q = np.full((n, G), 0.5)
    bad_q[3, 1] = -1e-3
    for call in (lambda: tr.sweep_from_source(bad_q), lambda: tr.sweep_units_from_source(bad_q, 0, 4)):
        with pytest.raises(MocError) as e:
            call()
        assert e.value.code == _moc.MOC_ERR_INVALID_ARG
    nan_q = np.full((n, G), 0.5)
    nan_q[0, 0] = np.nan
    with pytest.raises(MocError):
        tr.sweep_from_source(nan_q)
    phi = np.ones((n, G))
    phi[5, 0] = -1.0
    with pytest.raises(MocError):
        tr.set_flux(phi, 1.0)
    with pytest.raises(MocError):
        tr.set_flux(np.ones((n, G)), 0.0)
    with pytest.raises(MocError):
        tr.psi(0, 0, tr_first_index(tr), 0, value=-np.ones(G))
    # the valid forms still work
    tr.set_flux(np.ones((n, G)), 1.0)
    tr.sweep_from_source(np.full((n, G), 0.5))
    tr.close()


def tr_first_index(tr):
    """Lattice index of the first track of stack (0, 0)."""
    ti, _, _, _ = tr.stack_segments(0, 0)
    return int(ti[0])
