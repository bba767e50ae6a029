"""ctypes binding of the C ABI declared in ``include/moc.h``.

Argument marshalling only: every step of the solve runs inside
``libmoc3d.so`` (host tracking in C++, everything else in CUDA kernels).
There is no fallback: if the library is missing or fails to load, every call
raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmoc3d.so")

MOC_OK = 0
MOC_ERR_INVALID_ARG = 1
MOC_ERR_OUT_OF_MEMORY = 2
MOC_ERR_CUDA = 3
MOC_ERR_NOT_CONVERGED = 4
MOC_ERR_TIMEOUT = 5
MOC_ERR_UNSUPPORTED = 6
MOC_FP32 = 0
MOC_FP64 = 1
MOC_SCHED_UNITS_NATURAL = 1
MOC_SCHED_TRACKS_NATURAL = 2
MOC_SCHED_ROWS_WITH_SIGMA = 4
MOC_TALLY_AUTO = 0
MOC_TALLY_SHARED = 1
MOC_TALLY_GLOBAL = 2

i32p = C.POINTER(C.c_int32)
i64p = C.POINTER(C.c_int64)
f32p = C.POINTER(C.c_float)
f64p = C.POINTER(C.c_double)


class moc_geometry_desc(C.Structure):
    _fields_ = [("ncx", C.c_int32), ("ncy", C.c_int32), ("pitch", C.c_double),
                ("fuel_radius", C.c_double), ("height", C.c_double), ("n_layers", C.c_int32),
                ("has_pin", i32p), ("mat_in", i32p), ("mat_out", i32p), ("bc", C.c_int32 * 6),
                ("fuel_rings", C.c_int32), ("moderator_rings", C.c_int32), ("sectors", C.c_int32),
                ("layer_z", f64p)]


class moc_materials(C.Structure):
    _fields_ = [("num_materials", C.c_int32), ("num_groups", C.c_int32),
                ("sigma_t", f64p), ("sigma_s", f64p), ("nu_sigma_f", f64p), ("chi", f64p),
                ("ext_source", f64p)]


class moc_track_params(C.Structure):
    _fields_ = [("n_azim", C.c_int32), ("n_polar", C.c_int32), ("radial_spacing", C.c_double),
                ("axial_spacing", C.c_double), ("precision", C.c_int32),
                ("preload_budget_bytes", C.c_int64), ("tally_mode", C.c_int32),
                ("block_threads", C.c_int32), ("blocks_per_sm", C.c_int32), ("device", C.c_int32),
                ("groups_per_lane", C.c_int32), ("schedule", C.c_int32),
                ("chunk_segments", C.c_int32), ("trace_on_device", C.c_int32),
                ("sync_block", C.c_int32)]


class moc_server_params(C.Structure):
    _fields_ = [("device", C.c_int32), ("max_active", C.c_int32),
                ("memory_budget_bytes", C.c_int64), ("iterations_per_poll", C.c_int32)]


class moc_solve_params(C.Structure):
    _fields_ = [("tol_k", C.c_double), ("tol_src", C.c_double), ("max_iter", C.c_int32),
                ("use_graph", C.c_int32)]


class moc_result(C.Structure):
    _fields_ = [("k", C.c_double), ("residual", C.c_double), ("dk", C.c_double),
                ("production", C.c_double), ("absorption", C.c_double), ("leakage", C.c_double),
                ("seconds", C.c_double), ("integrations", C.c_double), ("iterations", C.c_int32),
                ("converged", C.c_int32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


# name -> (restype, argtypes); every symbol include/moc.h declares
SIGNATURES = {
    "moc_last_error": (C.c_char_p, []),
    "moc_create_geometry": (C.c_int, [C.POINTER(moc_geometry_desc), C.POINTER(moc_materials),
                                      C.POINTER(C.c_void_p)]),
    "moc_destroy_geometry": (None, [C.c_void_p]),
    "moc_query_footprint": (C.c_int, [C.c_void_p, C.POINTER(moc_track_params), i64p, i64p]),
    "moc_generate_tracks": (C.c_int, [C.c_void_p, C.POINTER(moc_track_params),
                                      C.POINTER(C.c_void_p)]),
    "moc_destroy_tracks": (None, [C.c_void_p]),
    "moc_state_create": (C.c_int, [C.c_void_p, f64p, C.POINTER(C.c_void_p)]),
    "moc_get_segments2d": (C.c_int, [C.c_void_p, C.c_int32, C.c_int64, i32p, f64p, f64p, i64p]),
    "moc_state_destroy": (None, [C.c_void_p]),
    "moc_batch_step": (C.c_int, [C.POINTER(C.c_void_p), C.c_int32, C.c_void_p]),
    "moc_sweep": (C.c_int, [C.c_void_p, C.c_void_p]),
    "moc_update_source": (C.c_int, [C.c_void_p, C.c_double, C.c_void_p]),
    "moc_solve_eigen": (C.c_int, [C.c_void_p, C.POINTER(moc_solve_params), C.POINTER(moc_result)]),
    "moc_solve_fixed_source": (C.c_int, [C.c_void_p, C.POINTER(moc_solve_params),
                                         C.POINTER(moc_result)]),
    "moc_reset": (C.c_int, [C.c_void_p]),
    "moc_iterate": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.POINTER(moc_result)]),
    "moc_get_flux": (C.c_int, [C.c_void_p, f64p, f64p]),
    "moc_get_flux_device": (C.c_int, [C.c_void_p, C.POINTER(C.c_void_p), C.POINTER(C.c_void_p),
                                      i64p, i32p]),
    "moc_set_flux": (C.c_int, [C.c_void_p, f64p, C.c_double]),
    "moc_get_volumes": (C.c_int, [C.c_void_p, f64p]),
    "moc_tracks_info": (C.c_int, [C.c_void_p, i64p, C.c_int32]),
    "moc_get_stack_segments": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_int64, C.c_int64,
                                         i64p, i32p, i32p, f64p, i64p, i64p]),
    "moc_track_psi": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_int64, C.c_int32, f64p,
                                C.c_int32]),
    "moc_sweep_from_source": (C.c_int, [C.c_void_p, f64p, f64p, f64p]),
    "moc_sweep_units_from_source": (C.c_int, [C.c_void_p, f64p, C.c_int32, C.c_int32, f64p, f64p]),
    "moc_group_rates_static": (C.c_int, [C.c_void_p, C.c_void_p, f64p]),
    "moc_measure_ex2_rate": (C.c_int, [C.c_int32, f64p, f64p]),
    "moc_measure_unit_rates": (C.c_int, [C.c_int32, f64p, C.c_int32]),
    "moc_eval_attenuation_f64": (C.c_int, [C.c_int32, f64p, C.c_int64, f64p, f64p]),
    "moc_eval_attenuation_f32": (C.c_int, [C.c_int32, f32p, C.c_int64, f32p]),
    "moc_autotune": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p, f64p, C.c_int32,
                               f64p, i32p]),
    "moc_server_create": (C.c_int, [C.c_void_p, C.c_void_p]),
    "moc_server_destroy": (None, [C.c_void_p]),
    "moc_server_submit": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, i64p]),
    "moc_server_step": (C.c_int, [C.c_void_p, i32p, i32p]),
    "moc_server_result": (C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, f64p, C.c_int64, f64p, i32p]),
    "moc_server_stats": (C.c_int, [C.c_void_p, i64p, C.c_int32]),
    "moc_enqueue_source": (C.c_int, [C.c_void_p, C.c_void_p]),
    "moc_enqueue_sweep": (C.c_int, [C.c_void_p, C.c_void_p]),
    "moc_enqueue_update": (C.c_int, [C.c_void_p, C.c_void_p]),
    "moc_read_result": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(moc_result)]),
}

_lib = None


class MocError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"moc error {code}: {msg}")
        self.code = code


def load(path: str = LIB_PATH):
    """Load libmoc3d.so (raises if it is missing: there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build it with __graft_entry__.build()")
        lib = C.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
    return _lib


def _check(rc):
    if rc != MOC_OK:
        raise MocError(rc, load().moc_last_error().decode())
    return rc


def _ptr(a, t):
    return a.ctypes.data_as(t)


class Geometry:
    """moc_create_geometry over a ``synth.Problem``-like object."""

    def __init__(self, prob):
        lib = load()
        self._keep = []

        def arr(a, dt):
            a = np.ascontiguousarray(a, dtype=dt)
            self._keep.append(a)
            return a

        d = moc_geometry_desc()
        d.ncx, d.ncy, d.pitch = prob.ncx, prob.ncy, prob.pitch
        d.fuel_radius, d.height, d.n_layers = prob.fuel_radius, prob.height, prob.n_layers
        d.has_pin = _ptr(arr(prob.has_pin, np.int32), i32p)
        d.mat_in = _ptr(arr(prob.mat_in, np.int32), i32p)
        d.mat_out = _ptr(arr(prob.mat_out, np.int32), i32p)
        for i in range(6):
            d.bc[i] = int(prob.bc[i])
        d.fuel_rings = int(getattr(prob, "fuel_rings", 1))
        d.moderator_rings = int(getattr(prob, "moderator_rings", 0))
        d.sectors = int(getattr(prob, "sectors", 1))
        lz = getattr(prob, "layer_z", None)
        d.layer_z = _ptr(arr(lz, np.float64), f64p) if lz is not None else f64p()
        m = moc_materials()
        m.num_materials, m.num_groups = prob.num_materials, prob.num_groups
        m.sigma_t = _ptr(arr(prob.sigma_t, np.float64), f64p)
        m.sigma_s = _ptr(arr(prob.sigma_s, np.float64), f64p)
        m.nu_sigma_f = _ptr(arr(prob.nu_sigma_f, np.float64), f64p)
        m.chi = _ptr(arr(prob.chi, np.float64), f64p)
        m.ext_source = (_ptr(arr(prob.ext_source, np.float64), f64p)
                        if prob.ext_source is not None else f64p())
        h = C.c_void_p()
        _check(lib.moc_create_geometry(C.byref(d), C.byref(m), C.byref(h)))
        self._h = h
        self._keep = []
        self.prob = prob

    def footprint(self, params):
        r, p = C.c_int64(), C.c_int64()
        _check(load().moc_query_footprint(self._h, C.byref(params), C.byref(r), C.byref(p)))
        return r.value, p.value

    def __del__(self):
        try:
            if self._h:
                load().moc_destroy_geometry(self._h)
        except Exception:
            pass


def track_params(prob, precision=MOC_FP32, preload_budget_bytes=-1, tally_mode=MOC_TALLY_AUTO,
                 block_threads=0, blocks_per_sm=0, device=0, groups_per_lane=0, schedule=0,
                 chunk_segments=0, trace_on_device=0, sync_block=0):
    p = moc_track_params()
    p.n_azim, p.n_polar = prob.n_azim, prob.n_polar
    p.radial_spacing, p.axial_spacing = prob.radial_spacing, prob.axial_spacing
    p.precision = precision
    p.preload_budget_bytes = preload_budget_bytes
    p.tally_mode = tally_mode
    p.block_threads = block_threads
    p.blocks_per_sm = blocks_per_sm
    p.device = device
    p.groups_per_lane = groups_per_lane
    p.schedule = schedule
    p.chunk_segments = chunk_segments
    p.trace_on_device = trace_on_device
    p.sync_block = sync_block
    return p


INFO_KEYS = ["n_fsr", "groups", "tracks2d", "stacks", "tracks3d", "segments3d",
             "integrations_per_sweep", "stored_segments", "preloaded_stacks", "device_bytes",
             "n_z", "cells_per_layer", "sweep_blocks", "sweep_threads", "tally_mode", "precision",
             "sweep_smem_bytes", "tile_entries", "lanes_per_track", "max_segments_per_track",
             "h2d_bytes", "groups_per_lane", "chunk_segments", "sync_block", "sweep_slots",
             "off_lattice", "tally_bits", "material_keys"]


class Tracks:
    """moc_generate_tracks + the solve entry points."""

    def __init__(self, geom: Geometry, params: moc_track_params, _handle=None, _owner=None):
        self.geom = geom
        self.params = params
        if _handle is None:
            h = C.c_void_p()
            _check(load().moc_generate_tracks(geom._h, C.byref(params), C.byref(h)))
        else:
            h = _handle
        self._h = h
        self._owner = _owner  # a state keeps its layout's Python object alive
        self.info = self._info()
        self.n_fsr = self.info["n_fsr"]
        self.G = self.info["groups"]

    def segments2d(self, t):
        """moc_get_segments2d: (regions, lengths, boundary positions) of 2D track t."""
        n = C.c_int64()
        lib = load()
        _check(lib.moc_get_segments2d(self._h, int(t), 0, i32p(), f64p(), f64p(), C.byref(n)))
        reg = np.zeros(n.value, dtype=np.int32)
        ln = np.zeros(n.value)
        pos = np.zeros(n.value + 1)
        _check(lib.moc_get_segments2d(self._h, int(t), n.value, _ptr(reg, i32p), _ptr(ln, f64p),
                                      _ptr(pos, f64p), C.byref(n)))
        return reg, ln, pos

    def state(self, ext_source=None):
        """moc_state_create: another solve on this layout (optionally with its
        own external source [M, G]); a Tracks object."""
        src = None
        if ext_source is not None:
            src = np.ascontiguousarray(ext_source, dtype=np.float64)
        h = C.c_void_p()
        _check(load().moc_state_create(self._h, _ptr(src, f64p) if src is not None else f64p(),
                                       C.byref(h)))
        t = Tracks(self.geom, self.params, _handle=h, _owner=self)
        t._src_keep = src
        return t

    def _info(self):
        out = np.zeros(len(INFO_KEYS), dtype=np.int64)
        _check(load().moc_tracks_info(self._h, _ptr(out, i64p), len(INFO_KEYS)))
        return dict(zip(INFO_KEYS, [int(x) for x in out]))

    def close(self):
        if getattr(self, "_h", None):
            load().moc_destroy_tracks(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def sweep(self, stream=None):
        _check(load().moc_sweep(self._h, stream))

    def update_source(self, k, stream=None):
        _check(load().moc_update_source(self._h, float(k), stream))

    def reset(self):
        _check(load().moc_reset(self._h))

    def enqueue_source(self, stream=None):
        _check(load().moc_enqueue_source(self._h, stream))

    def enqueue_sweep(self, stream=None):
        _check(load().moc_enqueue_sweep(self._h, stream))

    def enqueue_update(self, stream=None):
        _check(load().moc_enqueue_update(self._h, stream))

    def read_result(self, stream=None):
        r = moc_result()
        _check(load().moc_read_result(self._h, stream, C.byref(r)))
        return r.as_dict()

    def iterate(self, n, use_graph=True):
        r = moc_result()
        _check(load().moc_iterate(self._h, int(n), int(bool(use_graph)), C.byref(r)))
        return r.as_dict()

    def _solve(self, fn, tol_k, tol_src, max_iter, use_graph, check):
        sp = moc_solve_params()
        sp.tol_k, sp.tol_src, sp.max_iter, sp.use_graph = tol_k, tol_src, max_iter, int(use_graph)
        r = moc_result()
        rc = fn(self._h, C.byref(sp), C.byref(r))
        if check or rc not in (MOC_OK, MOC_ERR_NOT_CONVERGED):
            _check(rc)
        return r.as_dict()

    def solve_eigen(self, tol_k=1e-6, tol_src=1e-5, max_iter=5000, use_graph=True, check=True):
        return self._solve(load().moc_solve_eigen, tol_k, tol_src, max_iter, use_graph, check)

    def solve_fixed_source(self, tol_src=1e-5, max_iter=5000, use_graph=True, check=True):
        return self._solve(load().moc_solve_fixed_source, 0.0, tol_src, max_iter, use_graph, check)

    def flux(self):
        phi = np.zeros(self.n_fsr * self.G)
        k = C.c_double()
        _check(load().moc_get_flux(self._h, _ptr(phi, f64p), C.byref(k)))
        return phi.reshape(self.n_fsr, self.G), k.value

    def flux_device(self):
        """moc_get_flux_device: (phi, scale) as read-only device arrays that
        expose ``__cuda_array_interface__`` (``torch.as_tensor(phi,
        device="cuda")`` views them without a copy): phi [n_fsr, G] FP64, the
        flux iterate, and scale [1], its normalisation (the normalised flux
        is phi * scale).  The library owns the memory: the views are valid
        until this handle is closed and change with every iteration."""
        p, sc = C.c_void_p(), C.c_void_p()
        n, g = C.c_int64(), C.c_int32()
        _check(load().moc_get_flux_device(self._h, C.byref(p), C.byref(sc), C.byref(n), C.byref(g)))
        return (DeviceArray(p.value, (n.value, g.value), self),
                DeviceArray(sc.value, (1,), self))

    def set_flux(self, phi, k):
        phi = np.ascontiguousarray(phi, dtype=np.float64).ravel()
        _check(load().moc_set_flux(self._h, _ptr(phi, f64p), float(k)))

    def volumes(self):
        v = np.zeros(self.n_fsr)
        _check(load().moc_get_volumes(self._h, _ptr(v, f64p)))
        return v

    def stack_segments(self, t, p):
        nt, ns = C.c_int64(), C.c_int64()
        lib = load()
        rc = lib.moc_get_stack_segments(self._h, t, p, 0, 0, i64p(), i32p(), i32p(), f64p(),
                                        C.byref(nt), C.byref(ns))
        if rc not in (MOC_OK, MOC_ERR_INVALID_ARG):
            _check(rc)
        ti = np.zeros(max(nt.value, 1), dtype=np.int64)
        nseg = np.zeros(max(nt.value, 1), dtype=np.int32)
        fsr = np.zeros(max(ns.value, 1), dtype=np.int32)
        ln = np.zeros(max(ns.value, 1), dtype=np.float64)
        _check(lib.moc_get_stack_segments(self._h, t, p, nt.value, ns.value, _ptr(ti, i64p),
                                          _ptr(nseg, i32p), _ptr(fsr, i32p), _ptr(ln, f64p),
                                          C.byref(nt), C.byref(ns)))
        return ti[:nt.value], nseg[:nt.value], fsr[:ns.value], ln[:ns.value]

    def psi(self, t, p, i, sense, value=None):
        v = np.zeros(self.G) if value is None else np.ascontiguousarray(value, dtype=np.float64).copy()
        _check(load().moc_track_psi(self._h, t, p, int(i), sense, _ptr(v, f64p),
                                    0 if value is None else 1))
        return v

    def sweep_from_source(self, Q):
        Q = np.ascontiguousarray(Q, dtype=np.float64).ravel()
        tally = np.zeros(self.n_fsr * self.G)
        leak = C.c_double()
        _check(load().moc_sweep_from_source(self._h, _ptr(Q, f64p), _ptr(tally, f64p),
                                            C.byref(leak)))
        return tally.reshape(self.n_fsr, self.G), leak.value

    def sweep_units_from_source(self, Q, t0, t1):
        """Tally and leakage of one sweep of the 2D tracks [t0, t1) from source
        Q with zero incoming fluxes (the boundary fluxes are undefined after)."""
        Q = np.ascontiguousarray(Q, dtype=np.float64).ravel()
        tally = np.zeros(self.n_fsr * self.G)
        leak = C.c_double()
        _check(load().moc_sweep_units_from_source(self._h, _ptr(Q, f64p), int(t0), int(t1),
                                                  _ptr(tally, f64p), C.byref(leak)))
        return tally.reshape(self.n_fsr, self.G), leak.value

    def group_rates_static(self, stream=None):
        """(production[G], absorption[G]) of the normalised flux, computed by
        the library without allocating device memory."""
        out = np.zeros(2 * self.G)
        _check(load().moc_group_rates_static(self._h, stream, _ptr(out, f64p)))
        return out[:self.G].copy(), out[self.G:].copy()


class DeviceArray:
    """An FP64 device array owned by the library, described by
    ``__cuda_array_interface__`` (version 3) so that PyTorch or any other
    consumer can view it in place; keeps its owner handle alive.  The
    library's contract makes it read-only for the caller; the interface
    itself does not carry the flag (PyTorch refuses read-only arrays)."""

    def __init__(self, ptr, shape, owner):
        self.ptr = int(ptr)
        self.shape = tuple(int(s) for s in shape)
        self._owner = owner

    @property
    def __cuda_array_interface__(self):
        return {"shape": self.shape, "typestr": "<f8", "data": (self.ptr, False),
                "version": 3, "strides": None}


def batch_step(solves, stream=None):
    """moc_batch_step: one outer iteration of every solve (a Tracks and its
    states), their sweeps in one persistent launch."""
    arr = (C.c_void_p * len(solves))(*[t._h for t in solves])
    _check(load().moc_batch_step(arr, len(solves), stream))


def measure_ex2_rate(device=0):
    """(exponentials per second of the whole device, SM count): throughput of
    the ex2 unit that bounds the sweep (one exponential per integration)."""
    rate, sms = C.c_double(), C.c_double()
    _check(load().moc_measure_ex2_rate(device, C.byref(rate), C.byref(sms)))
    return rate.value, int(sms.value)


UNIT_RATES = ["sm_count", "sm_mhz", "fp32_fma_scalar_per_s", "fp32_fma_packed_lane_ops_per_s",
              "smem_red_s32_per_s", "smem_load_bytes_per_s", "f2i_per_s"]


def measure_unit_rates(device=0):
    """Measured throughput of the units the FP32 sweep issues to (dict, see
    moc_measure_unit_rates): SM count and clock, FP32 FMA lane operations per
    second scalar and as packed pairs, conflict-free shared-memory integer
    reductions and load bytes per second, float-to-integer conversions per
    second."""
    out = np.zeros(len(UNIT_RATES))
    _check(load().moc_measure_unit_rates(device, _ptr(out, f64p), len(UNIT_RATES)))
    d = dict(zip(UNIT_RATES, out.tolist()))
    d["sm_count"] = int(d["sm_count"])
    return d


def eval_attenuation_f64(x, device=0):
    """(the FP64 sweep's e^{-x}, CUDA's exp(-x)) for a float64 array x,
    both evaluated on the device."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    y, y_lib = np.empty_like(x), np.empty_like(x)
    _check(load().moc_eval_attenuation_f64(device, _ptr(x, f64p), x.size, _ptr(y, f64p), _ptr(y_lib, f64p)))
    return y, y_lib


def eval_attenuation_f32(b, device=0):
    """The FP32 sweep's e^{-tau} = 2^{-b} for a float32 array b = tau log2 e,
    evaluated on the device."""
    b = np.ascontiguousarray(b, dtype=np.float32)
    e = np.empty_like(b)
    _check(load().moc_eval_attenuation_f32(device, _ptr(b, f32p), b.size, _ptr(e, f32p)))
    return e


SERVER_STATS = ["queued", "resident", "admitted", "retired", "bytes_resident", "budget",
                "max_resident"]


class Server:
    """moc_server_*: solves of different problems resident on one device and
    advanced together as they arrive (continuous batching)."""

    def __init__(self, device=0, max_active=0, memory_budget_bytes=0, iterations_per_poll=0):
        p = moc_server_params()
        p.device, p.max_active = device, max_active
        p.memory_budget_bytes, p.iterations_per_poll = memory_budget_bytes, iterations_per_poll
        h = C.c_void_p()
        _check(load().moc_server_create(C.byref(p), C.byref(h)))
        self._h = h
        self._shape = {}

    def submit(self, geom, params, tol_k=1e-6, tol_src=1e-5, max_iter=5000):
        """Queue a solve of `geom` (a Geometry) with track parameters `params`;
        returns the ticket."""
        sp = moc_solve_params()
        sp.tol_k, sp.tol_src, sp.max_iter, sp.use_graph = tol_k, tol_src, max_iter, 1
        t = C.c_int64()
        _check(load().moc_server_submit(self._h, geom._h, C.byref(params), C.byref(sp), C.byref(t)))
        prob = geom.prob
        # every FSR of the geometry: rings and sectors of the pin cells included
        self._shape[t.value] = (int(prob.n_fsr), prob.num_groups)
        return t.value

    def step(self):
        """One engine step; returns (solves retired by it, requests left)."""
        f, p = C.c_int32(), C.c_int32()
        _check(load().moc_server_step(self._h, C.byref(f), C.byref(p)))
        return f.value, p.value

    def result(self, ticket, check=True):
        """None while pending, else (result dict, phi [n_fsr, G], seconds
        queued, seconds from submission to retirement, status)."""
        n_fsr, G = self._shape[ticket]
        r = moc_result()
        phi = np.zeros(n_fsr * G)
        times = np.zeros(2)
        ready = C.c_int32()
        rc = load().moc_server_result(self._h, C.c_int64(ticket), C.byref(r), _ptr(phi, f64p),
                                      phi.size, _ptr(times, f64p), C.byref(ready))
        if not ready.value:
            _check(rc)
            return None
        del self._shape[ticket]
        if check:
            _check(rc)
        return r.as_dict(), phi.reshape(n_fsr, G), float(times[0]), float(times[1]), rc

    def stats(self):
        out = np.zeros(len(SERVER_STATS), dtype=np.int64)
        _check(load().moc_server_stats(self._h, _ptr(out, i64p), len(SERVER_STATS)))
        return dict(zip(SERVER_STATS, (int(v) for v in out)))

    def close(self):
        if self._h:
            load().moc_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def autotune(geom, params, iterations=5):
    """moc_autotune: (best track parameters, seconds per iteration, table of
    the candidates [groups per lane, tally mode, preload budget, stored
    pieces, seconds per iteration, tracks per synchronous block])."""
    best = moc_track_params()
    sec = C.c_double()
    rep = np.zeros((64, 6))
    n = C.c_int32()
    _check(load().moc_autotune(geom._h, C.byref(params), int(iterations), C.byref(best),
                               C.byref(sec), 64, _ptr(rep, f64p), C.byref(n)))
    return best, sec.value, rep[:n.value].copy()
