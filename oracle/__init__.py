"""ctypes wrapper of the FP64 CPU oracle (``oracle/moc_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may use it; the GPU library never does.  It
follows the paper's Alg. 1 loop order and Eqs. 3-11 (see the C file header)
and shares nothing with the CUDA path except the seeded inputs of ``synth``.

Parity status of each oracle function (what pins it, see tests/test_oracle_*):

* 2D cyclic laydown, links, cycles ........ pinned (closed forms, bijection, brute force)
* 2D segments ............................. pinned (brute-force point classifier)
* z-stack index sets, Eqs. 6-11 ............ pinned (brute-force ray marching per track)
* tracked volumes ......................... pinned (analytic volumes, exact area sums)
* Eq. 3 sweep + Eq. 4 tally ............... pinned (pure absorber closed form, flat source)
* source iteration / k-eff ................ pinned (infinite medium k, fixed-source closed
                                              form, neutron balance)
* heterogeneous k and flux ................ parity unpinned beyond the above invariants
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "moc_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

i32p = C.POINTER(C.c_int32)
i64p = C.POINTER(C.c_int64)
f64p = C.POINTER(C.c_double)


class _Input(C.Structure):
    _fields_ = [
        ("ncx", C.c_int), ("ncy", C.c_int), ("n_layers", C.c_int),
        ("pitch", C.c_double), ("radius", C.c_double), ("height", C.c_double),
        ("has_pin", i32p), ("mat_in", i32p), ("mat_out", i32p),
        ("bc", C.c_int * 6),
        ("M", C.c_int), ("G", C.c_int),
        ("sigma_t", f64p), ("sigma_s", f64p), ("nu_sigma_f", f64p), ("chi", f64p),
        ("ext_source", f64p),
        ("n_azim", C.c_int), ("n_polar", C.c_int),
        ("radial_spacing", C.c_double), ("axial_spacing", C.c_double),
        ("n_threads", C.c_int),
        ("light", C.c_int),
        ("fuel_rings", C.c_int), ("mod_rings", C.c_int), ("sectors", C.c_int),
        ("layer_z", f64p),
    ]


def build(force: bool = False) -> str:
    """Compile the oracle (plain C, FP64, no fused multiply-add)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared", "-o", _LIB,
               _SRC, "-lm"]
        subprocess.run(cmd, check=True)
    return _LIB


_lib = None


def _load():
    global _lib
    if _lib is None:
        build()
        lib = C.CDLL(_LIB)
        lib.orc_create.restype = C.c_void_p
        lib.orc_create.argtypes = [C.POINTER(_Input), C.c_char_p, C.c_int]
        lib.orc_destroy.argtypes = [C.c_void_p]
        for name in ["orc_counts"]:
            getattr(lib, name).argtypes = [C.c_void_p, i64p]
        lib.orc_azimuth.argtypes = [C.c_void_p, C.c_int, f64p]
        lib.orc_polar.argtypes = [C.c_void_p, C.c_int, C.c_int, f64p]
        lib.orc_track2d.argtypes = [C.c_void_p, C.c_int, f64p]
        lib.orc_segments2d.argtypes = [C.c_void_p, C.c_int, i32p, f64p, f64p]
        lib.orc_stack_zeta.argtypes = [C.c_void_p, C.c_int, C.c_int, f64p]
        lib.orc_stack.restype = C.c_int64
        lib.orc_stack.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int64, C.c_int64, i64p, i32p,
                                  i32p, f64p, i64p]
        lib.orc_stack_range.argtypes = [C.c_void_p, C.c_int, C.c_int, i64p]
        lib.orc_link.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int64, C.c_int, i64p]
        lib.orc_volumes.argtypes = [C.c_void_p, f64p]
        lib.orc_fsr_materials.argtypes = [C.c_void_p, i32p]
        lib.orc_set_threads.argtypes = [C.c_void_p, C.c_int]
        lib.orc_reset.argtypes = [C.c_void_p]
        lib.orc_iterate.argtypes = [C.c_void_p, C.c_int, C.c_double, C.c_double, f64p]
        lib.orc_get_flux.argtypes = [C.c_void_p, f64p]
        lib.orc_set_flux.argtypes = [C.c_void_p, f64p, C.c_double]
        lib.orc_sweep_once.argtypes = [C.c_void_p, f64p, f64p, f64p]
        lib.orc_sweep_sample.restype = C.c_int64
        lib.orc_sweep_sample.argtypes = [C.c_void_p, f64p, C.c_int, C.c_int, f64p]
        lib.orc_psi.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int64, C.c_int, f64p, C.c_int]
        lib.orc_clear_psi.argtypes = [C.c_void_p]
        lib.orc_last_error.restype = C.c_char_p
        _lib = lib
    return _lib


def _p(a, t):
    return a.ctypes.data_as(t)


class Oracle:
    """FP64 CPU oracle for one synthetic problem (see ``synth.Problem``)."""

    def __init__(self, prob, n_threads: int | None = None, light: bool = False):
        """light: tracks and segments only (stack, sweep_sample): no links,
        boundary fluxes or volumes, for sampled checks of large problems."""
        lib = _load()
        self.prob = prob
        self._keep = []

        def arr(a, dt):
            a = np.ascontiguousarray(a, dtype=dt)
            self._keep.append(a)
            return a

        inp = _Input()
        inp.ncx, inp.ncy, inp.n_layers = prob.ncx, prob.ncy, prob.n_layers
        inp.pitch, inp.radius, inp.height = prob.pitch, prob.fuel_radius, prob.height
        inp.has_pin = _p(arr(prob.has_pin, np.int32), i32p)
        inp.mat_in = _p(arr(prob.mat_in, np.int32), i32p)
        inp.mat_out = _p(arr(prob.mat_out, np.int32), i32p)
        for i in range(6):
            inp.bc[i] = int(prob.bc[i])
        inp.M, inp.G = prob.num_materials, prob.num_groups
        inp.sigma_t = _p(arr(prob.sigma_t, np.float64), f64p)
        inp.sigma_s = _p(arr(prob.sigma_s, np.float64), f64p)
        inp.nu_sigma_f = _p(arr(prob.nu_sigma_f, np.float64), f64p)
        inp.chi = _p(arr(prob.chi, np.float64), f64p)
        inp.ext_source = (_p(arr(prob.ext_source, np.float64), f64p)
                          if prob.ext_source is not None else f64p())
        inp.n_azim, inp.n_polar = prob.n_azim, prob.n_polar
        inp.radial_spacing, inp.axial_spacing = prob.radial_spacing, prob.axial_spacing
        inp.n_threads = int(n_threads or os.cpu_count() or 1)
        inp.light = 1 if light else 0
        inp.fuel_rings = int(getattr(prob, "fuel_rings", 1))
        inp.mod_rings = int(getattr(prob, "moderator_rings", 0))
        inp.sectors = int(getattr(prob, "sectors", 1))
        lz = getattr(prob, "layer_z", None)
        inp.layer_z = _p(arr(lz, np.float64), f64p) if lz is not None else f64p()
        self.n_threads = inp.n_threads
        err = C.create_string_buffer(256)
        h = lib.orc_create(C.byref(inp), err, 256)
        if not h:
            raise ValueError("oracle: " + err.value.decode())
        self._h = C.c_void_p(h)
        self._lib = lib
        c = np.zeros(16, dtype=np.int64)
        lib.orc_counts(self._h, _p(c, i64p))
        (self.n_fsr, self.n_regions, self.n_tracks2d, self.n_stacks, self.n_tracks3d,
         self.n_segments2d, self.n_azim_quadrant, self.n_polar_half, self.n_z,
         self.cells_per_layer) = [int(x) for x in c[:10]]
        self.G = prob.num_groups

    def __del__(self):
        try:
            self._lib.orc_destroy(self._h)
        except Exception:
            pass

    # --- laydown queries -------------------------------------------------
    def azimuth(self, m):
        out = np.zeros(8)
        assert self._lib.orc_azimuth(self._h, m, _p(out, f64p)) == 0
        keys = ["nx", "ny", "gcd", "Mcyc", "phi_eff", "delta_eff", "span", "step"]
        return dict(zip(keys, out.tolist()))

    def polar(self, m, ph):
        out = np.zeros(8)
        assert self._lib.orc_polar(self._h, m, ph, _p(out, f64p)) == 0
        keys = ["c", "cot", "sin", "cos", "weight", "mu", "w_gl", "track_weight"]
        return dict(zip(keys, out.tolist()))

    def track2d(self, t):
        out = np.zeros(16)
        assert self._lib.orc_track2d(self._h, t, _p(out, f64p)) == 0
        keys = ["azim", "sface", "sk", "eface", "ek", "steps", "M", "x0", "y0", "length",
                "succ_t0", "succ_s0", "succ_t1", "succ_s1", "nseg"]
        d = dict(zip(keys, out.tolist()))
        for k in keys:
            if k not in ("x0", "y0", "length"):
                d[k] = int(d[k])
        return d

    def segments2d(self, t):
        n = self.track2d(t)["nseg"]
        reg = np.zeros(n, dtype=np.int32)
        ln = np.zeros(n)
        pos = np.zeros(n + 1)
        self._lib.orc_segments2d(self._h, t, _p(reg, i32p), _p(ln, f64p), _p(pos, f64p))
        return reg, ln, pos

    def stack_zeta(self, t, p):
        n = self.track2d(t)["nseg"]
        z = np.zeros(n + 1)
        self._lib.orc_stack_zeta(self._h, t, p, _p(z, f64p))
        return z

    def stack_range(self, t, p):
        out = np.zeros(2, dtype=np.int64)
        self._lib.orc_stack_range(self._h, t, p, _p(out, i64p))
        return int(out[0]), int(out[1])

    def stack(self, t, p):
        """Segments of every track of stack (t, p): (track indices, per-track
        counts, fsr ids, lengths) in traversal order along the 2D track."""
        cap_t, cap_s = 4096, 1 << 16
        while True:
            ti = np.zeros(cap_t, dtype=np.int64)
            ns = np.zeros(cap_t, dtype=np.int32)
            fs = np.zeros(cap_s, dtype=np.int32)
            ln = np.zeros(cap_s)
            tot = np.zeros(1, dtype=np.int64)
            n = self._lib.orc_stack(self._h, t, p, cap_t, cap_s, _p(ti, i64p), _p(ns, i32p),
                                    _p(fs, i32p), _p(ln, f64p), _p(tot, i64p))
            if n >= 0:
                m = int(tot[0])
                return ti[:n].copy(), ns[:n].copy(), fs[:m].copy(), ln[:m].copy()
            cap_t *= 4
            cap_s = max(cap_s * 4, int(tot[0]) + 1)

    def link(self, t, p, i, sense):
        out = np.zeros(4, dtype=np.int64)
        rc = self._lib.orc_link(self._h, t, p, i, sense, _p(out, i64p))
        if rc != 0:
            raise IndexError((t, p, i, sense))
        return tuple(int(x) for x in out)

    def psi(self, t, p, i, sense, value=None):
        """Get (or set) the incoming boundary flux of one track direction."""
        v = np.zeros(self.G) if value is None else np.ascontiguousarray(value, dtype=np.float64)
        rc = self._lib.orc_psi(self._h, t, p, int(i), sense, _p(v, f64p), 0 if value is None else 1)
        if rc != 0:
            raise IndexError((t, p, i, sense))
        return v

    def clear_psi(self):
        self._lib.orc_clear_psi(self._h)

    def volumes(self):
        v = np.zeros(self.n_fsr)
        self._lib.orc_volumes(self._h, _p(v, f64p))
        return v

    def fsr_materials(self):
        m = np.zeros(self.n_fsr, dtype=np.int32)
        self._lib.orc_fsr_materials(self._h, _p(m, i32p))
        return m

    # --- iteration ---------------------------------------------------------
    def set_threads(self, n):
        self._lib.orc_set_threads(self._h, int(n))
        self.n_threads = int(n)

    def reset(self):
        self._lib.orc_reset(self._h)

    def iterate(self, max_iter, tol_k=0.0, tol_src=0.0):
        out = np.zeros(8)
        self._lib.orc_iterate(self._h, int(max_iter), float(tol_k), float(tol_src), _p(out, f64p))
        keys = ["k", "iterations", "residual", "production", "absorption", "leakage",
                "converged", "dk"]
        d = dict(zip(keys, out.tolist()))
        d["iterations"] = int(d["iterations"])
        d["converged"] = bool(d["converged"])
        return d

    def flux(self):
        phi = np.zeros(self.n_fsr * self.G)
        self._lib.orc_get_flux(self._h, _p(phi, f64p))
        return phi.reshape(self.n_fsr, self.G)

    def set_flux(self, phi, k):
        phi = np.ascontiguousarray(phi, dtype=np.float64).ravel()
        self._lib.orc_set_flux(self._h, _p(phi, f64p), float(k))

    def sweep_once(self, Q):
        Q = np.ascontiguousarray(Q, dtype=np.float64).ravel()
        tally = np.zeros(self.n_fsr * self.G)
        leak = np.zeros(1)
        self._lib.orc_sweep_once(self._h, _p(Q, f64p), _p(tally, f64p), _p(leak, f64p))
        return tally.reshape(self.n_fsr, self.G), float(leak[0])

    def sweep_sample(self, Q, t0, t1):
        Q = np.ascontiguousarray(Q, dtype=np.float64).ravel()
        tally = np.zeros(self.n_fsr * self.G)
        n = self._lib.orc_sweep_sample(self._h, _p(Q, f64p), int(t0), int(t1), _p(tally, f64p))
        return int(n), tally.reshape(self.n_fsr, self.G)

    def solve(self, tol_k=1e-6, tol_src=1e-5, max_iter=5000):
        self.reset()
        return self.iterate(max_iter, tol_k, tol_src)
