"""Pins of the FP64 oracle against closed forms, invariants and brute force.

Each test fixes something the paper or the mathematics determines
independently of the oracle's own code:

* Gauss-Legendre polar nodes against numpy's leggauss;
* the cyclic laydown against its closed form, exact area sums, reflective
  bijection and the unfolded-torus cycle length;
* 2D and 3D segments (Eqs. 5-11) against dense ray sampling with direct
  point location;
* Eq. 3 on one track of a pure absorber against e^(-Sigma_t l);
* tracked volumes against analytic volumes;
* k of the infinite homogeneous medium against nu-Sigma_f^T (Sigma_t - S^T)^-1 chi,
  the fixed-source infinite medium against (Sigma_t - S^T)^-1 S, and neutron
  balance P/k = absorption + leakage at convergence.
"""
import math

import numpy as np
import pytest

import synth
from tests import bruteforce as bf


@pytest.fixture(scope="module")
def pin(oracle_mod):
    p = synth.pin_cell(1)
    return p, oracle_mod.Oracle(p, n_threads=2)


@pytest.fixture(scope="module")
def lat3r(oracle_mod):
    """lat3 with finer pin-cell regions: 2 fuel rings, 1 moderator ring, 8 sectors."""
    p = synth.lattice(3, n=3, G=3, height=4.0, n_layers=4, n_azim=8, n_polar=4,
                      radial_spacing=0.15, axial_spacing=0.5, bc=(1, 1, 1, 1, 1, 1),
                      n_gt=2, name="lat3r")
    p = p.with_tracks(fuel_rings=2, moderator_rings=1, sectors=8)
    return p, oracle_mod.Oracle(p, n_threads=2)


@pytest.fixture(scope="module")
def lat3z(oracle_mod):
    """lat3 with unequal layers on the axial lattice: 0.5, 1.0, 1.5, 1.0 cm."""
    p = synth.lattice(3, n=3, G=3, height=4.0, n_layers=4, n_azim=8, n_polar=4,
                      radial_spacing=0.15, axial_spacing=0.5, bc=(1, 1, 1, 1, 1, 1),
                      n_gt=2, name="lat3z")
    p = p.with_tracks(layer_z=np.array([0.0, 0.5, 1.5, 3.0, 4.0]))
    return p, oracle_mod.Oracle(p, n_threads=2)


@pytest.fixture(scope="module")
def lat3o(oracle_mod):
    """lat3 with layer planes off the axial lattice (0.6, 1.7 and 3.1 cm with
    0.5 cm spacing: plane fractions 0.2, 0.4 and 0.2 of a spacing)."""
    p = synth.lattice(3, n=3, G=3, height=4.0, n_layers=4, n_azim=8, n_polar=4,
                      radial_spacing=0.15, axial_spacing=0.5, bc=(1, 1, 1, 1, 1, 1),
                      n_gt=2, name="lat3o")
    p = p.with_tracks(layer_z=np.array([0.0, 0.6, 1.7, 3.1, 4.0]))
    return p, oracle_mod.Oracle(p, n_threads=2)


@pytest.fixture(scope="module")
def lat3(oracle_mod):
    p = synth.lattice(3, n=3, G=3, height=4.0, n_layers=4, n_azim=8, n_polar=4,
                      radial_spacing=0.15, axial_spacing=0.5, bc=(1, 1, 1, 1, 1, 1),
                      n_gt=2, name="lat3")
    return p, oracle_mod.Oracle(p, n_threads=2)


# --------------------------------------------------------------- quadrature

def test_gauss_legendre_matches_numpy(oracle_mod):
    for P in (2, 4, 6, 8, 12):
        p = synth.pin_cell(1, n_polar=P)
        o = oracle_mod.Oracle(p, n_threads=1)
        x, w = np.polynomial.legendre.leggauss(P // 2)
        mu_ref = np.sort(0.5 * (1 + x))
        w_ref = 0.5 * w[np.argsort(0.5 * (1 + x))]
        mu = np.array([o.polar(0, j)["mu"] for j in range(P // 2)])
        wg = np.array([o.polar(0, j)["w_gl"] for j in range(P // 2)])
        np.testing.assert_allclose(mu, mu_ref, rtol=0, atol=1e-14)
        np.testing.assert_allclose(wg, w_ref, rtol=0, atol=1e-14)


def test_polar_correction_closes_cycles(pin, lat3):
    for p, o in (pin, lat3):
        for m in range(o.n_azim_quadrant):
            az = o.azimuth(m)
            Lc = az["Mcyc"] * az["step"]
            for j in range(o.n_polar_half):
                pl = o.polar(m, j)
                dz = p.height / o.n_z
                assert abs(Lc * pl["cot"] / dz - round(Lc * pl["cot"] / dz)) < 1e-9
                cot_gl = pl["mu"] / math.sqrt(1 - pl["mu"] ** 2)
                assert abs(pl["cot"] - cot_gl) <= 0.5 * dz / Lc + 1e-12 or pl["c"] == 1
                assert abs(pl["sin"] ** 2 + pl["cos"] ** 2 - 1) < 1e-14


# --------------------------------------------------------------- 2D laydown

def test_laydown_closed_form(pin):
    p, o = pin
    # phi_0 = 22.5 deg over a 1.26 cm cell with 0.1 cm spacing: nx = ceil(4.82) = 5,
    # ny = ceil(11.64) = 12, tan(phi_eff) = 5/12, delta_eff = 0.252 * 5/13
    az = o.azimuth(0)
    assert (az["nx"], az["ny"]) == (5, 12)
    assert abs(az["phi_eff"] - math.atan2(5, 12)) < 1e-15
    assert abs(az["delta_eff"] - 0.252 * 5 / 13) < 1e-15
    for m in range(o.n_azim_quadrant):
        ref = bf.laydown(p, m)
        az = o.azimuth(m)
        assert (az["nx"], az["ny"]) == (ref["nx"], ref["ny"])
        assert abs(az["phi_eff"] - ref["phi_eff"]) < 1e-14
        assert abs(az["delta_eff"] - ref["delta_eff"]) < 1e-14
        # both face spacings give the same perpendicular spacing
        assert abs((ref["W_y"] / ref["ny"]) * math.cos(ref["phi_eff"]) - az["delta_eff"]) < 1e-14
    spans = [o.azimuth(m)["span"] for m in range(o.n_azim_quadrant)]
    assert abs(sum(spans) - math.pi / 2) < 1e-14


def test_cycle_length_unfolded_torus(pin, lat3):
    for p, o in (pin, lat3):
        for m in range(o.n_azim_quadrant):
            az = o.azimuth(m)
            W_x, W_y = p.ncx * p.pitch, p.ncy * p.pitch
            L = 2 * math.hypot(W_x * az["ny"], W_y * az["nx"]) / math.gcd(int(az["nx"]), int(az["ny"]))
            assert abs(az["Mcyc"] * az["step"] - L) < 1e-11 * L


def test_track_area_sums_exact(pin, lat3):
    """Parallel tracks at half-offsets tile the rectangle exactly: the sum of
    delta_eff * length per azimuth equals the domain area."""
    for p, o in (pin, lat3):
        area = p.ncx * p.pitch * p.ncy * p.pitch
        sums = {}
        for t in range(o.n_tracks2d):
            tr = o.track2d(t)
            m = tr["azim"] if tr["azim"] < o.n_azim_quadrant else p.n_azim // 2 - 1 - tr["azim"]
            sums[tr["azim"]] = sums.get(tr["azim"], 0.0) + o.azimuth(m)["delta_eff"] * tr["length"]
        for a, s in sums.items():
            assert abs(s - area) < 1e-12 * area, (a, s, area)


def test_2d_links_are_reflections(pin, lat3):
    for p, o in (pin, lat3):
        seen = set()
        for t in range(o.n_tracks2d):
            tr = o.track2d(t)
            x0, y0, dx, dy, _ = bf.track_start_dir(p, tr)
            L = bf.exit_length(p, x0, y0, dx, dy)
            assert abs(L - tr["length"]) < 1e-12
            assert abs(x0 - tr["x0"]) < 1e-13 and abs(y0 - tr["y0"]) < 1e-13
            for sense in (0, 1):
                ex, ey = (x0 + L * dx, y0 + L * dy) if sense == 0 else (x0, y0)
                ddx, ddy = (dx, dy) if sense == 0 else (-dx, -dy)
                W_x, W_y = p.ncx * p.pitch, p.ncy * p.pitch
                if abs(ex) < 1e-12 or abs(ex - W_x) < 1e-12:
                    rdx, rdy = -ddx, ddy
                else:
                    rdx, rdy = ddx, -ddy
                t2, s2 = tr[f"succ_t{sense}"], tr[f"succ_s{sense}"]
                assert (t2, s2) not in seen
                seen.add((t2, s2))
                tr2 = o.track2d(t2)
                x2, y2, dx2, dy2, _ = bf.track_start_dir(p, tr2)
                L2 = bf.exit_length(p, x2, y2, dx2, dy2)
                px, py = (x2, y2) if s2 == 0 else (x2 + L2 * dx2, y2 + L2 * dy2)
                qx, qy = (dx2, dy2) if s2 == 0 else (-dx2, -dy2)
                assert abs(px - ex) < 1e-11 and abs(py - ey) < 1e-11
                assert abs(qx - rdx) < 1e-12 and abs(qy - rdy) < 1e-12
        assert len(seen) == 2 * o.n_tracks2d


def test_cycle_positions_chain(pin, lat3):
    """A forward-to-forward link advances the cycle position by the track's
    length in steps (mod the cycle)."""
    for p, o in (pin, lat3):
        for t in range(o.n_tracks2d):
            tr = o.track2d(t)
            m = tr["azim"] if tr["azim"] < o.n_azim_quadrant else p.n_azim // 2 - 1 - tr["azim"]
            Mc = int(o.azimuth(m)["Mcyc"])
            t2, s2 = tr["succ_t0"], tr["succ_s0"]
            tr2 = o.track2d(t2)
            if s2 == 0:
                assert tr2["M"] == (tr["M"] + tr["steps"]) % Mc
            else:
                assert tr2["M"] == (Mc - (tr["M"] + tr["steps"]) - tr2["steps"]) % Mc


def test_2d_segments_bruteforce(pin, lat3, lat3r):
    for p, o in (pin, lat3, lat3r):
        for t in range(0, o.n_tracks2d, max(1, o.n_tracks2d // 25)):
            tr = o.track2d(t)
            reg, ln, pos = o.segments2d(t)
            assert abs(ln.sum() - tr["length"]) < 1e-12
            assert abs(pos[-1] - tr["length"]) < 1e-12
            x0, y0, dx, dy, _ = bf.track_start_dir(p, tr)
            ids, lens, h = bf.ray_regions(p, x0, y0, dx, dy, tr["length"])
            a_i, a_l = bf.drop_short(reg.astype(np.int64), ln, 4 * h)
            b_i, b_l = bf.drop_short(ids, lens, 4 * h)
            np.testing.assert_array_equal(a_i, b_i)
            np.testing.assert_allclose(a_l, b_l, atol=6 * h)


# --------------------------------------------------------------- 3D stacks

def _stack_checks(p, o, t, p_idx):
    tr = o.track2d(t)
    x0, y0, dx, dy, _ = bf.track_start_dir(p, tr)
    a = tr["azim"]
    m = a if a < o.n_azim_quadrant else p.n_azim // 2 - 1 - a
    Ph = o.n_polar_half
    pl = o.polar(m, p_idx % Ph)
    cot = pl["cot"] if p_idx < Ph else -pl["cot"]
    dz = p.height / o.n_z
    zeta = o.stack_zeta(t, p_idx)
    # z_0 of the reading: dz/2 + S_T cot (mod dz), S_T = M steps
    az = o.azimuth(m)
    z0_ref = (0.5 + tr["M"] * az["step"] * cot / dz) % 1.0
    assert abs(zeta[0] - z0_ref) < 1e-9 or abs(abs(zeta[0] - z0_ref) - 1) < 1e-9
    ti, ns, fs, ln = o.stack(t, p_idx)
    imin, n = o.stack_range(t, p_idx)
    assert len(ti) == n and (n == 0 or (ti[0] == imin and ti[-1] == imin + n - 1))
    offs = np.concatenate([[0], np.cumsum(ns)])
    for k in range(0, len(ti), max(1, len(ti) // 6)):
        i = ti[k]
        f = fs[offs[k]:offs[k + 1]].astype(np.int64)
        l = ln[offs[k]:offs[k + 1]]
        ids, lens, h = bf.ray_fsrs_3d(p, x0, y0, dx, dy, tr["length"], (i + zeta[0]) * dz, cot,
                                      n_samples=100000)
        # compare the pieces longer than a threshold that no exact piece lies
        # near: a sampled run is within one sample length h of its piece
        thr = next(T * h for T in (4, 8, 12, 16, 24, 32)
                   if not np.any(np.abs(l - T * h) < 1.5 * h))
        a_i, a_l = bf.drop_short(f, l, thr)
        b_i, b_l = bf.drop_short(ids, lens, thr)
        np.testing.assert_array_equal(a_i, b_i)
        np.testing.assert_allclose(a_l, b_l, atol=8 * h)
        # total 3D length inside the box from the clipped line
        s_lo = max(0.0, (0 - (i + zeta[0]) * dz) / cot) if cot > 0 else max(0.0, (p.height - (i + zeta[0]) * dz) / cot)
        s_hi = min(tr["length"], (p.height - (i + zeta[0]) * dz) / cot) if cot > 0 else min(tr["length"], (0 - (i + zeta[0]) * dz) / cot)
        sin = 1 / math.sqrt(1 + cot * cot)
        assert abs(l.sum() - (s_hi - s_lo) / sin) < 1e-9


def test_3d_segments_bruteforce(pin, lat3, lat3r, lat3z, lat3o):
    for p, o in (pin, lat3, lat3r, lat3z, lat3o):
        for t in range(0, o.n_tracks2d, max(1, o.n_tracks2d // 8)):
            for p_idx in range(p.n_polar):
                _stack_checks(p, o, t, p_idx)


def test_3d_links_bijection(pin, lat3):
    """All six faces reflective: every track direction receives exactly one
    incoming flux, and reflective links preserve the track weight."""
    for p, o in (pin, lat3):
        dest = {}
        for t in range(o.n_tracks2d):
            for p_idx in range(p.n_polar):
                imin, n = o.stack_range(t, p_idx)
                for i in range(imin, imin + n):
                    for s in (0, 1):
                        d = o.link(t, p_idx, i, s)
                        assert d[0] >= 0
                        assert d not in dest, (t, p_idx, i, s, d)
                        dest[d] = (t, p_idx, i, s)
                        a1 = o.track2d(t)["azim"]
                        a2 = o.track2d(d[0])["azim"]
                        nq = o.n_azim_quadrant
                        m1 = a1 if a1 < nq else p.n_azim // 2 - 1 - a1
                        m2 = a2 if a2 < nq else p.n_azim // 2 - 1 - a2
                        assert m1 == m2 and p_idx % o.n_polar_half == d[1] % o.n_polar_half
        assert len(dest) == 2 * o.n_tracks3d


def test_3d_links_land_on_exit_point(lat3):
    p, o = lat3
    dz = p.height / o.n_z
    H = p.height
    rng = np.random.default_rng(0)

    def geom(t, p_idx):
        tr = o.track2d(t)
        x0, y0, dx, dy, _ = bf.track_start_dir(p, tr)
        a = tr["azim"]
        m = a if a < o.n_azim_quadrant else p.n_azim // 2 - 1 - a
        pl = o.polar(m, p_idx % o.n_polar_half)
        cot = pl["cot"] if p_idx < o.n_polar_half else -pl["cot"]
        return x0, y0, dx, dy, tr["length"], cot, o.stack_zeta(t, p_idx)[0]

    def endpoints(t, p_idx, i):
        x0, y0, dx, dy, L, cot, z0 = geom(t, p_idx)
        zs = (i + z0) * dz
        s_lo = max(0.0, -zs / cot) if cot > 0 else max(0.0, (H - zs) / cot)
        s_hi = min(L, (H - zs) / cot) if cot > 0 else min(L, -zs / cot)
        P0 = np.array([x0 + s_lo * dx, y0 + s_lo * dy, zs + s_lo * cot])
        P1 = np.array([x0 + s_hi * dx, y0 + s_hi * dy, zs + s_hi * cot])
        return P0, P1

    for _ in range(300):
        t = int(rng.integers(o.n_tracks2d))
        p_idx = int(rng.integers(p.n_polar))
        imin, n = o.stack_range(t, p_idx)
        i = imin + int(rng.integers(n))
        s = int(rng.integers(2))
        P0, P1 = endpoints(t, p_idx, i)
        exit_pt = P1 if s == 0 else P0
        t2, p2, i2, s2 = o.link(t, p_idx, i, s)
        Q0, Q1 = endpoints(t2, p2, i2)
        entry = Q0 if s2 == 0 else Q1
        assert np.abs(exit_pt - entry).max() < 1e-9


# --------------------------------------------------------------- volumes

def test_tracked_volumes_match_analytic(oracle_mod):
    errs = []
    for spacing in (0.1, 0.05, 0.02):
        p = synth.pin_cell(1, radial_spacing=spacing, n_azim=16)
        o = oracle_mod.Oracle(p, n_threads=2)
        V = o.volumes().reshape(2, p.n_layers)
        h = p.height / p.n_layers
        fuel = math.pi * p.fuel_radius ** 2 * h
        mod = p.pitch ** 2 * h - fuel
        # total volume is exact (area sums are exact and every layer is covered)
        assert abs(V.sum() - p.pitch ** 2 * p.height) < 1e-9 * p.pitch ** 2 * p.height
        errs.append(max(abs(V[0] / fuel - 1).max(), abs(V[1] / mod - 1).max()))
    # midpoint-rule chord sums: well inside 1 % at these spacings
    assert max(errs) < 0.005, errs


def _ring_sector_volumes(p):
    """Analytic volume of every radial region of a one-pin cell with rings and
    sectors (2, 4 or 8 sectors: the square's corner region splits evenly)."""
    from tests.bruteforce import circle_radii2
    r2 = circle_radii2(p)
    S = p.sectors
    areas = [math.pi * (r2[0])] + [math.pi * (r2[k] - r2[k - 1]) for k in range(1, len(r2))]
    areas.append(p.pitch ** 2 - math.pi * r2[-1])
    return np.repeat(np.array(areas) / S, S) * (p.height / p.n_layers)


@pytest.mark.parametrize("sectors", [1, 4, 8])
def test_ring_sector_volumes_match_analytic(oracle_mod, sectors):
    """Tracked volumes of rings and sectors converge to the analytic areas
    under track refinement; the cell total stays exact."""
    errs = []
    for spacing in (0.04, 0.02, 0.01):
        p = synth.pin_cell(1, radial_spacing=spacing, n_azim=32).with_tracks(
            fuel_rings=3, moderator_rings=2, sectors=sectors)
        o = oracle_mod.Oracle(p, n_threads=4)
        V = o.volumes().reshape(p.pin_regions, p.n_layers)
        ref = _ring_sector_volumes(p)
        assert abs(V.sum() - p.pitch ** 2 * p.height) < 1e-9 * p.pitch ** 2 * p.height
        errs.append(np.abs(V / ref[:, None] - 1).max())
    assert errs[-1] < 0.01 and errs[-1] < errs[0], errs


# --------------------------------------------------------------- Eq. 3

def test_eq3_single_track_pure_absorber(lat3):
    """Q = 0: a flux entering one track leaves it attenuated by
    exp(-sum Sigma_t l), and each FSR tallies W times the flux drop inside it."""
    p, o = lat3
    G = p.num_groups
    mat = o.fsr_materials()
    rng = np.random.default_rng(3)
    for _ in range(5):
        t = int(rng.integers(o.n_tracks2d))
        p_idx = int(rng.integers(p.n_polar))
        ti, ns, fs, ln = o.stack(t, p_idx)
        k = int(rng.integers(len(ti)))
        i = int(ti[k])
        offs = np.concatenate([[0], np.cumsum(ns)])
        f = fs[offs[k]:offs[k + 1]]
        l = ln[offs[k]:offs[k + 1]]
        for sense in (0, 1):
            o.clear_psi()
            psi_in = rng.uniform(0.5, 2.0, size=G)
            o.psi(t, p_idx, i, sense, psi_in)
            tally, leak = o.sweep_once(np.zeros((o.n_fsr, G)))
            order = range(len(f)) if sense == 0 else range(len(f) - 1, -1, -1)
            psi = psi_in.copy()
            a = o.track2d(t)["azim"]
            m = a if a < o.n_azim_quadrant else p.n_azim // 2 - 1 - a
            W = o.polar(m, p_idx % o.n_polar_half)["track_weight"]
            ref = np.zeros((o.n_fsr, G))
            for j in order:
                att = np.exp(-p.sigma_t[mat[f[j]]] * l[j])
                ref[f[j]] += W * psi * (1 - att)
                psi = psi * att
            d = o.link(t, p_idx, i, sense)
            np.testing.assert_allclose(o.psi(*d), psi, rtol=1e-13)
            np.testing.assert_allclose(tally, ref, rtol=1e-12, atol=1e-300)
            assert leak == 0.0
    o.reset()


def test_eq3_flat_source_equilibrium(oracle_mod):
    """Homogeneous medium with psi_in = Q / Sigma_t everywhere: every segment
    keeps psi = Q / Sigma_t and tallies nothing."""
    p = synth.pin_cell(2, homogeneous=True, G=2)
    o = oracle_mod.Oracle(p, n_threads=2)
    G = p.num_groups
    Q = np.tile(np.array([0.7, 0.3]), (o.n_fsr, 1))
    eq = Q[0] / p.sigma_t[0]
    for t in range(o.n_tracks2d):
        for p_idx in range(p.n_polar):
            imin, n = o.stack_range(t, p_idx)
            for i in range(imin, imin + n):
                for s in (0, 1):
                    o.psi(t, p_idx, i, s, eq)
    tally, _ = o.sweep_once(Q)
    assert np.abs(tally).max() < 1e-14
    d = o.link(0, 0, o.stack_range(0, 0)[0], 0)
    np.testing.assert_allclose(o.psi(*d), eq, rtol=1e-14)


# --------------------------------------------------------------- iteration

@pytest.mark.parametrize("layers", ["equal", "unequal"])
def test_infinite_medium_k_closed_form(oracle_mod, layers):
    for G, seed in ((2, 1), (4, 7)):
        if layers == "unequal":
            p = synth.pin_cell(seed, G=G, homogeneous=True, n_layers=3).with_tracks(
                layer_z=np.array([0.0, 0.5, 1.5, 2.0]))
        else:
            p = synth.pin_cell(seed, G=G, homogeneous=True)
        o = oracle_mod.Oracle(p, n_threads=2)
        r = o.solve(tol_k=1e-13, tol_src=1e-12, max_iter=20000)
        assert r["converged"]
        st, ss, nsf, chi = p.sigma_t[0], p.sigma_s[0], p.nu_sigma_f[0], p.chi[0]
        A = np.diag(st) - ss.T
        spec = np.linalg.solve(A, chi)
        kinf = nsf @ spec
        assert abs(r["k"] - kinf) < 1e-9
        phi = o.flux()
        # flat in space, spectrum (Sigma_t - S^T)^-1 chi
        np.testing.assert_allclose(phi, np.tile(phi[0], (o.n_fsr, 1)), rtol=1e-9)
        np.testing.assert_allclose(phi[0] / phi[0].sum(), spec / spec.sum(), rtol=1e-9)


def test_infinite_medium_fixed_source_closed_form(oracle_mod):
    p = synth.pin_cell(5, G=3, homogeneous=True)
    p = p.with_tracks(nu_sigma_f=np.zeros_like(p.nu_sigma_f),
                      ext_source=np.tile([[1.0, 0.4, 0.2]], (p.num_materials, 1)))
    o = oracle_mod.Oracle(p, n_threads=2)
    r = o.solve(tol_k=0, tol_src=1e-13, max_iter=20000)
    assert r["converged"]
    A = np.diag(p.sigma_t[0]) - p.sigma_s[0].T
    ref = np.linalg.solve(A, p.ext_source[0])
    np.testing.assert_allclose(o.flux(), np.tile(ref, (o.n_fsr, 1)), rtol=1e-10)


def test_neutron_balance_with_leakage(oracle_mod):
    p = synth.lattice(2, n=3, G=3, height=4.0, n_layers=2, n_azim=8, n_polar=4,
                      radial_spacing=0.2, axial_spacing=0.5, bc=(1, 0, 1, 1, 0, 1), n_gt=1)
    o = oracle_mod.Oracle(p, n_threads=2)
    r = o.solve(tol_k=1e-12, tol_src=1e-11, max_iter=20000)
    assert r["converged"]
    assert r["leakage"] > 0.01 * r["absorption"]
    assert abs(r["production"] / r["k"] - (r["absorption"] + r["leakage"])) < 1e-9 * r["production"] / r["k"]


def test_pin_cell_axial_mirror_symmetry(pin):
    """All six faces reflective and an axially uniform cell.  The laydown is
    symmetric under z -> H - z (each downward stack is the mirror image of an
    upward one), so layer L and layer NL-1-L carry the same flux exactly; the
    layers differ from each other only by the discretisation (small)."""
    p, o = pin
    r = o.solve(tol_k=1e-12, tol_src=1e-11, max_iter=20000)
    assert r["converged"]
    phi = o.flux().reshape(2, p.n_layers, p.num_groups)
    np.testing.assert_allclose(phi, phi[:, ::-1, :], rtol=1e-10)
    for reg in range(2):
        np.testing.assert_allclose(phi[reg], np.tile(phi[reg, 0], (p.n_layers, 1)), rtol=2e-3)
    V = o.volumes().reshape(2, p.n_layers)
    np.testing.assert_allclose(V, V[:, ::-1], rtol=1e-12)
    assert abs(r["production"] / r["k"] - r["absorption"]) < 1e-9 * r["absorption"]


def test_unequal_layer_volumes_match_analytic(oracle_mod):
    """Unequal layers (0.5, 1.0, 0.5 cm on the 0.5 cm axial lattice): each
    FSR's tracked volume is its radial area times its layer's height, the
    area from the same per-azimuth chord sums in every layer."""
    p = synth.pin_cell(1, radial_spacing=0.02, n_azim=32, n_layers=3).with_tracks(
        layer_z=np.array([0.0, 0.5, 1.5, 2.0]))
    o = oracle_mod.Oracle(p, n_threads=4)
    V = o.volumes().reshape(2, 3)
    h = np.diff(p.layer_z)
    fuel = math.pi * p.fuel_radius ** 2
    np.testing.assert_allclose(V[0] / h, fuel, rtol=0.005)
    np.testing.assert_allclose(V[1] / h, p.pitch ** 2 - fuel, rtol=0.005)
    # every layer sees the same radial areas: the ratios are exact up to rounding
    np.testing.assert_allclose(V[:, 1] / V[:, 0], h[1] / h[0], rtol=1e-9)
    assert abs(V.sum() - p.pitch ** 2 * p.height) < 1e-9 * p.pitch ** 2 * p.height


def test_layers_off_the_lattice_volumes_match_analytic(oracle_mod):
    """Layer planes off the axial lattice (0.6 and 1.3 cm, Sec. 2.2's local
    axial mesh): each FSR's tracked volume is its radial area times its
    layer's height, within the sampling of the track layout, and closer as
    the axial spacing is refined; the total volume stays exact."""
    errs = []
    for dz in (0.5, 0.1):
        p = synth.pin_cell(1, radial_spacing=0.02, n_azim=32, n_layers=3,
                           axial_spacing=dz).with_tracks(layer_z=np.array([0.0, 0.6, 1.3, 2.0]))
        o = oracle_mod.Oracle(p, n_threads=4)
        V = o.volumes().reshape(2, 3)
        h = np.diff(p.layer_z)
        fuel = math.pi * p.fuel_radius ** 2
        ref = np.array([fuel * h, (p.pitch ** 2 - fuel) * h])
        errs.append(np.abs(V / ref - 1).max())
        assert abs(V.sum() - p.pitch ** 2 * p.height) < 1e-9 * p.pitch ** 2 * p.height
    assert errs[0] < 0.01 and errs[1] < errs[0], errs


def test_layers_off_the_lattice_infinite_medium_k(oracle_mod):
    """An off-lattice axial mesh of the homogeneous, all-reflective pin cell
    is still an infinite medium: k = nuSigma_f^T (Sigma_t - S^T)^-1 chi."""
    p = synth.pin_cell(1, homogeneous=True, n_layers=3).with_tracks(
        layer_z=np.array([0.0, 0.35, 1.45, 2.0]))
    o = oracle_mod.Oracle(p, n_threads=2)
    r = o.solve(tol_k=1e-12, tol_src=1e-11, max_iter=4000)
    m = 0
    A = np.diag(p.sigma_t[m]) - p.sigma_s[m].T
    kinf = p.nu_sigma_f[m] @ np.linalg.solve(A, p.chi[m])
    assert abs(r["k"] - kinf) < 1e-9, (r["k"], kinf)


def test_layer_planes_must_rise_from_zero_to_the_height(oracle_mod):
    for lz in ([0.1, 0.6, 1.5, 2.0], [0.0, 0.6, 1.5, 1.9], [0.0, 1.5, 0.6, 2.0]):
        p = synth.pin_cell(1, n_layers=3).with_tracks(layer_z=np.array(lz))
        with pytest.raises(ValueError):
            oracle_mod.Oracle(p, n_threads=1)


def test_equal_layers_off_the_lattice(oracle_mod):
    """Three equal layers of 2/3 cm with a 0.5 cm axial spacing: their planes
    lie 4/3 and 8/3 spacings up, off the lattice, and are taken as a plane
    list L H / n_layers.  Volumes per layer match the analytic ones and the
    3D segments the brute-force ray march."""
    p = synth.pin_cell(1, radial_spacing=0.02, n_azim=32, n_layers=3, axial_spacing=0.5)
    o = oracle_mod.Oracle(p, n_threads=4)
    V = o.volumes().reshape(2, 3)
    fuel = math.pi * p.fuel_radius ** 2
    h = p.height / 3
    ref = np.array([[fuel * h] * 3, [(p.pitch ** 2 - fuel) * h] * 3])
    assert np.abs(V / ref - 1).max() < 0.01
    assert abs(V.sum() - p.pitch ** 2 * p.height) < 1e-9 * p.pitch ** 2 * p.height
    q = synth.pin_cell(1, n_layers=3, axial_spacing=0.5)
    oq = oracle_mod.Oracle(q, n_threads=2)
    for t in range(0, oq.n_tracks2d, max(1, oq.n_tracks2d // 6)):
        for p_idx in range(q.n_polar):
            _stack_checks(q, oq, t, p_idx)


def _track_pieces(o, t, p_idx, i):
    ti, ns, fs, ln = o.stack(t, p_idx)
    k = int(np.flatnonzero(ti == i)[0])
    a = int(ns[:k].sum())
    return fs[a:a + ns[k]], ln[a:a + ns[k]]


@pytest.mark.parametrize("down", [False, True])
def test_plane_ties_are_exact(oracle_mod, down):
    """A layer plane placed exactly at the height where a track starts (the
    2D track's first boundary): an upward track that starts on the plane lies
    above it from its first piece, a downward one below it.  Its pieces are
    those of the same track with the plane moved by 1e-7 spacings to the
    side the convention puts the track on (no piece of zero or rounding
    length at the tie), and differ from the other side's (a short first
    piece in the other layer)."""
    base = synth.pin_cell(1, n_layers=3)
    dz = 0.5
    o0 = oracle_mod.Oracle(base.with_tracks(layer_z=np.array([0.0, 0.6, 1.3, 2.0])), n_threads=1)
    p_idx = base.n_polar // 2 if down else 0
    t = next(t for t in range(o0.n_tracks2d)
             if 0.05 < o0.stack_zeta(t, p_idx)[0] % 1.0 < 0.95)
    z0 = o0.stack_zeta(t, p_idx)[0]
    f0 = z0 - math.floor(z0)
    i = 1 - math.floor(z0)  # the track at u = i + z0 = 1 + f0 at its start

    def pieces(eps):
        mesh = np.array([0.0, (1.0 + f0 + eps) * dz, 1.3, 2.0])
        o = oracle_mod.Oracle(base.with_tracks(layer_z=mesh), n_threads=1)
        return _track_pieces(o, t, p_idx, i)

    f_tie, l_tie = pieces(0.0)
    f_lo, l_lo = pieces(-1e-7)   # the plane just below the start
    f_hi, l_hi = pieces(1e-7)    # just above
    assert l_tie.min() > 1e-6
    same, other = (f_hi, f_lo) if down else (f_lo, f_hi)
    np.testing.assert_array_equal(f_tie, same)
    assert len(other) == len(f_tie) + 1
    assert f_tie[0] % 3 == (0 if down else 1)
