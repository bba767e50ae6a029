"""Seeded synthetic problem generators for the 3D MOC sweep.

This module is shared by the FP64 CPU oracle (``oracle/``) and the GPU
library binding (``paper_2503_17743_gb300``).  It holds no transport
arithmetic: it only draws lattice layouts and multigroup cross sections from
a seeded generator and returns plain numpy arrays.  Every workload here is
synthetic.  The paper measures on the C5G7 3D extension benchmark (Sec. 5.1,
Table 2), whose data is not available; these lattices only mimic its shapes
(17x17 pin lattices, pitch 1.26 cm, fuel radius 0.54 cm, 7 groups, reflector
assemblies, an axially inserted absorber) and use none of its numbers.

Conventions shared by both consumers (they are inputs, not arithmetic):

* cells are indexed ``c = cy * ncx + cx`` with ``cx`` along x;
* a pin cell has (circles + 1) x sectors radial regions, numbered
  ``ring * sectors + sector`` from the centre outwards: ``fuel_rings`` rings
  of equal area inside the fuel circle, ``moderator_rings`` circles whose
  squared radii step evenly from the fuel radius towards half the pitch,
  then the rest of the cell; sector s covers the angles
  [2 pi s / S, 2 pi (s+1) / S) counterclockwise from +x about the cell
  centre.  Rings inside the fuel circle hold ``mat_in``, the others
  ``mat_out``.  With the defaults (1, 0, 1) a pin cell has two regions
  (circle, then moderator).  Every other cell is one region; radial regions
  are numbered cell by cell;
* a flat source region (FSR) is ``region * n_layers + layer`` (layer 0 at
  z = 0); layers are equal unless ``layer_z`` lists the n_layers + 1 planes
  from 0 to the height, each a whole number of axial spacings;
* ``bc`` lists the faces xmin, xmax, ymin, ymax, zmin, zmax with 1 =
  reflective and 0 = vacuum;
* ``sigma_s[m, g, h]`` is the scattering cross section from group g into
  group h; ``ext_source[m, g]`` is an isotropic volumetric source density.
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace
from typing import Optional

import numpy as np

PITCH = 1.26          # cm, pin pitch of the C5G7-like lattices (Sec. 5.1)
FUEL_RADIUS = 0.54    # cm
ASSEMBLY = 17         # pins per assembly side

# material slots used by the generators
MAT_FUEL, MAT_MOD, MAT_GT, MAT_ABS = 0, 1, 2, 3


@dataclass
class Problem:
    """One synthetic 3D MOC problem: geometry, cross sections, track layout."""

    name: str
    ncx: int
    ncy: int
    pitch: float
    fuel_radius: float
    height: float
    n_layers: int
    has_pin: np.ndarray          # int32 [ncy*ncx]
    mat_in: np.ndarray           # int32 [ncy*ncx*n_layers], material inside the circle
    mat_out: np.ndarray          # int32 [ncy*ncx*n_layers], moderator / whole-cell material
    bc: tuple                    # (xmin, xmax, ymin, ymax, zmin, zmax), 1 reflective, 0 vacuum
    sigma_t: np.ndarray          # float64 [M, G]
    sigma_s: np.ndarray          # float64 [M, G, G]  (from g into h)
    nu_sigma_f: np.ndarray       # float64 [M, G]
    chi: np.ndarray              # float64 [M, G]
    ext_source: Optional[np.ndarray]  # float64 [M, G] or None
    n_azim: int
    n_polar: int                 # total over both hemispheres
    radial_spacing: float
    axial_spacing: float
    seed: int = 0
    fuel_rings: int = 1
    moderator_rings: int = 0
    sectors: int = 1
    layer_z: Optional[np.ndarray] = None   # float64 [n_layers + 1] planes, or None: equal layers
    meta: dict = field(default_factory=dict)

    @property
    def num_groups(self) -> int:
        return int(self.sigma_t.shape[1])

    @property
    def num_materials(self) -> int:
        return int(self.sigma_t.shape[0])

    @property
    def pin_regions(self) -> int:
        return (self.fuel_rings + self.moderator_rings + 1) * self.sectors

    @property
    def n_regions(self) -> int:
        return int(np.sum(np.where(self.has_pin != 0, self.pin_regions, 1)))

    @property
    def n_fsr(self) -> int:
        return self.n_regions * self.n_layers

    @property
    def fixed_source(self) -> bool:
        return self.ext_source is not None

    def with_tracks(self, **kw) -> "Problem":
        return replace(self, **kw)


# ---------------------------------------------------------------------------
# cross sections


def make_cross_sections(rng: np.random.Generator, G: int, kinds: list[str],
                        sigt_range=(0.2, 2.0), scat_range=(0.5, 0.95),
                        upscatter_groups: int = 3):
    """Draw one material per entry of ``kinds`` (fuel / mod / gt / abs).

    Sigma_t ~ U(sigt_range).  Scatter ratio c_g ~ U(scat_range) (absorber
    c ~ U(0.4, 0.6)), split among target groups with uniform random weights:
    downscatter to h >= g, and for the last ``upscatter_groups`` groups also
    upscatter inside that thermal block.  Fuel gets nu-Sigma_f =
    U(0.5, 1.5) * Sigma_a; chi is spread over the first three groups (first
    group only when G <= 2).
    """
    M = len(kinds)
    st = np.zeros((M, G))
    ss = np.zeros((M, G, G))
    nsf = np.zeros((M, G))
    chi = np.zeros((M, G))
    n_chi = 1 if G <= 2 else min(3, G)
    w_chi = rng.uniform(0.2, 1.0, size=n_chi)
    w_chi /= w_chi.sum()
    thermal0 = max(0, G - upscatter_groups) if G > upscatter_groups else G
    for m, kind in enumerate(kinds):
        sig = rng.uniform(*sigt_range, size=G)
        if kind == "abs":
            c = rng.uniform(0.4, 0.6, size=G)
            sig = rng.uniform(max(sigt_range[0], 0.5 * sigt_range[1]), sigt_range[1], size=G)
        else:
            c = rng.uniform(*scat_range, size=G)
        st[m] = sig
        for g in range(G):
            if g >= thermal0 and G > upscatter_groups:
                targets = np.arange(thermal0, G)
                targets = targets[targets >= g - 2]
            else:
                targets = np.arange(g, min(G, g + 3))
            w = rng.uniform(0.05, 1.0, size=targets.size)
            # keep most of the scattering in-group or one group down
            w[targets == g] += 1.0
            w /= w.sum()
            ss[m, g, targets] = c[g] * sig[g] * w
        if kind == "fuel":
            sig_a = st[m] - ss[m].sum(axis=1)
            nsf[m] = rng.uniform(0.5, 1.5, size=G) * sig_a
            chi[m, :n_chi] = w_chi
    return st, ss, nsf, chi


# ---------------------------------------------------------------------------
# lattices


def _guide_tube_mask(rng: np.random.Generator, n: int = ASSEMBLY, n_gt: int = 25) -> np.ndarray:
    """Seeded guide-tube positions in one n x n assembly (not a published map)."""
    mask = np.zeros(n * n, dtype=bool)
    mask[rng.choice(n * n, size=n_gt, replace=False)] = True
    return mask.reshape(n, n)


def _assemble(ncx, ncy, nl, pin, gt, refl, mat_fuel_layers=None):
    """Fill the per-(cell, layer) material maps from boolean cell masks."""
    has_pin = np.zeros((ncy, ncx), dtype=np.int32)
    mat_in = np.full((ncy, ncx, nl), MAT_MOD, dtype=np.int32)
    mat_out = np.full((ncy, ncx, nl), MAT_MOD, dtype=np.int32)
    has_pin[pin | gt] = 1
    mat_in[pin] = MAT_FUEL
    mat_in[gt] = MAT_GT
    mat_out[refl] = MAT_MOD
    return has_pin, mat_in, mat_out


def pin_cell(seed: int = 1, G: int = 2, homogeneous: bool = False,
             n_azim: int = 8, n_polar: int = 4, radial_spacing: float = 0.1,
             axial_spacing: float = 0.5, height: float = 2.0, n_layers: int = 4,
             bc=(1, 1, 1, 1, 1, 1)) -> Problem:
    """Single square pin cell, pitch 1.26 cm, fuel r = 0.54 cm, 2 groups.

    Sigma_t in 0.3-1.5 /cm, scatter ratio 0.5-0.9, fission only in fuel.
    ``homogeneous`` fills both regions with the fuel material (the infinite
    medium case when every face is reflective).
    """
    rng = np.random.default_rng(seed)
    st, ss, nsf, chi = make_cross_sections(rng, G, ["fuel", "mod"], sigt_range=(0.3, 1.5),
                                           scat_range=(0.5, 0.9), upscatter_groups=0)
    has_pin = np.ones((1, 1), dtype=np.int32)
    mat_in = np.full((1, 1, n_layers), MAT_FUEL, dtype=np.int32)
    mat_out = np.full((1, 1, n_layers), MAT_FUEL if homogeneous else MAT_MOD, dtype=np.int32)
    return Problem("pin_cell" + ("_homog" if homogeneous else ""), 1, 1, PITCH, FUEL_RADIUS,
                   height, n_layers, has_pin.ravel(), mat_in.ravel(), mat_out.ravel(),
                   tuple(bc), st, ss, nsf, chi, None, n_azim, n_polar, radial_spacing,
                   axial_spacing, seed)


def lattice(seed: int = 1, n: int = ASSEMBLY, G: int = 7, height: float = 20.0,
            n_layers: int = 10, n_azim: int = 32, n_polar: int = 4,
            radial_spacing: float = 0.05, axial_spacing: float = 0.5,
            bc=(1, 1, 1, 1, 0, 0), n_gt: Optional[int] = None,
            fixed_source: bool = False, name: Optional[str] = None) -> Problem:
    """n x n pin lattice with seeded guide tubes, 3 materials (fuel, mod, gt).

    With the defaults this is the 17x17 workload: 264 fuel pins, 25 guide
    tubes, 7 groups (Sigma_t 0.2-2.0 /cm, upscatter in the last 3 groups,
    scatter ratio 0.5-0.95), 20 cm high in 10 layers, reflective radially and
    vacuum axially, 32 azimuths x 4 polar angles, 0.05 cm radial and 0.5 cm
    axial spacing.  ``fixed_source`` makes the medium non-multiplying and adds
    a seeded uniform volumetric source in every material.
    """
    rng = np.random.default_rng(seed)
    st, ss, nsf, chi = make_cross_sections(rng, G, ["fuel", "mod", "gt"])
    if n_gt is None:
        n_gt = 25 if n == ASSEMBLY else max(0, (n * n) // 12)
    gt = np.zeros((n, n), dtype=bool)
    if n_gt:
        gt.ravel()[rng.choice(n * n, size=n_gt, replace=False)] = True
    pin = ~gt
    refl = np.zeros_like(gt)
    has_pin, mat_in, mat_out = _assemble(n, n, n_layers, pin, gt, refl)
    ext = None
    if fixed_source:
        nsf = np.zeros_like(nsf)
        ext = np.repeat(rng.uniform(0.5, 1.5, size=(1, G)), st.shape[0], axis=0)
    return Problem(name or f"lattice{n}", n, n, PITCH, FUEL_RADIUS, height, n_layers,
                   has_pin.ravel(), mat_in.ravel(), mat_out.ravel(), tuple(bc), st, ss, nsf,
                   chi, ext, n_azim, n_polar, radial_spacing, axial_spacing, seed)


def assemblies(seed: int = 1, n_asm: int = 3, refl_sides: str = "two", G: int = 7,
               height: float = 64.0, n_layers: int = 32, absorber_height: float = 16.0,
               n_azim: int = 64, n_polar: int = 6, radial_spacing: float = 0.05,
               axial_spacing: float = 0.25, bc=(1, 0, 1, 0, 1, 0)) -> Problem:
    """n_asm x n_asm 17x17 assemblies plus a one-assembly moderator reflector.

    ``refl_sides`` = "two" puts the reflector on the x-max and y-max sides
    (quarter-core style, reflective on x-min, y-min, z-min); "ring" surrounds
    the core on all four sides (full core, use all-vacuum ``bc``).  Seeded
    guide tubes carry an absorber in the top ``absorber_height`` cm.
    Reflector cells are single-region moderator cells at pin pitch.
    """
    rng = np.random.default_rng(seed)
    st, ss, nsf, chi = make_cross_sections(rng, G, ["fuel", "mod", "gt", "abs"])
    a = ASSEMBLY
    if refl_sides == "two":
        off = 0
        ncx = ncy = (n_asm + 1) * a
    elif refl_sides == "ring":
        off = a
        ncx = ncy = (n_asm + 2) * a
    else:
        raise ValueError(refl_sides)
    gt = np.zeros((ncy, ncx), dtype=bool)
    pin = np.zeros((ncy, ncx), dtype=bool)
    for ay in range(n_asm):
        for ax in range(n_asm):
            m = _guide_tube_mask(rng)
            y0, x0 = off + ay * a, off + ax * a
            gt[y0:y0 + a, x0:x0 + a] = m
            pin[y0:y0 + a, x0:x0 + a] = ~m
    refl = ~(gt | pin)
    has_pin, mat_in, mat_out = _assemble(ncx, ncy, n_layers, pin, gt, refl)
    # absorber inserted into the top of a seeded half of the guide tubes
    n_abs_layers = int(round(absorber_height / (height / n_layers)))
    gts = np.argwhere(gt)
    if n_abs_layers > 0 and len(gts):
        pick = gts[rng.random(len(gts)) < 0.5]
        for (y, x) in pick:
            mat_in[y, x, n_layers - n_abs_layers:] = MAT_ABS
    name = f"asm{n_asm}x{n_asm}_{refl_sides}"
    return Problem(name, ncx, ncy, PITCH, FUEL_RADIUS, height, n_layers, has_pin.ravel(),
                   mat_in.ravel(), mat_out.ravel(), tuple(bc), st, ss, nsf, chi, None, n_azim,
                   n_polar, radial_spacing, axial_spacing, seed)


def core_7x7(seed: int = 1) -> Problem:
    """7x7 assemblies with a one-assembly reflector ring, 200 cm in 100 layers,
    128 azimuths x 6 polar, vacuum on all six faces."""
    return assemblies(seed, n_asm=7, refl_sides="ring", height=200.0, n_layers=100,
                      absorber_height=0.0, n_azim=128, n_polar=6, radial_spacing=0.05,
                      axial_spacing=0.5, bc=(0, 0, 0, 0, 0, 0))


def serving_request(seed: int, index: int) -> Problem:
    """One request of the serving stream: an n x n lattice (n ~ U{1..17}),
    2-7 groups, height 2-20 cm in 2 cm layers, 16-64 azimuths x 2-4 polar,
    half eigenvalue and half fixed-source (uniform volumetric source,
    non-multiplying medium).  Radial spacing 0.1 cm, axial 0.5 cm, reflective
    radially and vacuum axially."""
    rng = np.random.default_rng([seed, index])
    n = int(rng.integers(1, 18))
    G = int(rng.integers(2, 8))
    nl = int(rng.integers(1, 11))
    A = int(rng.choice([16, 32, 48, 64]))
    P = int(rng.choice([2, 4]))
    fixed = bool(index % 2)
    p = lattice(seed=int(rng.integers(1, 2**31)), n=n, G=G, height=2.0 * nl, n_layers=nl,
                n_azim=A, n_polar=P, radial_spacing=0.1, axial_spacing=0.5,
                bc=(1, 1, 1, 1, 0, 0), fixed_source=fixed, name=f"req{index}")
    p.meta["arrival_index"] = index
    return p


# ---------------------------------------------------------------------------
# named workloads


def workload(name: str, seed: int = 1) -> Problem:
    """Named workloads.

    * ``pin_cell``   - single pin cell, 2 groups, all reflective, 8 azim x 4 polar
    * ``lattice17``  - 17x17 lattice, 7 groups, 32 azim x 4 polar, the main
                       throughput workload
    * ``lattice17_small`` - the same lattice with a coarse track layout for
                       fast parity runs
    * ``lattice5_rings`` - 5x5 lattice with 3 fuel rings, 1 moderator ring
                       and 8 sectors per pin cell
    * ``pin_cell_rings`` - the pin cell with 3 fuel rings, 2 moderator rings
                       and 4 sectors
    * ``lattice5_axial`` - lattice5 with unequal layers (0.5, 1, 1.5, 1 cm)
    * ``lattice5_offaxial`` - lattice5 with layer planes off the axial lattice
                       (0.7, 1.85, 3.15 cm)
    * ``asm1_absorber`` - one assembly + reflector on two sides, 8 cm, absorber
                       in the top layer of half the guide tubes
    * ``asm3x3``     - 3x3 assemblies + reflector on two sides, 64 cm
    * ``core7x7``    - 7x7 assemblies + reflector ring, 200 cm
    """
    if name == "pin_cell":
        return pin_cell(seed)
    if name == "pin_cell_homog":
        return pin_cell(seed, homogeneous=True)
    if name == "lattice17":
        return lattice(seed)
    if name == "lattice17_small":
        return lattice(seed, n_azim=8, n_polar=4, radial_spacing=0.4, axial_spacing=1.0,
                       height=8.0, n_layers=4, name="lattice17_small")
    if name == "lattice5":
        return lattice(seed, n=5, n_azim=16, n_polar=4, radial_spacing=0.1,
                       axial_spacing=0.5, height=4.0, n_layers=4, name="lattice5")
    if name == "lattice5_rings":
        # finer FSRs: 3 fuel rings, 1 moderator ring, 8 sectors (40 regions a pin)
        return replace(lattice(seed, n=5, n_azim=16, n_polar=4, radial_spacing=0.1,
                               axial_spacing=0.5, height=4.0, n_layers=4, name="lattice5_rings"),
                       fuel_rings=3, moderator_rings=1, sectors=8)
    if name == "lattice5_axial":
        # unequal layers on the 0.5 cm axial lattice: 0.5, 1.0, 1.5 and 1.0 cm
        return replace(lattice(seed, n=5, n_azim=16, n_polar=4, radial_spacing=0.1,
                               axial_spacing=0.5, height=4.0, n_layers=4, name="lattice5_axial"),
                       layer_z=np.array([0.0, 0.5, 1.5, 3.0, 4.0]))
    if name == "lattice5_offaxial":
        # layer planes off the 0.5 cm axial lattice (Sec. 2.2's local axial
        # mesh): 0.7, 1.85 and 3.15 cm, 0.4, 0.7 and 0.3 of a spacing above
        # a lattice plane
        return replace(lattice(seed, n=5, n_azim=16, n_polar=4, radial_spacing=0.1,
                               axial_spacing=0.5, height=4.0, n_layers=4, name="lattice5_offaxial"),
                       layer_z=np.array([0.0, 0.7, 1.85, 3.15, 4.0]))
    if name == "pin_cell_rings":
        return replace(pin_cell(seed), name="pin_cell_rings", fuel_rings=3, moderator_rings=2,
                       sectors=4)
    if name == "asm1_absorber":
        # one assembly, reflector on two sides, absorber in the top layer of a
        # seeded half of the guide tubes (a small reflected, axially varying case)
        return assemblies(seed=2 if seed == 1 else seed, n_asm=1, height=8.0, n_layers=4,
                          absorber_height=2.0, n_azim=8, n_polar=4, radial_spacing=0.1,
                          axial_spacing=0.5)
    if name == "asm3x3":
        return assemblies(seed)
    if name == "core7x7":
        return core_7x7(seed)
    raise KeyError(name)
