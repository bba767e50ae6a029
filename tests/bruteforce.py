"""Brute-force geometry used to pin the oracle (test helper, pure numpy).

Nothing here follows the oracle's or the GPU library's algorithms: it samples
points densely along a ray and classifies each point by direct point location
in the pin lattice, then run-length encodes the region sequence.
"""
from __future__ import annotations

import math

import numpy as np


def circle_radii2(prob):
    """Squared radii of a pin cell's circles, from the problem's conventions:
    equal-area rings of the fuel circle, then equal steps of r^2 from the fuel
    radius towards half the pitch (half the pitch itself excluded)."""
    F = max(1, getattr(prob, "fuel_rings", 1))
    Mr = getattr(prob, "moderator_rings", 0)
    rf2, rh2 = prob.fuel_radius ** 2, (0.5 * prob.pitch) ** 2
    return np.array([rf2 * k / F for k in range(1, F + 1)] +
                    [rf2 + (rh2 - rf2) * k / (Mr + 1) for k in range(1, Mr + 1)])


def region_ids(prob, x, y):
    """Radial region of points (x, y) by direct point location: cell by cell;
    in a pin cell, ring (number of circles the point lies outside) times the
    sector count plus the sector (angle about the centre from +x)."""
    r2 = circle_radii2(prob)
    S = max(1, getattr(prob, "sectors", 1))
    cx = np.clip(np.floor(x / prob.pitch).astype(np.int64), 0, prob.ncx - 1)
    cy = np.clip(np.floor(y / prob.pitch).astype(np.int64), 0, prob.ncy - 1)
    c = cy * prob.ncx + cx
    nreg = np.where(prob.has_pin != 0, (len(r2) + 1) * S, 1)
    base = np.concatenate([[0], np.cumsum(nreg)[:-1]])
    ux = x - (cx + 0.5) * prob.pitch
    uy = y - (cy + 0.5) * prob.pitch
    d2 = ux ** 2 + uy ** 2
    ring = np.sum(d2[..., None] >= r2, axis=-1)
    ang = np.mod(np.arctan2(uy, ux), 2 * math.pi)
    sec = np.minimum(S - 1, np.floor(ang * S / (2 * math.pi)).astype(np.int64))
    pin = prob.has_pin[c] != 0
    return np.where(pin, base[c] + ring * S + sec, base[c])


def laydown(prob, m):
    """Closed-form cyclic laydown of first-quadrant azimuth m."""
    W_x = prob.ncx * prob.pitch
    W_y = prob.ncy * prob.pitch
    phi = 2 * math.pi * (m + 0.5) / prob.n_azim
    nx = math.ceil(W_x * abs(math.sin(phi)) / prob.radial_spacing)
    ny = math.ceil(W_y * abs(math.cos(phi)) / prob.radial_spacing)
    phi_eff = math.atan2(W_y * nx, W_x * ny)
    return dict(nx=nx, ny=ny, phi_eff=phi_eff, W_x=W_x, W_y=W_y,
                delta_eff=(W_x / nx) * math.sin(phi_eff))


def track_start_dir(prob, tr):
    """Start point and unit direction of a 2D track from its face/index."""
    A = prob.n_azim
    a = tr["azim"]
    nq = A // 4
    m = a if a < nq else A // 2 - 1 - a
    ld = laydown(prob, m)
    nx, ny, W_x, W_y = ld["nx"], ld["ny"], ld["W_x"], ld["W_y"]
    k = tr["sk"]
    face = tr["sface"]
    if face == 2:      # ymin
        x0, y0 = (k + 0.5) * W_x / nx, 0.0
    elif face == 0:    # xmin
        x0, y0 = 0.0, (k + 0.5) * W_y / ny
    else:              # xmax
        x0, y0 = W_x, (k + 0.5) * W_y / ny
    phi = ld["phi_eff"] if a < nq else math.pi - ld["phi_eff"]
    return x0, y0, math.cos(phi), math.sin(phi), ld


def exit_length(prob, x0, y0, dx, dy):
    W_x = prob.ncx * prob.pitch
    W_y = prob.ncy * prob.pitch
    ts = []
    if dx > 0:
        ts.append((W_x - x0) / dx)
    if dx < 0:
        ts.append(-x0 / dx)
    if dy > 0:
        ts.append((W_y - y0) / dy)
    return min(ts)


def rle(ids, step):
    """Run-length encode a sampled id sequence: (ids, lengths)."""
    ids = np.asarray(ids)
    if ids.size == 0:
        return np.zeros(0, dtype=np.int64), np.zeros(0)
    change = np.flatnonzero(np.diff(ids)) + 1
    starts = np.concatenate([[0], change])
    ends = np.concatenate([change, [ids.size]])
    return ids[starts], (ends - starts) * step


def drop_short(ids, lens, min_len):
    """Remove runs shorter than min_len and merge equal neighbours."""
    keep = lens >= min_len
    ids, lens = ids[keep], lens[keep]
    if ids.size == 0:
        return ids, lens
    out_i, out_l = [ids[0]], [lens[0]]
    for i, l in zip(ids[1:], lens[1:]):
        if i == out_i[-1]:
            out_l[-1] += l
        else:
            out_i.append(i)
            out_l.append(l)
    return np.array(out_i), np.array(out_l)


def ray_regions(prob, x0, y0, dx, dy, L, n_samples=200000):
    h = L / n_samples
    s = (np.arange(n_samples) + 0.5) * h
    ids = region_ids(prob, x0 + s * dx, y0 + s * dy)
    return rle(ids, h) + (h,)


def ray_fsrs_3d(prob, x0, y0, dx, dy, L, z_start, cot, n_samples=200000):
    """FSR sequence and 3D lengths of the 3D line z(s) = z_start + s cot over the
    2D track, sampled densely, keeping only the part inside 0 < z < H."""
    h = L / n_samples
    s = (np.arange(n_samples) + 0.5) * h
    z = z_start + s * cot
    inside = (z > 0) & (z < prob.height)
    s, z = s[inside], z[inside]
    reg = region_ids(prob, x0 + s * dx, y0 + s * dy)
    lz = getattr(prob, "layer_z", None)
    if lz is None:
        layer = np.floor(z / (prob.height / prob.n_layers)).astype(np.int64)
    else:
        layer = np.searchsorted(np.asarray(lz), z, side="right") - 1
    fsr = reg * prob.n_layers + layer
    sin = 1.0 / math.sqrt(1.0 + cot * cot)
    ids, lens = rle(fsr, h / sin)
    return ids, lens, h / sin


def layer_of(prob, z):
    """Axial layer of heights z (equal layers, or the listed planes)."""
    lz = getattr(prob, "layer_z", None)
    if lz is None:
        return np.minimum(prob.n_layers - 1,
                          np.floor(z / (prob.height / prob.n_layers)).astype(np.int64))
    return np.minimum(prob.n_layers - 1, np.searchsorted(np.asarray(lz), z, side="right") - 1)


def point_material(prob, x, y, z):
    """Material at points (x, y, z) by direct location, without any region
    numbering: the cell's mat_in inside its pin's fuel circle (radius
    fuel_radius about the cell centre), mat_out elsewhere in the cell; the
    layer from z."""
    cx = np.clip(np.floor(x / prob.pitch).astype(np.int64), 0, prob.ncx - 1)
    cy = np.clip(np.floor(y / prob.pitch).astype(np.int64), 0, prob.ncy - 1)
    c = cy * prob.ncx + cx
    L = layer_of(prob, z)
    ux = x - (cx + 0.5) * prob.pitch
    uy = y - (cy + 0.5) * prob.pitch
    inside = (prob.has_pin[c] != 0) & (ux ** 2 + uy ** 2 < prob.fuel_radius ** 2)
    mi = np.asarray(prob.mat_in)[c * prob.n_layers + L]
    mo = np.asarray(prob.mat_out)[c * prob.n_layers + L]
    return np.where(inside, mi, mo)


def fsr_materials(prob):
    """Material of every FSR from the documented numbering alone: radial
    regions cell by cell, a pin cell's region = ring * sectors + sector with
    the rings inside the fuel circle (the first fuel_rings) holding mat_in and
    the others mat_out; FSR = region * n_layers + layer."""
    F = max(1, getattr(prob, "fuel_rings", 1))
    S = max(1, getattr(prob, "sectors", 1))
    rings = F + getattr(prob, "moderator_rings", 0) + 1
    NL = prob.n_layers
    out = []
    for c in range(prob.ncx * prob.ncy):
        mi = np.asarray(prob.mat_in)[c * NL:(c + 1) * NL]
        mo = np.asarray(prob.mat_out)[c * NL:(c + 1) * NL]
        if prob.has_pin[c]:
            for ring in range(rings):
                for _ in range(S):
                    out.append(mi if ring < F else mo)
        else:
            out.append(mo)
    return np.concatenate(out).astype(np.int32)


def fsr_centres(prob):
    """(x, y, z) of the centre of every FSR's cell and layer, from the
    documented numbering (regions cell by cell, FSR = region * n_layers +
    layer)."""
    R = prob.pin_regions
    NL = prob.n_layers
    cells = np.concatenate([np.full(R if prob.has_pin[c] else 1, c)
                            for c in range(prob.ncx * prob.ncy)])
    cx = (cells % prob.ncx + 0.5) * prob.pitch
    cy = (cells // prob.ncx + 0.5) * prob.pitch
    lz = getattr(prob, "layer_z", None)
    planes = np.asarray(lz) if lz is not None else np.linspace(0.0, prob.height, NL + 1)
    zc = 0.5 * (planes[:-1] + planes[1:])
    x = np.repeat(cx, NL)
    y = np.repeat(cy, NL)
    z = np.tile(zc, cells.size)
    return x, y, z
