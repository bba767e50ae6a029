"""Element-by-element comparison of GPU tallies and fluxes with the FP64
oracle's (test helper).

* check_tally: every FSR-group tally whose magnitude is at least
  floor_frac x the largest is within `rel` of the oracle's, relatively; the
  others within abs_frac x the largest, absolutely (a tally is a sum of
  attenuated differences and can cancel to near zero, where only an
  absolute bar means anything); the worst relative error below the floor
  is returned for the record.
* check_flux: the scalar flux a sweep's tallies give (Eq. 4,
  phi = (4 pi Q + tally / V) / Sigma_t, the oracle's volumes for both) within
  `rel` of the oracle's on every FSR-group, with no floor.
* shaped_source: a seeded source peaked at the centre of the core and falling
  to `floor` of the peak at its edges, like the flux of a bare core, so that
  regions of very different flux share one 2D track.
"""
import math

import numpy as np

from tests import bruteforce as bf


def tally_stats(gt, ot, floor_frac=1e-3):
    gt = np.asarray(gt)
    ot = np.asarray(ot)
    scale = np.abs(ot).max()
    err = np.abs(gt - ot)
    big = np.abs(ot) >= floor_frac * scale
    rel_big = (err[big] / np.abs(ot[big])).max() if big.any() else 0.0
    small = ~big
    rel_small = (err[small] / np.maximum(np.abs(ot[small]), 1e-300)).max() if small.any() else 0.0
    stats = {"max_rel_above_floor": float(rel_big), "n_above_floor": int(big.sum()),
             "max_rel_below_floor": float(rel_small), "n_below_floor": int(small.sum()),
             "max_abs_over_scale": float(err.max() / scale) if scale > 0 else 0.0}
    # the worst relative error by magnitude decade of the oracle's tally
    for d in (1e-1, 1e-2, 1e-3, 1e-4):
        m = (np.abs(ot) >= d * scale) & (np.abs(ot) < 10 * d * scale)
        if m.any():
            stats[f"rel_{d:g}"] = float((err[m] / np.abs(ot[m])).max())
    return stats, scale, err


def check_tally(gt, ot, rel=1e-4, floor_frac=1e-3, abs_frac=2e-5, what=""):
    stats, scale, err = tally_stats(gt, ot, floor_frac)
    stats["what"] = what
    print("tally parity", stats)
    assert scale > 0, what
    assert stats["max_rel_above_floor"] <= rel, stats
    assert err.max() <= abs_frac * scale, stats
    return stats


def check_flux(gt, ot, Q, vol, sigt_fsr, rel=1e-4, what=""):
    V = np.asarray(vol)[:, None]
    phi_o = (4 * math.pi * Q + ot / V) / sigt_fsr
    phi_g = (4 * math.pi * Q + gt / V) / sigt_fsr
    assert np.all(phi_o > 0), what
    r = np.abs(phi_g / phi_o - 1).max()
    print("flux parity", what, float(r))
    assert r <= rel, (what, float(r))
    return float(r)


def shaped_source(prob, G, seed, floor=1e-3):
    x, y, z = bf.fsr_centres(prob)
    W, H = prob.ncx * prob.pitch, prob.height
    shape = (np.cos(math.pi * (x / W - 0.5)) * np.cos(math.pi * (y / (prob.ncy * prob.pitch) - 0.5))
             * np.cos(math.pi * (z / H - 0.5)))
    shape = floor + (1 - floor) * np.clip(shape, 0, None) ** 2
    rng = np.random.default_rng(seed)
    return shape[:, None] * rng.uniform(0.5, 1.0, size=(x.size, G))
