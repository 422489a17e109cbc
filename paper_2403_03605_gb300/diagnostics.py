"""Accuracy figures of a run read back from the library (host-side, numpy).

These summarise a result against another run of the same problem (typically
the FP32-bulk path against the FP64 path): displacement rel-L2, the fraction
of directed bonds whose status differs, and the crack-tip position error.
They operate on arrays already copied to the host and are not part of the
substep path.
"""
from __future__ import annotations

import numpy as np


def rel_l2(a, ref) -> float:
    """||a - ref|| / ||ref|| (the absolute norm when ref is zero)."""
    a = np.asarray(a, dtype=np.float64).ravel()
    ref = np.asarray(ref, dtype=np.float64).ravel()
    den = float(np.linalg.norm(ref))
    num = float(np.linalg.norm(a - ref))
    return num / den if den > 0 else num


def crack_tip(X, phi, normal: int, level: float, along: int, band: float, threshold: float = 0.35):
    """(lo, hi): the extreme coordinates along `along` of the nodes with damage
    >= threshold within `band` of the crack plane x[normal] = level; (nan, nan)
    if there are none. The paper gives no crack-tip definition; this is the
    reading used for the crack-tip error. A node next to a fully separated
    lattice plane (delta = 3.015 dx) has lost 11 of 28 bonds in 2D and 47 of
    122 in 3D, the next row 6 of 28: the default threshold lies between."""
    X = np.asarray(X, dtype=np.float64)
    phi = np.asarray(phi, dtype=np.float64)
    sel = (phi >= threshold) & (np.abs(X[normal] - level) <= band)
    if not np.any(sel):
        return float("nan"), float("nan")
    xs = X[along][sel]
    return float(xs.min()), float(xs.max())


def tip_error(tip, tip_ref) -> float:
    """Largest difference of the two crack-tip extremes [m] (nan-safe: 0 when
    both runs have no damaged node in the band, inf when only one has)."""
    err = 0.0
    for a, b in zip(tip, tip_ref):
        if np.isnan(a) and np.isnan(b):
            continue
        if np.isnan(a) or np.isnan(b):
            return float("inf")
        err = max(err, abs(a - b))
    return err


def bond_mismatch(mu, mu_ref):
    """(fraction of directed bonds whose status differs, the same count over
    the bonds broken in the reference run)."""
    mu = np.asarray(mu)
    mu_ref = np.asarray(mu_ref)
    diff = int(np.count_nonzero(mu != mu_ref))
    broken = int(np.count_nonzero(mu_ref == 0))
    return diff / max(len(mu_ref), 1), (diff / broken if broken else 0.0)


def compare(run, ref, X, crack, band):
    """Accuracy of `run` against `ref`; each is a dict with u (PD displacement),
    mu (bond status), phi (damage) and optionally uf (FE displacement). crack
    = (normal, level, along) of the crack plane."""
    normal, level, along = crack
    tip = crack_tip(X, run["phi"], normal, level, along, band)
    tip_ref = crack_tip(X, ref["phi"], normal, level, along, band)
    mm, mm_broken = bond_mismatch(run["mu"], ref["mu"])
    out = {"u_pd_rel_l2": rel_l2(run["u"], ref["u"]), "broken_mismatch_frac": mm,
           "broken_mismatch_of_broken": mm_broken, "n_broken_ref": int(np.count_nonzero(ref["mu"] == 0)),
           "n_broken": int(np.count_nonzero(run["mu"] == 0)),
           "crack_tip_m": tip[1], "crack_tip_ref_m": tip_ref[1], "crack_tip_error_m": tip_error(tip, tip_ref)}
    if "uf" in run and "uf" in ref:
        out["u_fe_rel_l2"] = rel_l2(run["uf"], ref["uf"])
    return out
