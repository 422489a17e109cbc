"""Crack-tip reading and accuracy figures (CPU).

The paper does not define a crack tip. The reading used: the extreme
coordinates along the crack direction of the nodes with damage (Eq. 5) of at
least 0.35 within a band around the crack plane. The oracle's plain loop is
pinned on hand-made damage fields whose answer is read off by eye; the
library's host-side numpy version must agree with it on random fields.
"""
import math

import numpy as np

import oracle
from paper_2403_03605_gb300 import diagnostics as D
from paper_2403_03605_gb300 import workloads as W


def _grid(nx, ny, dx=1.0):
    lat = W.Lattice((nx, ny), dx, (0.0, 0.0))
    return lat, lat.X


def test_oracle_crack_tip_hand_field():
    lat, X = _grid(10, 6)
    phi = np.zeros(lat.n)
    idx = lat.idx
    # a damaged row at y = 2.5 (iy = 2) from ix = 3 to ix = 7, and a damaged
    # node far from the plane (iy = 5, ix = 9) that the band must exclude
    phi[(idx[1] == 2) & (idx[0] >= 3) & (idx[0] <= 7)] = 0.5
    phi[(idx[1] == 5) & (idx[0] == 9)] = 1.0
    # below the threshold: ignored
    phi[(idx[1] == 3) & (idx[0] == 8)] = 0.34
    lo, hi = oracle.crack_tip(X, phi, normal=1, level=2.5, along=0, band=1.0)
    assert (lo, hi) == (3.5, 7.5)
    # a band that reaches iy = 5 picks up x = 9.5
    assert oracle.crack_tip(X, phi, 1, 2.5, 0, 3.0) == (3.5, 9.5)
    # exactly at the threshold counts (phi >= 0.35)
    phi[(idx[1] == 3) & (idx[0] == 8)] = 0.35
    assert oracle.crack_tip(X, phi, 1, 2.5, 0, 1.0) == (3.5, 8.5)
    # no damaged node: nan
    lo, hi = oracle.crack_tip(X, np.zeros(lat.n), 1, 2.5, 0, 1.0)
    assert math.isnan(lo) and math.isnan(hi)
    # the crack plane normal to x, the tip along y
    phi2 = np.zeros(lat.n)
    phi2[(idx[0] == 4) & (idx[1] <= 3)] = 0.6
    assert oracle.crack_tip(X, phi2, 0, 4.5, 1, 0.5) == (0.5, 3.5)


def test_library_crack_tip_matches_oracle():
    rng = np.random.default_rng(11)
    lat, X = _grid(37, 23, dx=0.25e-3)
    for _ in range(20):
        phi = rng.random(lat.n) * rng.random()
        level = rng.uniform(0, 23 * 0.25e-3)
        band = rng.uniform(0, 3e-3)
        for normal, along in ((1, 0), (0, 1)):
            a = oracle.crack_tip(X, phi, normal, level, along, band)
            b = D.crack_tip(X, phi, normal, level, along, band)
            assert (math.isnan(a[0]) and math.isnan(b[0])) or a == b


def test_tip_error_and_mismatch():
    assert D.tip_error((0.0, 0.02), (0.0, 0.021)) == 0.0010000000000000009
    assert D.tip_error((float("nan"),) * 2, (float("nan"),) * 2) == 0.0
    assert D.tip_error((float("nan"),) * 2, (0.0, 1.0)) == float("inf")
    mu_ref = np.array([1, 0, 0, 1, 1, 0, 1, 1], np.uint8)
    mu = np.array([1, 0, 1, 1, 0, 0, 1, 1], np.uint8)
    frac, of_broken = D.bond_mismatch(mu, mu_ref)
    assert frac == 2 / 8 and of_broken == 2 / 3


def test_precracked_plate_tip_at_cut_end():
    # damage of a plate whose only broken bonds are an edge pre-crack on the
    # plane y = 10 mm for 0 <= x < 12 mm: the rows next to the cut lose 11 of
    # their 28 bonds, the next rows 6, so the tip lies within one horizon of
    # the cut's end (nodes near the end lose only part of their crossing bonds)
    pb = W.plate2d(40, 40, 0.5e-3, cuts_mm=[(1, 10e-3, 0, 0.0, 12e-3)], nsteps=0)
    rp, col = oracle.family(pb.lat.X, pb.delta)
    mu, ncut = oracle.precrack(pb.lat.P, rp, col, [c.in_half_units(pb.lat) for c in pb.cuts])
    opd = oracle.PD(pb.lat.X, pb.vol, pb.delta, pb.c, pb.s0, pb.mat.rho, pb.dt)
    phi = oracle.damage(opd, rp, col, mu)
    lo, hi = oracle.crack_tip(pb.lat.X, phi, 1, 10e-3, 0, 2 * pb.delta)
    assert ncut > 0
    idx = pb.lat.idx
    assert np.allclose(phi[(idx[1] == 19) & (idx[0] >= 3) & (idx[0] < 20)], 11 / 28, rtol=0, atol=1e-15)
    assert np.allclose(phi[(idx[1] == 18) & (idx[0] >= 3) & (idx[0] < 20)], 6 / 28, rtol=0, atol=1e-15)
    assert lo == 0.25e-3
    assert 12e-3 - pb.delta <= hi <= 12e-3 + pb.delta
