"""Pins of the MTS Arlequin oracle against what the method fixes (CPU only)."""
import numpy as np
import pytest

from oracle.mts import MTSOracle, band_weight, monolithic_step
from paper_2403_03605_gb300 import workloads as W


def test_weights_partition_the_mass():
    """alpha weights FE mass, 1 - alpha PD mass (Eq. 17, Eq. 34): with linear
    weights and cell-centred PD nodes the two add up to the plate's mass."""
    cp = W.small_coupled()
    o = MTSOracle(cp)
    total = ((1 - o.alpha) * cp.pd.mat.rho * cp.pd.vol).sum() + o.fe.M[:o.nfe].sum()
    assert abs(total / (cp.pd.mat.rho * 0.02 * 0.01 * cp.pd.mat.thickness) - 1) < 1e-12
    # weights: 1 on the FE side of a band, 0 on the PD side, linear in between
    b = cp.bands[0]
    y = np.array([[0.0, 0.0, 0.0], [b.lo, 0.5 * (b.lo + b.hi), b.hi]])
    np.testing.assert_allclose(band_weight(y, cp.bands, 1, 0.0), [1.0, 0.5, 0.0])
    np.testing.assert_allclose(band_weight(y, cp.bands, 2, 0.0), [1.0, 0.125, 0.0])


def test_m1_equals_monolithic_single_step_scheme():
    """With m = 1 the MTS algorithm is the single-step coupled scheme of Eq. 33
    (Sec. 2.5): one KKT solve per step for (a_FE, a_PD, lambda)."""
    cp = W.small_coupled(m=1, crack=False)
    o = MTSOracle(cp, breaking=False)
    ref = MTSOracle(cp, breaking=False)
    state = (ref.uf.copy(), ref.vf.copy(), ref.af.copy(), ref.u.copy(), ref.v.copy(), ref.a.copy())
    for _ in range(6):
        lam = o.coarse_step()
        state, lam_ref = monolithic_step(ref, state)
        uf, vf, af, u, v, a = state
        scale = np.abs(uf).max()
        assert np.abs(o.uf - uf).max() <= 1e-10 * scale
        assert np.abs(o.u - u).max() <= 1e-10 * max(np.abs(u).max(), 1e-30) + 1e-12 * scale
        assert np.abs(lam - lam_ref).max() <= 1e-9 * np.abs(lam_ref).max()


def test_uniform_velocity_patch():
    """A uniform velocity with no load stays uniform in both subdomains for any
    m, and the multiplier stays zero (G_FE v = G_PD v exactly for constant v)."""
    cp = W.small_coupled(m=5, crack=False, traction=0.0)
    v0 = np.array([3.0, -1.5])
    o = MTSOracle(cp, v0=v0)
    for _ in range(4):
        lam = o.coarse_step()
    t = 4 * cp.m * cp.dt_pd
    assert np.abs(o.v - v0.reshape(2, 1)).max() <= 1e-12 * np.abs(v0).max()
    assert np.abs(o.vf - np.repeat(v0, o.nfe)).max() <= 1e-12 * np.abs(v0).max()
    np.testing.assert_allclose(o.u, v0.reshape(2, 1) * t * np.ones((1, o.npd)), rtol=1e-12)
    force_scale = cp.pd.mat.rho * np.abs(v0).max() / (cp.m * cp.dt_pd)
    assert np.abs(lam).max() <= 1e-9 * force_scale


def test_constraint_residual_and_interface_operator_symmetry():
    """After every coarse step G_FE v_FE = G_PD v_PD to rounding (Eq. 41); the
    interface operator of Eq. 49 is symmetric (linear responses are reciprocal)."""
    cp = W.small_coupled(m=4, n_coarse=8)
    o = MTSOracle(cp).advance(8)
    assert max(o.residuals) <= 1e-12
    H = o.H
    assert np.abs(H - H.T).max() <= 1e-10 * np.abs(H).max()
    assert np.all(np.linalg.eigvalsh(0.5 * (H + H.T)) < 0)  # negative definite


def test_rebuild_rule_matches_rebuilding_every_step():
    """Rebuilding the unit responses only after a break within (m + 1) delta of an
    overlap band gives the same result as rebuilding after every step."""
    cp = W.small_coupled(m=4, n_coarse=12, traction=30e6)
    a = MTSOracle(cp, rebuild="auto").advance(12)
    b = MTSOracle(cp, rebuild="always").advance(12)
    assert (b.mu != 1).sum() > (a.mu != 1).sum() - 1 and (a.mu == 0).sum() > 0
    assert np.array_equal(a.u, b.u) and np.array_equal(a.uf, b.uf) and np.array_equal(a.mu, b.mu)
    assert a.n_rebuilds < b.n_rebuilds


def test_3d_coupling_constraint_operator_and_patch():
    """3D (Hex8 FE, bond-based PD through the thickness): the velocity constraint
    holds after every coarse step, the interface operator is symmetric negative
    definite, and a uniform velocity field stays uniform with lambda = 0."""
    cp = W.small_coupled3d(m=3, n_coarse=3)
    o = MTSOracle(cp).advance(3)
    assert max(o.residuals) <= 1e-12
    H = o.H
    assert np.abs(H - H.T).max() <= 1e-12 * np.abs(H).max()
    assert np.linalg.eigvalsh(0.5 * (H + H.T)).max() < 0
    v0 = np.array([1.0, -2.0, 0.5])
    cp2 = W.small_coupled3d(m=2, n_coarse=2, crack=False, traction=0.0)
    o2 = MTSOracle(cp2, v0=v0).advance(2)
    assert np.abs(o2.v - v0.reshape(3, 1)).max() <= 1e-12 * 2.0
    assert np.abs(o2.vf - np.repeat(v0, o2.nfe)).max() <= 1e-12 * 2.0
    force_scale = cp2.pd.mat.rho * 2.0 / (cp2.m * cp2.dt_pd)
    assert np.abs(o2.lam).max() <= 1e-9 * force_scale


def test_hex8_stiffness_rigid_modes_and_volume():
    """The Hex8 element stiffness has exactly the six rigid-body modes as its
    null space, and the lumped mass sums to rho times the volume."""
    from oracle.mts import FE
    X, conn = W.hex8_block(0.0, 0.0, 0.0, 1, 1, 1, 2e-3)
    mesh = W.FEMesh(X, conn, 2e-3)
    fe = FE(mesh, 72e9, 0.25, 2440.0, 1.0, [], 1, np.zeros((0, 4), np.int32), np.zeros((0, 3)))
    K = fe.K.toarray()
    ev = np.linalg.eigvalsh(K)
    assert np.sum(np.abs(ev) <= 1e-9 * ev.max()) == 6
    assert abs(fe.M.sum() / 3 - 2440.0 * (2e-3) ** 3) <= 1e-12 * 2440.0 * (2e-3) ** 3
