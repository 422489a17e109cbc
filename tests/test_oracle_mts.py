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


# ---------------------------------------------------------------------------
# Dirichlet elimination and the undecomposed FE reference (Sec. 3.2, Table 1)
# ---------------------------------------------------------------------------
def _modal_newmark(fp, n_steps):
    """Closed-form Newmark response of the fixed-end beam started at rest
    under a constant load, mode by mode: with mass-normalised modes of
    (K_ff, M_ff), each modal coordinate is q_s (1 - cos(n theta)) with
    q_s = phi' P / omega^2 and tan(theta / 2) = omega dt / 2 for the average
    acceleration scheme (beta = 1/4, gamma = 1/2), cos(theta) = 1 - (omega
    dt)^2 / 2 for the explicit one (beta = 0, lumped mass)."""
    import scipy.linalg as sla
    from oracle.mts import FE
    mat = fp.mat
    fe = FE(fp.mesh, mat.E, mat.nu, mat.rho, mat.thickness, [], 0, fp.faces, fp.face_traction)
    nd = 3 * fe.n
    free = np.setdiff1d(np.arange(nd), fp.fixed)
    K = fe.K.toarray()[np.ix_(free, free)]
    w2, phi = sla.eigh(K, np.diag(fe.M[free]))
    om = np.sqrt(w2)
    qs = phi.T @ fe.P[free] / w2
    if fp.beta == 0.25:
        th = 2.0 * np.arctan(om * fp.dt / 2.0)
    else:
        assert fp.beta == 0.0 and np.all(om * fp.dt < 2.0)
        th = np.arccos(1.0 - (om * fp.dt) ** 2 / 2.0)
    n = np.arange(1, n_steps + 1)[:, None]
    out = np.zeros((n_steps, nd))
    out[:, free] = (qs * (1.0 - np.cos(n * th))) @ phi.T
    return out


@pytest.mark.parametrize("beta", [0.25, 0.0])
def test_fixed_end_newmark_matches_modal_closed_form(beta):
    from oracle.mts import newmark_fe
    fp = W.beam3d_fe(dx=0.25, n_steps=60, beta=beta, length=1.5, width=0.5)
    nd = 3 * fp.mesh.n
    got = newmark_fe(fp, fp.n_steps, np.arange(nd))
    ref = _modal_newmark(fp, fp.n_steps)
    assert np.all(got[:, fp.fixed] == 0.0)
    assert np.abs(got - ref).max() <= 1e-9 * np.abs(ref).max()
    # the tip moves: a dropped load or a wrongly fixed face would not
    assert np.abs(got[:, fp.record["A"]]).max() > 1e-4


def test_fixed_end_static_bar_is_exact_for_zero_poisson():
    """With nu = 0 the clamped end exerts no lateral constraint and the static
    solution of the fixed-end bar under an end traction is u_x = P x / E,
    which trilinear elements reproduce exactly."""
    from oracle.mts import FE
    mat = W.Material(E=6.5e9, nu=0.0, rho=2235.0, G0=0.0, thickness=1.0)
    fp = W.beam3d_fe(dx=0.25, length=1.5, width=0.5, mat=mat)
    fe = FE(fp.mesh, mat.E, mat.nu, mat.rho, mat.thickness, [], 0, fp.faces, fp.face_traction)
    nd = 3 * fe.n
    free = np.setdiff1d(np.arange(nd), fp.fixed)
    u = np.zeros(nd)
    u[free] = np.linalg.solve(fe.K.toarray()[np.ix_(free, free)], fe.P[free])
    x = fp.mesh.X[0]
    np.testing.assert_allclose(u[:fe.n], W.BEAM_TRACTION * x / mat.E, rtol=0, atol=1e-12 * W.BEAM_TRACTION / mat.E)
    assert np.abs(u[fe.n:]).max() <= 1e-12 * W.BEAM_TRACTION / mat.E
    # total load = traction x end area
    assert abs(fe.P[:fe.n].sum() - W.BEAM_TRACTION * 0.25) < 1e-6


def test_exp_micromodulus_constant_matches_quadrature():
    """c0 of the exponential micromodulus against a numerical quadrature of
    its defining integral (Sec. 3.2)."""
    from scipy.integrate import quad
    delta = 3.03 * 0.1
    ell = delta / 16
    integral, _ = quad(lambda r: r ** 6 * np.exp(-r / ell), 0.0, delta, epsabs=0, epsrel=1e-13, limit=200)
    c0 = W.exp_micromodulus_c0(6.5e9, delta, ell)
    assert abs(c0 - 3 * 6.5e9 / (np.pi * integral)) <= 1e-10 * c0


def test_coupled_beam_oracle_tracks_the_fe_reference():
    """The coupled beam follows the undecomposed FE beam at point A within a
    few percent over one round trip of the axial wave (480 coarse steps, a
    coarse 0.25 m mesh, m = 2), and cubic weights over 3 dx beat constant
    weights over dx, the ordering of Table 1."""
    from oracle.mts import newmark_fe
    n = 480
    fp = W.beam3d_fe(dx=0.25, n_steps=n)
    ref = newmark_fe(fp, n, np.array([fp.record["A"]]))[:, 0]
    errs = {}
    for kind, cells in [(0, 1), (2, 3)]:
        cp = W.beam3d(dx=0.25, overlap_cells=cells, weight_kind=kind, m=2, n_coarse=n)
        orc = MTSOracle(cp, breaking=False)
        ia = cp.pd.extra["record"]["A"]
        got = np.zeros(n)
        for k in range(n):
            orc.coarse_step()
            got[k] = orc.uf[ia]
        assert np.all(orc.uf[cp.fixed] == 0.0)
        errs[kind] = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert max(errs.values()) < 0.05, errs
    assert errs[2] < errs[0], errs


def test_free_and_link_runs_superpose_to_the_interpolated_multiplier():
    """With breaking off the PD and FE subdomains are linear, so the split of
    a coarse step into a free run and a link run (Eq. 47-48, U = V + Y lambda_m)
    must equal one direct run under the full interface load: on the PD side m
    substeps whose multiplier is interpolated linearly between lambda_0 and
    lambda_m (Eq. 42, the free run's (1 - j/m) lambda_0 plus the link run's
    (j/m) lambda_m); on the FE side one Newmark step under -G_FE^T lambda_m.
    For m > 1 this pins the free run's lambda_0 term, which vanishes at
    m = 1 and so escapes the monolithic m = 1 pin."""
    from oracle import pd_run
    cp = W.small_coupled(m=4, n_coarse=6)
    o = MTSOracle(cp, breaking=False)
    o.advance(3)  # a state with lambda_0 != 0
    u, v, a = o.u.copy(), o.v.copy(), o.a.copy()
    uf, vf, af = o.uf.copy(), o.vf.copy(), o.af.copy()
    lam0 = o.lam.copy()
    lam_m = o.coarse_step()
    assert np.linalg.norm(lam0) > 0 and np.linalg.norm(lam_m) > 0
    m = cp.m
    g0, gm = o.interface_force_density(lam0), o.interface_force_density(lam_m)
    mu = o.mu.copy()
    for j in range(1, m + 1):
        gj = (1.0 - j / m) * g0 + (j / m) * gm
        pd_run(o.pd, o.rp, o.col, mu, u, v, a, 1, alpha=o.alpha, b=None, g=np.ascontiguousarray(gj),
               theta=np.ones(1), breaking=False)
    for x, y in [(u, o.u), (v, o.v), (a, o.a)]:
        assert np.linalg.norm(x - y) <= 1e-11 * np.linalg.norm(y)
    # FE: one implicit Newmark step with the load P - G_FE^T lambda_m
    dtf, be, ga = o.dt_fe, o.beta, o.gamma
    ut = uf + dtf * vf + (0.5 - be) * dtf * dtf * af
    vt = vf + (1 - ga) * dtf * af
    an = o.solver.solve(o.fe.P - o.Gfe.T @ lam_m - o.fe.K @ ut)
    for x, y in [(ut + be * dtf * dtf * an, o.uf), (vt + ga * dtf * an, o.vf), (an, o.af)]:
        assert np.linalg.norm(x - y) <= 1e-11 * np.linalg.norm(y)


@pytest.mark.parametrize("dim", [2, 3])
def test_fe_patch_affine_field_energy_and_interior_balance(dim):
    """Patch test of the Q4 (plane stress) and Hex8 elements on a block of
    rectangular (non-square) elements: an affine displacement u = F x leaves
    every interior node in equilibrium (K u = 0 there), and the strain energy
    (1/2) u' K u equals the continuum energy of the uniform strain times the
    volume, written with Lame constants: mu e:e + (lam'/2) (tr e)^2, where
    lam' = 2 lam mu / (lam + 2 mu) in plane stress and lam' = lam in 3D. The
    lumped mass sums to rho times the volume."""
    from oracle.mts import FE
    E, nu, rho, t = 72e9, 0.3, 2440.0, 1e-3
    rng = np.random.default_rng(5)
    if dim == 2:
        X0, c0 = W.q4_block(0.0, 0.0, 4, 3, 1e-3)
        X = X0 * np.array([[1.0], [1.7]])  # rectangles 1 x 1.7 mm
        ne, vol = 4 * 3, 4e-3 * 3 * 1.7e-3 * t
        fe = FE(W.FEMesh(X, c0, 1e-3), E, nu, rho, t, [], 1, np.zeros((0, 2), np.int32), np.zeros((0, 2)))
    else:
        X0, c0 = W.hex8_block(0.0, 0.0, 0.0, 3, 3, 3, 1e-3)
        X = X0 * np.array([[1.0], [1.4], [0.8]])
        vol = 3e-3 * 3 * 1.4e-3 * 3 * 0.8e-3
        fe = FE(W.FEMesh(X, c0, 1e-3), E, nu, rho, 1.0, [], 1, np.zeros((0, 4), np.int32), np.zeros((0, 3)))
    F = rng.standard_normal((dim, dim)) * 1e-4
    u = (F @ X).reshape(-1)  # SoA: all x, then all y (, all z)
    K = fe.K.toarray()
    f = K @ u
    n = X.shape[1]
    lo, hi = X.min(axis=1, keepdims=True), X.max(axis=1, keepdims=True)
    interior = np.all((X > lo + 1e-12) & (X < hi - 1e-12), axis=0)
    assert interior.sum() > 0
    scale = np.abs(f).max()
    for d in range(dim):
        assert np.abs(f[d * n:(d + 1) * n][interior]).max() <= 1e-9 * scale
    eps = 0.5 * (F + F.T)
    mu = E / (2 * (1 + nu))
    lam = E * nu / ((1 + nu) * (1 - 2 * nu))
    if dim == 2:
        lam = 2 * lam * mu / (lam + 2 * mu)
    w = mu * np.sum(eps * eps) + 0.5 * lam * np.trace(eps) ** 2
    energy = 0.5 * u @ f
    assert abs(energy - w * vol) <= 1e-11 * w * vol
    assert abs(fe.M.sum() / dim - rho * vol) <= 1e-12 * rho * vol
    # one element: exactly the rigid-body modes in the null space (3 in 2D,
    # 6 in 3D; under-integration would add hourglass modes)
    if dim == 2:
        X1, c1 = W.q4_block(0.0, 0.0, 1, 1, 1e-3)
        one = FE(W.FEMesh(X1 * np.array([[1.0], [1.7]]), c1, 1e-3), E, nu, rho, t, [], 1,
                 np.zeros((0, 2), np.int32), np.zeros((0, 2)))
    else:
        X1, c1 = W.hex8_block(0.0, 0.0, 0.0, 1, 1, 1, 1e-3)
        one = FE(W.FEMesh(X1 * np.array([[1.0], [1.4], [0.8]]), c1, 1e-3), E, nu, rho, 1.0, [], 1,
                 np.zeros((0, 4), np.int32), np.zeros((0, 3)))
    ev = np.linalg.eigvalsh(one.K.toarray())
    assert np.sum(np.abs(ev) <= 1e-9 * ev.max()) == (3 if dim == 2 else 6)
