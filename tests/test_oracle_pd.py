"""Pins of the FP64 PD oracle against what the mathematics fixes (CPU only).

Each test checks the oracle against something other than itself: closed-form
solutions, invariants of the method, exact brute force on small inputs, or
counts obtained by independent integer arithmetic. A dropped term, a wrong sign
or index, or a transposed operand anywhere in the oracle fails at least one.
"""
import itertools
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2403_03605_gb300 import workloads as W

MAT = W.Material()


def _lattice_offsets(dim, m):
    r = int(math.floor(m))
    offs = []
    for o in itertools.product(range(-r, r + 1), repeat=dim):
        if any(o) and sum(x * x for x in o) <= m * m:
            offs.append(o)
    return offs


# ---------------------------------------------------------------- family ----
def test_interior_family_sizes():
    """28 neighbours in 2D and 122 in 3D at delta = 3.015 dx (integer enumeration)."""
    assert len(_lattice_offsets(2, W.HORIZON_FACTOR)) == 28
    assert len(_lattice_offsets(3, W.HORIZON_FACTOR)) == 122
    lat = W.Lattice((13, 11), 1e-3, (0.0, 0.0))
    rp, col = oracle.family(lat.X, W.HORIZON_FACTOR * 1e-3)
    deg = np.diff(rp).reshape(11, 13)
    assert deg[5, 6] == 28 and deg.max() == 28
    lat3 = W.Lattice((9, 9, 9), 1e-3, (0.0, 0.0, 0.0))
    rp3, _ = oracle.family(lat3.X, W.HORIZON_FACTOR * 1e-3)
    assert np.diff(rp3).max() == 122 and np.diff(rp3)[4 + 9 * (4 + 9 * 4)] == 122


def test_family_total_100x100_by_offset_counting():
    """Directed-bond total of the 100 x 100 plate equals sum over stencil offsets of
    (nx - |di|)(ny - |dj|), an integer count independent of the float search."""
    pb = W.plate_100x100()
    rp, col = oracle.family(pb.lat.X, pb.delta)
    nx, ny = pb.lat.shape
    total = sum((nx - abs(a)) * (ny - abs(b)) for a, b in _lattice_offsets(2, W.HORIZON_FACTOR))
    assert total == 272836
    assert rp[-1] == total


def test_family_matches_brute_force_on_random_cloud():
    rng = np.random.default_rng(1)
    for dim in (2, 3):
        n = 300 if dim == 2 else 400
        X = rng.uniform(0, 1e-2, size=(dim, n))
        delta = 1.7e-3
        rp, col = oracle.family(X, delta)
        d2 = ((X[:, :, None] - X[:, None, :]) ** 2).sum(0)
        for i in range(n):
            ref = np.nonzero((d2[i] <= delta * delta) & (np.arange(n) != i))[0]
            np.testing.assert_array_equal(col[rp[i]:rp[i + 1]], ref)


# -------------------------------------------------------------- pre-crack ----
def _crosses_exact(p, q, cut):
    na, level, pa, lo, hi = cut
    a, b = Fraction(p[na]), Fraction(q[na])
    if not ((a < level < b) or (b < level < a)):
        return False
    t = (Fraction(level) - a) / (b - a)
    xc = Fraction(p[pa]) + t * (Fraction(q[pa]) - Fraction(p[pa]))
    return lo <= xc < hi


def test_precrack_matches_exact_rational_brute_force():
    lat = W.Lattice((24, 14), 1e-3, (0.0, 0.0))
    rp, col = oracle.family(lat.X, W.HORIZON_FACTOR * 1e-3)
    P = lat.P
    # cuts in half-dx units: tips on node columns, between columns, vertical cut
    cuts = [(1, 14, 0, 8, 26), (1, 6, 0, 0, 13), (0, 30, 1, 4, 18)]
    mu, cnt = oracle.precrack(P, rp, col, cuts)
    ref = 0
    for i in range(lat.n):
        for k in range(rp[i], rp[i + 1]):
            j = col[k]
            cut = any(_crosses_exact(P[:, i], P[:, j], c) for c in cuts)
            assert mu[k] == (0 if cut else 1), (i, j)
            ref += cut
    assert cnt == ref > 0


def test_precrack_count_100x100():
    """Centred 10 mm crack of the 100 x 100 plate cuts 720 directed bonds."""
    pb = W.plate_100x100()
    rp, col = oracle.family(pb.lat.X, pb.delta)
    mu, cnt = oracle.precrack(pb.lat.P, rp, col, [c.in_half_units(pb.lat) for c in pb.cuts])
    assert cnt == 720
    # symmetric: (i, j) cut iff (j, i) cut
    i_of = np.repeat(np.arange(pb.n), np.diff(rp))
    cut_pairs = set(zip(i_of[mu == 0].tolist(), col[mu == 0].tolist()))
    assert all((j, i) in cut_pairs for i, j in cut_pairs)


# ------------------------------------------------------- two-node bond -------
def _two_nodes(L, ang, micro=oracle.MICRO_POWER, c=1e20, l=0.0, force=oracle.FORCE_LINEAR):
    e = np.array([math.cos(ang), math.sin(ang)])
    X = np.stack([np.zeros(2), L * e], axis=1)
    V = 2.5e-10
    pd = oracle.PD(X, V, delta=1.5 * L, c=c, s0=10.0, rho=2440.0, dt=1e-9, micro=micro, l=l, force=force,
                   breaking=False)
    rp, col = oracle.family(X, pd.delta)
    return pd, rp, col, e


@pytest.mark.parametrize("micro", [oracle.MICRO_POWER, oracle.MICRO_EXP])
@pytest.mark.parametrize("force", [oracle.FORCE_LINEAR, oracle.FORCE_PMB])
def test_two_node_oscillator_closed_form(micro, force):
    """Stretch mode of one bond: q'' = -omega^2 q with omega^2 = 2 c(L) L^2 V / rho;
    the Verlet recurrence gives q_n = q0 cos(n theta), cos theta = 1 - omega^2 dt^2 / 2.
    A transverse relative displacement carries no linearised force."""
    L, ang = 7e-4, 0.37
    l = L / 2.5
    c = 6e22 if micro == oracle.MICRO_POWER else 3e27
    pd, rp, col, e = _two_nodes(L, ang, micro=micro, c=c, l=l, force=force)
    cL = c / L ** 3 if micro == oracle.MICRO_POWER else c * math.exp(-L / l)
    w2 = 2.0 * cL * L * L * pd.V[0] / pd.rho
    dt = 0.2 / math.sqrt(w2)
    pd.dt = dt
    q0 = 1e-7
    u = np.zeros((2, 2))
    u[:, 0] = -0.5 * q0 * e
    u[:, 1] = +0.5 * q0 * e
    v = np.zeros_like(u)
    a = np.zeros_like(u)
    mu = np.ones(len(col), np.uint8)
    theta = math.acos(1.0 - 0.5 * w2 * dt * dt)
    for n in range(1, 6):
        init = n == 1
        oracle.pd_run(pd, rp, col, mu, u, v, a, 40, init=init)
        q = float((u[:, 1] - u[:, 0]) @ e)
        ref = q0 * math.cos(40 * n * theta)
        tol = 1e-12 if force == oracle.FORCE_LINEAR else 1e-9  # PMB along the bond is linear up to O(q^2)
        assert abs(q - ref) <= tol * q0 + 1e-9 * abs(ref) * (force == oracle.FORCE_PMB), (n, q, ref)
    if force == oracle.FORCE_LINEAR:
        # transverse relative displacement: no force (xi (x) xi projects it out)
        et = np.array([-e[1], e[0]])
        u = np.zeros((2, 2))
        u[:, 1] = 1e-7 * et
        f, _ = oracle.pd_forces(pd, rp, col, mu, u)
        axial = cL * L * L * 1e-7 * pd.V[0]  # force density of the same |eta| along the bond
        assert np.abs(f).max() <= 1e-15 * axial


def test_weighted_two_node_oscillator():
    """With Arlequin weights the bond carries w = 1 - (a1 + a2)/2 and node masses are
    (1 - a_i) rho V: q'' = -w c L^2 V (1/m1 + 1/m2) q (per unit volume masses)."""
    L, ang = 5e-4, 1.1
    pd, rp, col, e = _two_nodes(L, ang, c=6e22)
    al = np.array([0.3, 0.75])
    w = 1.0 - 0.5 * (al[0] + al[1])
    k = w * (6e22 / L ** 3) * L * L * pd.V[0]
    w2 = k * (1.0 / ((1 - al[0]) * pd.rho) + 1.0 / ((1 - al[1]) * pd.rho))
    pd.dt = 0.15 / math.sqrt(w2)
    q0 = 2e-7
    u = np.zeros((2, 2))
    u[:, 1] = q0 * e
    v = np.zeros_like(u)
    a = np.zeros_like(u)
    mu = np.ones(len(col), np.uint8)
    oracle.pd_run(pd, rp, col, mu, u, v, a, 77, alpha=al, init=True)
    theta = math.acos(1.0 - 0.5 * w2 * pd.dt ** 2)
    q = float((u[:, 1] - u[:, 0]) @ e)
    assert abs(q - q0 * math.cos(77 * theta)) < 1e-12 * q0
    # momentum sum (1 - a_i) rho V v_i is conserved (zero)
    p = ((1 - al) * pd.rho * pd.V * v).sum(1)
    assert np.abs(p).max() < 1e-12 * np.abs((1 - al) * pd.rho * pd.V * v).max()


def test_constant_body_force_is_exact():
    """Verlet is exact for constant acceleration: u_n = b/rho (n dt)^2 / 2, also when
    the node carries an Arlequin weight (mass and load both scale by 1 - alpha)."""
    X = np.array([[0.0, 1.0], [0.0, 0.0]])
    pd = oracle.PD(X, 1e-9, delta=0.1, c=1.0, s0=1.0, rho=2000.0, dt=1e-8)
    rp, col = oracle.family(X, pd.delta)
    assert rp[-1] == 0
    b = np.array([[3e9, -1e9], [2e9, 5e9]])
    u = np.zeros((2, 2)); v = np.zeros_like(u); a = np.zeros_like(u)
    mu = np.ones(0, np.uint8)
    oracle.pd_run(pd, rp, col, mu, u, v, a, 250, b=b, alpha=np.array([0.0, 0.4]), init=True)
    t = 250 * pd.dt
    np.testing.assert_allclose(u, 0.5 * b / pd.rho * t * t, rtol=1e-12)
    np.testing.assert_allclose(v, b / pd.rho * t, rtol=1e-12)


# ------------------------------------------------------------- invariants --
def _small_pd(nx=16, ny=12, dim=2, breaking=False, nz=6):
    if dim == 2:
        pb = W.plate2d(nx, ny, 0.5e-3, traction=0.0)
    else:
        pb = W.plate3d(nx, ny, nz, 0.5e-3, traction=0.0)
    pd = oracle.PD(pb.lat.X, pb.vol, pb.delta, pb.c, pb.s0, pb.mat.rho, 20e-9, breaking=breaking)
    rp, col = oracle.family(pb.lat.X, pb.delta)
    return pb, pd, rp, col


@pytest.mark.parametrize("dim", [2, 3])
def test_affine_deformation_gives_zero_interior_force(dim):
    pb, pd, rp, col = _small_pd(14, 13, dim, nz=9)
    rng = np.random.default_rng(3)
    F = rng.standard_normal((dim, dim)) * 1e-4
    u = F @ pb.lat.X
    mu = np.ones(len(col), np.uint8)
    f, _ = oracle.pd_forces(pd, rp, col, mu, u)
    full = 28 if dim == 2 else 122
    interior = np.diff(rp) == full
    scale = full * pb.c * np.abs(F).max() * pb.vol / pb.lat.dx
    assert interior.sum() > 10
    assert np.abs(f[:, interior]).max() <= 1e-13 * scale
    assert np.abs(f[:, ~interior]).max() > 1e-6 * scale  # surface effect is real


@pytest.mark.parametrize("dim", [2, 3])
def test_newtons_third_law(dim):
    """sum_i f_i V_i = 0 for any u, any symmetric bond status and any weights."""
    pb, pd, rp, col = _small_pd(15, 11, dim)
    rng = np.random.default_rng(4)
    u = rng.standard_normal((dim, pb.n)) * 1e-7
    i_of = np.repeat(np.arange(pb.n), np.diff(rp))
    broken_pairs = {(min(i, j), max(i, j)) for i, j in zip(i_of, col) if rng.random() < 0.2}
    mu = np.array([0 if (min(i, j), max(i, j)) in broken_pairs else 1 for i, j in zip(i_of, col)], np.uint8)
    alpha = rng.uniform(0, 0.9, pb.n)
    f, _ = oracle.pd_forces(pd, rp, col, mu, u, alpha=alpha)
    fv = f * pd.V
    assert np.abs(fv.sum(1)).max() <= 1e-13 * np.abs(fv).sum()


@pytest.mark.parametrize("dim", [2, 3])
def test_verlet_modified_energy_is_conserved(dim):
    """For a linear system velocity Verlet conserves exactly
    E~ = 1/2 v'Mv + 1/2 u'Ku - dt^2/8 a'Ma  (breaking off, no loads).
    Pi comes from the separate energy routine, so a force that is not the
    gradient of the bond energy (wrong factor, sign or index) breaks this."""
    pb, pd, rp, col = _small_pd(12, 10, dim)
    rng = np.random.default_rng(5)
    alpha = rng.uniform(0, 0.6, pb.n)
    u = rng.standard_normal((dim, pb.n)) * 1e-8
    v = np.zeros_like(u); a = np.zeros_like(u)
    mu = np.ones(len(col), np.uint8)
    # remove a few symmetric pairs so the mask is exercised as well
    i_of = np.repeat(np.arange(pb.n), np.diff(rp))
    gone = {(min(i, j), max(i, j)) for i, j in zip(i_of, col) if rng.random() < 0.1}
    for k, (i, j) in enumerate(zip(i_of, col)):
        if (min(i, j), max(i, j)) in gone:
            mu[k] = 0
    E = []
    for step in range(40):
        oracle.pd_run(pd, rp, col, mu, u, v, a, 25, alpha=alpha, init=(step == 0))
        m = (1 - alpha) * pd.rho * pd.V
        ke = oracle.kinetic_energy(pd, v, alpha)
        pe = oracle.strain_energy(pd, rp, col, mu, u, alpha)
        corr = pd.dt ** 2 / 8 * float((m * (a * a)).sum())
        E.append(ke + pe - corr)
        assert ke > 0 and pe > 0
    E = np.array(E)
    assert (E.max() - E.min()) <= 1e-11 * E.mean()


@pytest.mark.parametrize("dim,m,target,tol", [(2, 20.015, 1.5, 0.005), (3, 6.015, 3.0, 0.025)])
def test_micromodulus_reproduces_continuum_energy(dim, m, target, tol):
    """Under isotropic strain eps the bond energy density of a node with a full family
    tends to the classical value (2D plane stress nu = 1/3: 1.5 E eps^2; 3D nu = 1/4:
    3 E eps^2) as delta/dx grows; at delta = 3.015 dx the lattice over-estimates
    (2D by 2.5 %, 3D by 9.9 %). Nodes: a ball of lattice sites around the centre."""
    dx = 1e-4
    mat = W.Material() if dim == 2 else W.Material(nu=0.25)
    ratios = []
    for fac in (W.HORIZON_FACTOR, m):
        offs = [(0,) * dim] + _lattice_offsets(dim, fac)
        X = (np.array(offs, dtype=np.float64).T + 0.5) * dx
        delta = fac * dx
        c, s0 = W.pmb_constants(dim, mat, delta)
        vol = mat.thickness * dx * dx if dim == 2 else dx ** 3
        pd = oracle.PD(X, vol, delta, c, s0, mat.rho, 1e-9)
        rp, col = oracle.family(X, delta)
        assert rp[1] - rp[0] == len(offs) - 1
        mu = np.zeros(len(col), np.uint8)
        mu[rp[0]:rp[1]] = 1
        eps = 1e-4
        Pi = oracle.strain_energy(pd, rp, col, mu, eps * X)
        ratios.append(Pi / pd.V[0] / (target * mat.E * eps * eps))
    lattice_ratio, fine_ratio = ratios
    expect = 1.0253995 if dim == 2 else 1.0987100
    assert abs(lattice_ratio - expect) < 1e-6
    assert abs(fine_ratio - 1.0) < tol


def test_breaking_test_matches_literal_stretch_and_is_irreversible():
    """The squared test agrees with Eq. 3 evaluated literally (away from exact ties);
    the bond status never returns to 1 and stays symmetric."""
    pb = W.small_plate(30, 20, nsteps=0)
    pd = oracle.PD(pb.lat.X, pb.vol, pb.delta, pb.c, pb.s0, pb.mat.rho, pb.dt)
    rp, col = oracle.family(pb.lat.X, pb.delta)
    mu, _ = oracle.precrack(pb.lat.P, rp, col, [c.in_half_units(pb.lat) for c in pb.cuts])
    rng = np.random.default_rng(7)
    u = rng.standard_normal((2, pb.n)) * pb.s0 * pb.lat.dx * 0.6
    before = mu.copy()
    f, nb = oracle.pd_forces(pd, rp, col, mu, u)
    i_of = np.repeat(np.arange(pb.n), np.diff(rp))
    X = pb.lat.X
    checked = 0
    for k in np.nonzero(before)[0]:
        i, j = i_of[k], col[k]
        s = oracle.stretch_literal(X[:, j] - X[:, i], u[:, j] - u[:, i])
        if abs(s - pb.s0) < 1e-12:
            continue
        assert (mu[k] == 0) == (s >= pb.s0)
        checked += 1
    assert nb > 0 and checked > 1000
    # run on with breaking: monotone and symmetric
    v = np.zeros_like(u); a = np.zeros_like(u)
    prev = mu.copy()
    pair = {(i, j): k for k, (i, j) in enumerate(zip(i_of.tolist(), col.tolist()))}
    sym = np.array([pair[(j, i)] for i, j in zip(i_of.tolist(), col.tolist())])
    for _ in range(5):
        oracle.pd_run(pd, rp, col, mu, u, v, a, 20, b=pb.b, init=True)
        assert np.all(mu <= prev)
        assert np.array_equal(mu, mu[sym])
        prev = mu.copy()


@pytest.mark.parametrize("break_step", [1, 2])
def test_bond_breaks_before_it_carries_force(break_step):
    """Eq. 4 includes t' = t: a bond that reaches the critical stretch at a
    step carries no force at that step. Two nodes separating along their bond
    from rest positions: the Verlet recurrence with the bond force until the
    breaking step and none from it on is written out step by step; the bond
    (both directions) is cut exactly at that step."""
    L, ang, s0 = 7e-4, 0.37, 1e-3
    pd, rp, col, e = _two_nodes(L, ang, c=6e22)
    pd.s0, pd.breaking = s0, True
    cL = pd.c / L ** 3
    w2 = 2.0 * cL * L * L * pd.V[0] / pd.rho  # relative (stretch) mode
    dt = 0.2 / math.sqrt(w2)
    pd.dt = dt
    # relative speed: the stretch q / L first reaches s0 at step break_step
    q_at = (lambda v0: [dt * v0, dt * v0 + dt * (v0 - 0.5 * dt * w2 * dt * v0) - 0.5 * dt * dt * w2 * dt * v0])
    v0 = 1.5 * s0 * L / dt if break_step == 1 else 0.7 * s0 * L / dt
    q1, q2 = q_at(v0)
    assert (q1 / L >= s0) == (break_step == 1) and q2 / L >= s0
    u = np.zeros((2, 2)); v = np.zeros_like(u); a = np.zeros_like(u)
    v[:, 0], v[:, 1] = -0.5 * v0 * e, 0.5 * v0 * e
    mu = np.ones(len(col), np.uint8)
    oracle.pd_run(pd, rp, col, mu, u, v, a, 0, init=True)  # a_0 = 0 (no stretch yet)
    assert np.all(a == 0.0)
    # written-out recurrence of the relative coordinate q and speed w
    q, w, acc = 0.0, v0, 0.0
    for n in range(1, 4):
        oracle.pd_run(pd, rp, col, mu, u, v, a, 1)
        q_new = q + dt * w + 0.5 * dt * dt * acc
        acc_new = -w2 * q_new if n < break_step else 0.0
        w = w + 0.5 * dt * (acc + acc_new)
        q, acc = q_new, acc_new
        rel_q = float((u[:, 1] - u[:, 0]) @ e)
        rel_w = float((v[:, 1] - v[:, 0]) @ e)
        assert abs(rel_q - q) <= 1e-12 * abs(q) and abs(rel_w - w) <= 1e-12 * abs(v0)
        assert int(mu.sum()) == (2 if n < break_step else 0)


def test_damage_definition():
    """Eq. 5 on a hand-made family: phi = 1 - intact volume / family volume."""
    X = np.array([[0.0, 1.0, 2.0, 3.0], [0.0, 0.0, 0.0, 0.0]])
    V = np.array([1.0, 2.0, 3.0, 4.0])
    pd = oracle.PD(X, V, delta=2.5, c=1.0, s0=1.0, rho=1.0, dt=1.0)
    rp, col = oracle.family(X, 2.5)
    # families: 0:{1,2} 1:{0,2,3} 2:{0,1,3} 3:{1,2}
    assert col.tolist() == [1, 2, 0, 2, 3, 0, 1, 3, 1, 2]
    mu = np.array([1, 0, 1, 1, 0, 0, 1, 1, 1, 1], np.uint8)
    phi = oracle.damage(pd, rp, col, mu)
    np.testing.assert_allclose(phi, [1 - 2 / 5, 1 - 4 / 8, 1 - 6 / 7, 0.0], rtol=0, atol=1e-15)


def test_host_threads_give_the_same_bits():
    """The oracle's node loops on several host threads (each node writes only its
    own bond row and force) reproduce the one-thread run bit for bit, breaking
    included: the all-core CPU baseline times the same computation."""
    pb = W.small_plate(48, 30, nsteps=150)
    rp, col = oracle.family(pb.lat.X, pb.delta)
    cut = [c.in_half_units(pb.lat) for c in pb.cuts]
    runs = []
    for threads in (1, 4):
        assert oracle.set_threads(threads) in (1, threads)
        mu, _ = oracle.precrack(pb.lat.P, rp, col, cut)
        opd = oracle.PD(pb.lat.X, pb.vol, pb.delta, pb.c, pb.s0, MAT.rho, pb.dt)
        u = np.zeros((2, pb.n)); v = np.zeros_like(u); a = np.zeros_like(u)
        nb = oracle.pd_run(opd, rp, col, mu, u, v, a, pb.nsteps, b=pb.b, init=True)
        runs.append((u, v, a, mu, nb))
    oracle.set_threads(1)
    (u1, v1, a1, m1, n1), (u4, v4, a4, m4, n4) = runs
    assert n1 == n4 and n1 > 0
    for x, y in ((u1, u4), (v1, v4), (a1, a4), (m1, m4)):
        assert np.array_equal(x, y)
