"""GPU parity of the PD hot path against the FP64 oracle (through the C ABI).

FP64 build: identical arithmetic in the oracle's order, so displacements,
velocities, accelerations, damage and the broken-bond set must agree exactly;
the stated bar is rel-L2 <= 1e-10 and an identical broken set.
FP32-bulk build: rel-L2 of u <= 1e-4 and broken-bond mismatch <= 0.1 % against
the FP64 result (the stated tolerances of the FP32-bulk path), written into each test.
"""
import numpy as np
import pytest

import oracle
from gpu_common import GpuPDRun, OracleRun, rel_l2
from paper_2403_03605_gb300 import diagnostics as D
from paper_2403_03605_gb300 import pdmts as P
from paper_2403_03605_gb300 import workloads as W

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-10
FP32_TOL = 1e-4
FP32_MISMATCH = 1e-3
# crack plane of the 100 x 100 plate (normal y, level 25 mm, along x) and the band searched
# for the crack tip (5 mm: the loading layers at the faces stay outside)
PLATE100_CRACK = (1, 0.025, 0, 5e-3)


@pytest.fixture(scope="module")
def ctx():
    from paper_2403_03605_gb300 import build
    build.build()
    c = P.pdmts_ctx_create(0)
    yield c
    P.pdmts_ctx_destroy(c)


@pytest.fixture
def fresh(ctx):
    """A fresh context per test (one PD subdomain per context)."""
    made = []

    def mk():
        c = P.pdmts_ctx_create(0)
        made.append(c)
        return c
    yield mk
    for c in made:
        P.pdmts_ctx_destroy(c)


def _assert_fp64_identical(g: GpuPDRun, o: OracleRun):
    u, v, a = g.u(), g.v(), g.a()
    assert rel_l2(u, o.u) <= FP64_TOL
    assert rel_l2(v, o.v) <= FP64_TOL
    assert rel_l2(a, o.a) <= FP64_TOL
    # the parity build is bit-identical (signed zeros compare equal)
    assert np.array_equal(u, o.u) and np.array_equal(v, o.v) and np.array_equal(a, o.a)
    assert np.array_equal(g.mu(), o.mu)
    assert np.array_equal(g.damage(), o.damage())


def test_family_and_precrack_match_oracle(fresh):
    for pb in (W.plate_100x100(), W.plate3d(11, 9, 8, 0.5e-3, cuts_mm=[(1, 2.25e-3, 0, 0.0, 2.5e-3)])):
        ctx = fresh()
        g = GpuPDRun(ctx, pb, P.PDMTS_FP64)
        o = OracleRun(pb)
        rp, col = P.pd_read_family(g.pd)
        assert np.array_equal(rp, o.rp) and np.array_equal(col, o.col)
        mu = g.mu()
        assert np.array_equal(mu, o.mu)
        assert int((mu == 0).sum()) == o.ncut > 0


def test_plate_100x100_fp64_bit_identical(fresh):
    """100 x 100 plate, centred crack, 12 MPa, dt 25 ns, 500 steps: identical
    displacements and an identical broken-bond set, with breaking under way."""
    pb = W.plate_100x100()
    o = OracleRun(pb).run(pb.nsteps)
    assert o.broken > 1000  # the run breaks bonds beyond the pre-crack
    g = GpuPDRun(fresh(), pb, P.PDMTS_FP64).run(pb.nsteps)
    _assert_fp64_identical(g, o)
    # crack tips of the two runs (oracle rule on the oracle's damage, the
    # library's host-side rule on the GPU damage): identical
    tip_o = oracle.crack_tip(pb.lat.X, o.damage(), *PLATE100_CRACK)
    tip_g = D.crack_tip(pb.lat.X, g.damage(), *PLATE100_CRACK)
    print(f"100x100 plate crack tips: oracle {tip_o}, GPU FP64 {tip_g}")
    assert tip_o == tip_g and not np.isnan(tip_o[0])


VARIANTS = [
    dict(name="ragged_2d", pb=lambda: W.small_plate(37, 23, nsteps=120)),
    dict(name="weights_2d", pb=lambda: W.small_plate(41, 19, nsteps=100), alpha=True),
    dict(name="pmb_2d", pb=lambda: W.small_plate(33, 21, nsteps=100), force="pmb"),
    dict(name="exp_2d", pb=lambda: W.small_plate(35, 20, nsteps=100), micro="exp"),
    dict(name="plate_3d", pb=lambda: W.plate3d(15, 11, 8, 0.5e-3, cuts_mm=[(1, 2.75e-3, 0, 0.0, 3e-3)],
                                                 traction=40e6, nsteps=60)),
    dict(name="weights_pmb_3d", pb=lambda: W.plate3d(13, 10, 7, 0.5e-3, traction=40e6, nsteps=50),
         alpha=True, force="pmb"),
    dict(name="random_state_2d", pb=lambda: W.small_plate(30, 30, nsteps=80, crack=False), state=True),
]


@pytest.mark.parametrize("case", VARIANTS, ids=[c["name"] for c in VARIANTS])
def test_fp64_parity_variants(fresh, case):
    pb = case["pb"]()
    rng = np.random.default_rng(11)
    alpha = rng.uniform(0.0, 0.8, pb.n) if case.get("alpha") else None
    micro_o, micro_g, l, c = oracle.MICRO_POWER, P.PDMTS_MICRO_POWER, 0.0, None
    if case.get("micro") == "exp":
        micro_o, micro_g, l = oracle.MICRO_EXP, P.PDMTS_MICRO_EXP, pb.delta / 10.0
        c = pb.c / pb.delta ** 3 * 500.0  # comparable stiffness to the power law at |xi| = dx
    force_o = oracle.FORCE_PMB if case.get("force") == "pmb" else oracle.FORCE_LINEAR
    force_g = P.PDMTS_FORCE_PMB if case.get("force") == "pmb" else P.PDMTS_FORCE_LINEAR
    u0 = v0 = None
    if case.get("state"):
        u0 = rng.standard_normal((pb.dim, pb.n)) * pb.s0 * pb.lat.dx * 0.4
        v0 = rng.standard_normal((pb.dim, pb.n)) * 0.05
    o = OracleRun(pb, alpha=alpha, micro=micro_o, l=l, c=c, force=force_o, u0=u0, v0=v0).run(pb.nsteps)
    g = GpuPDRun(fresh(), pb, P.PDMTS_FP64, micro=micro_g, l=l, c=c, force=force_g, u0=u0, v0=v0,
               alpha=alpha).run(pb.nsteps)
    assert pb.n % 32 != 0 or case["name"] == "random_state_2d"
    _assert_fp64_identical(g, o)


def test_graph_chain_equals_single_steps(fresh):
    """Substeps replayed from a captured CUDA graph equal substeps launched one by one."""
    pb = W.small_plate(45, 30, nsteps=0)
    g1 = GpuPDRun(fresh(), pb, P.PDMTS_FP64).run(97)
    g2 = GpuPDRun(fresh(), pb, P.PDMTS_FP64)
    for _ in range(97):
        g2.run(1)
    assert np.array_equal(g1.u(), g2.u()) and np.array_equal(g1.mu(), g2.mu())
    st = P.pdmts_get_stats(g1.ctx)
    assert st["graph_launches"] >= 6 and st["pd_substeps"] == 97


LATTICE_CASES = [
    dict(name="plate_100x100", pb=lambda: W.plate_100x100(), steps=500),
    dict(name="weights", pb=lambda: W.small_plate(70, 45, nsteps=150), alpha=True, steps=150),
    dict(name="weights_nx72", pb=lambda: W.small_plate(72, 45, nsteps=150), alpha=True, steps=150),
    dict(name="pmb", pb=lambda: W.small_plate(66, 41, nsteps=150), force=True, steps=150),
    dict(name="tiny", pb=lambda: W.plate2d(5, 3, 0.5e-3, traction=60e6), steps=40),
]


def _lattice_pair(fresh, case):
    pb = case["pb"]()
    rng = np.random.default_rng(21)
    alpha = rng.uniform(0.0, 0.7, pb.n) if case.get("alpha") else None
    force = P.PDMTS_FORCE_PMB if case.get("force") else P.PDMTS_FORCE_LINEAR
    u0 = rng.standard_normal((2, pb.n)) * pb.s0 * pb.lat.dx * 0.2
    return pb, alpha, force, u0


@pytest.mark.parametrize("case", LATTICE_CASES, ids=[c["name"] for c in LATTICE_CASES])
def test_fp32_lattice_kernel_agrees_with_sliced_ell_kernel(fresh, case):
    """The 2D lattice kernel (bond words, shared-memory halo, strips of nodes per
    thread) and the sliced-ELL kernel evaluate the same bond law, the lattice
    kernel in its scaled form (q = lhs / |d|^2) and in stencil-column order:
    they agree to FP32 rounding, with the FP32 bar on the broken set."""
    pb, alpha, force, u0 = _lattice_pair(fresh, case)
    gl = GpuPDRun(fresh(), pb, P.PDMTS_FP32_BULK, alpha=alpha, force=force, u0=u0)
    gs = GpuPDRun(fresh(), pb, P.PDMTS_FP32_BULK_SELL, alpha=alpha, force=force, u0=u0)
    assert P.pd_info(gl.pd)["layout"] == 1 and P.pd_info(gs.pd)["layout"] == 0
    gl.run(case["steps"])
    gs.run(case["steps"])
    eu, ev = rel_l2(gl.u(), gs.u()), rel_l2(gl.v(), gs.v())
    mm = _mismatch(gl.mu(), gs.mu())
    print(f"lattice vs sliced-ELL {case['name']}: rel-L2 u {eu:.2e} v {ev:.2e}, broken mismatch {mm:.2e}")
    assert eu <= FP32_TOL and ev <= FP32_TOL, (eu, ev)
    assert mm <= FP32_MISMATCH, mm


@pytest.mark.parametrize("case", LATTICE_CASES, ids=[c["name"] for c in LATTICE_CASES])
def test_lattice_tile_configurations_bit_identical(fresh, case):
    """Every tile configuration of the lattice kernel (strip height, CTAs per SM)
    gives each node its bonds in the same order, and a warp that falls back to
    the bond-by-bond path without a break reproduces the fast path: identical
    bits, and the autotuner's choice cannot change results."""
    pb, alpha, force, u0 = _lattice_pair(fresh, case)
    runs = []
    for tile in [*range(P.PDMTS_LATTICE_TILES), P.PDMTS_LATTICE_TILE_AUTO]:
        g = GpuPDRun(fresh(), pb, P.PDMTS_FP32_BULK, alpha=alpha, force=force, u0=u0)
        P.pd_set_lattice_tile(g.pd, tile)
        g.run(case["steps"])
        got = P.pd_info(g.pd)["lattice_tile"]
        assert got == tile if tile >= 0 else 0 <= got < P.PDMTS_LATTICE_TILES
        runs.append((g.u(), g.v(), g.mu()))
    for u, v, mu in runs[1:]:
        assert np.array_equal(u, runs[0][0]) and np.array_equal(v, runs[0][1])
        assert np.array_equal(mu, runs[0][2])


def _mismatch(mu_a, mu_b):
    return float(np.count_nonzero(mu_a != mu_b)) / len(mu_a)


def test_plate_100x100_fp32_bulk_within_tolerance(fresh):
    pb = W.plate_100x100()
    g64 = GpuPDRun(fresh(), pb, P.PDMTS_FP64).run(pb.nsteps)
    g32 = GpuPDRun(fresh(), pb, P.PDMTS_FP32_BULK).run(pb.nsteps)
    err = rel_l2(g32.u(), g64.u())
    mm = _mismatch(g32.mu(), g64.mu())
    tip_err = D.tip_error(D.crack_tip(pb.lat.X, g32.damage(), *PLATE100_CRACK),
                          D.crack_tip(pb.lat.X, g64.damage(), *PLATE100_CRACK))
    print(f"100x100 plate fp32-bulk vs fp64: rel-L2 u {err:.2e}, broken mismatch {mm:.2e}, crack-tip error {tip_err:.2e} m")
    assert err <= FP32_TOL, err
    assert mm <= FP32_MISMATCH, mm
    assert tip_err <= pb.delta, tip_err  # reported; within one horizon


LATTICE3D_CASES = [
    dict(name="breaking", pb=lambda: W.plate3d(15, 11, 8, 0.5e-3, cuts_mm=[(1, 2.75e-3, 0, 0.0, 3e-3)],
                                               traction=40e6, nsteps=60)),
    dict(name="weights_pmb", pb=lambda: W.plate3d(13, 10, 7, 0.5e-3, traction=40e6, nsteps=50), alpha=True,
         force=True),
    dict(name="exp_state", pb=lambda: W.plate3d(12, 9, 10, 0.5e-3, traction=20e6, nsteps=40), micro=True, state=True),
    # weights only on the rows y >= 10: warps near them take the weighted code, the others skip the weights
    dict(name="wide_weights", pb=lambda: W.plate3d(75, 14, 9, 0.5e-3, cuts_mm=[(1, 3.5e-3, 0, 0.0, 8e-3)],
                                                   traction=40e6, nsteps=40), alpha="rows"),
]


@pytest.mark.parametrize("case", LATTICE3D_CASES, ids=[c["name"] for c in LATTICE3D_CASES])
def test_fp32_lattice3d_kernel_bit_identical_to_sliced_ell(fresh, case):
    """The 3D lattice kernel (implicit 122-offset family, four bond words per
    node; blocks of 32 x 4 or 32 x 8 nodes of one plane) takes the sliced-ELL
    kernel's operations in the same order: the same bits, breaks included, for
    both tile configurations (lattices of 12 to 75 nodes along x, so that
    warps run past the box, touch its x faces or lie inside, and 7 to 10
    along z)."""
    pb = case["pb"]()
    rng = np.random.default_rng(23)
    alpha = rng.uniform(0.0, 0.8, pb.n) if case.get("alpha") else None
    if case.get("alpha") == "rows":
        alpha[pb.lat.idx[1] < 10] = 0.0
    force = P.PDMTS_FORCE_PMB if case.get("force") else P.PDMTS_FORCE_LINEAR
    micro, l, c = P.PDMTS_MICRO_POWER, 0.0, None
    if case.get("micro"):
        micro, l, c = P.PDMTS_MICRO_EXP, pb.delta / 10.0, pb.c / pb.delta ** 3 * 500.0
    u0 = rng.standard_normal((3, pb.n)) * pb.s0 * pb.lat.dx * 0.3 if case.get("state") else None
    b = GpuPDRun(fresh(), pb, P.PDMTS_FP32_BULK_SELL, alpha=alpha, force=force, micro=micro, l=l, c=c, u0=u0)
    assert P.pd_info(b.pd)["layout"] == 0
    b.run(pb.nsteps)
    for tile in range(2):
        a = GpuPDRun(fresh(), pb, P.PDMTS_FP32_BULK, alpha=alpha, force=force, micro=micro, l=l, c=c, u0=u0)
        assert P.pd_info(a.pd)["layout"] == 2
        P.pd_set_lattice_tile(a.pd, tile)
        a.run(pb.nsteps)
        assert np.array_equal(a.u(), b.u()) and np.array_equal(a.v(), b.v()), tile
        assert np.array_equal(a.mu(), b.mu()), tile
        # damage from bond counts (lattice) or volume sums (sliced ELL, uniform V): equal up to FP64 rounding
        np.testing.assert_allclose(a.damage(), b.damage(), rtol=0, atol=1e-14)
    if case["name"] in ("breaking", "wide_weights"):
        assert (b.mu() == 0).sum() > 0
    with pytest.raises(P.PdmtsError):
        P.pd_set_lattice_tile(a.pd, 2)  # 3D lattices have two configurations


@pytest.mark.parametrize("dim", [2, 3])
def test_fp32_bulk_elastic_accuracy(fresh, dim):
    """Without breaking, FP32-bulk tracks the FP64 oracle closely (random initial state)."""
    if dim == 2:
        pb = W.small_plate(50, 40, nsteps=300, crack=False)
    else:
        pb = W.plate3d(16, 12, 9, 0.5e-3, traction=12e6, nsteps=150)
    rng = np.random.default_rng(5)
    u0 = rng.standard_normal((pb.dim, pb.n)) * 1e-9
    o = OracleRun(pb, breaking=False, u0=u0).run(pb.nsteps)
    g = GpuPDRun(fresh(), pb, P.PDMTS_FP32_BULK, breaking=False, u0=u0).run(pb.nsteps)
    eu, ev = rel_l2(g.u(), o.u), rel_l2(g.v(), o.v)
    print(f"fp32 elastic dim={dim}: rel-L2 u {eu:.2e} v {ev:.2e}")
    assert eu <= 1e-5, eu
    assert ev <= 1e-4, ev


def test_edge_cases(fresh):
    # one node, no bonds: free flight under its body force
    X = np.array([[1e-3], [2e-3]])
    ctx = fresh()
    pd = P.pd_create(ctx, X, horizon=1e-4, c=1e20, s0=1e-3, rho=1000.0, vol_uniform=1e-9)
    b = np.array([[2e9], [-1e9]])
    P.pd_set_body_force(pd, b)
    P.mts_set_time(ctx, 1e-8, 1)
    P.mts_advance(ctx, 10)
    np.testing.assert_allclose(P.pd_read_displacement(pd), 0.5 * b / 1000.0 * (1e-7) ** 2, rtol=1e-12)
    assert P.pd_info(pd)["n_bonds"] == 0
    # n = 0 is rejected
    with pytest.raises(P.PdmtsError) as e:
        P.pd_create(fresh(), np.zeros((2, 0)), horizon=1e-3, c=1.0, s0=1.0, rho=1.0, vol_uniform=1.0)
    assert e.value.code == -1
    # every bond pre-broken: nodes fly freely, damage 1 everywhere
    pb = W.plate2d(8, 8, 1e-3, traction=0.0)
    ctx = fresh()
    g = GpuPDRun(ctx, pb, P.PDMTS_FP64)
    P.pd_set_precrack(g.pd, [(1, (k + 1) * 1e-3, 0, -1.0, 1.0) for k in range(7)] +
                      [(0, (k + 1) * 1e-3, 1, -1.0, 1.0) for k in range(7)])
    mu = g.mu()
    assert mu.sum() == 0
    assert np.all(g.damage() == 1.0)
    # weights that leave no mass are rejected
    with pytest.raises(P.PdmtsError) as e:
        P.pd_set_weights(g.pd, np.ones(pb.n))
    assert e.value.code == -2
    # FP32 bulk off-lattice is unsupported, not silently degraded
    rng = np.random.default_rng(2)
    with pytest.raises(P.PdmtsError) as e:
        P.pd_create(fresh(), rng.uniform(0, 1e-2, (2, 200)), horizon=2e-3, c=1e20, s0=1e-3, rho=1e3,
                    vol_uniform=1e-9, precision=P.PDMTS_FP32_BULK)
    assert e.value.code == -8
    # dt above the stability bound
    with pytest.raises(P.PdmtsError) as e:
        P.mts_set_time(ctx, 1e-5, 1)
    assert e.value.code == -3


def test_newtons_third_law_full_size(fresh):
    """At the 800k-node strip size: sum_i (1 - alpha_i) rho V a_i = sum_i f_i V_i = 0
    for a random state (no loads), a property that holds at any size."""
    pb = W.strip_lattice_pd(2000, 400, 0.05e-3, 0.05, traction=0.0, dt=5e-9)
    rng = np.random.default_rng(3)
    u0 = rng.standard_normal((2, pb.n)) * 1e-9
    ctx = fresh()
    g = GpuPDRun(ctx, pb, P.PDMTS_FP64, u0=u0, body=False, breaking=False)
    a = g.a()
    m = pb.mat.rho * pb.vol
    assert np.abs((m * a).sum(1)).max() <= 1e-12 * np.abs(m * a).sum()


@pytest.mark.slow
def test_full_size_strip_fp64_and_fp32_against_oracle(fresh):
    """The 2000 x 400 (800k-node, 22.3M-bond) strip lattice: 12 substeps from a
    seeded random state, FP64 bit-identical and FP32-bulk within tolerance."""
    pb = W.strip_lattice_pd(2000, 400, 0.05e-3, 0.05, traction=12e6, dt=5e-9)
    rng = np.random.default_rng(9)
    u0 = rng.standard_normal((2, pb.n)) * pb.s0 * pb.lat.dx * 0.3
    nst = 12
    o = OracleRun(pb, u0=u0).run(nst)
    g64 = GpuPDRun(fresh(), pb, P.PDMTS_FP64, u0=u0).run(nst)
    _assert_fp64_identical(g64, o)
    g32 = GpuPDRun(fresh(), pb, P.PDMTS_FP32_BULK, u0=u0).run(nst)
    assert rel_l2(g32.u(), o.u) <= FP32_TOL
    assert _mismatch(g32.mu(), o.mu) <= FP32_MISMATCH
