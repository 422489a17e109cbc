"""GPU parity of the MTS Arlequin coupling (Algorithm 1) against the FP64 oracle."""
import numpy as np
import pytest

from gpu_common import GpuMTS, rel_l2
from oracle.mts import MTSOracle
from paper_2403_03605_gb300 import diagnostics as D
from paper_2403_03605_gb300 import pdmts as P
from paper_2403_03605_gb300 import workloads as W

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-10


@pytest.fixture
def fresh():
    from paper_2403_03605_gb300 import build
    build.build()
    made = []

    def mk():
        c = P.pdmts_ctx_create(0)
        made.append(c)
        return c
    yield mk
    for c in made:
        P.pdmts_ctx_destroy(c)


def _compare(g, o, tol, lam_tol, mu_exact=True):
    assert rel_l2(g.u(), o.u) <= tol
    assert rel_l2(g.v(), o.v) <= tol
    assert rel_l2(g.uf(), o.uf) <= tol
    assert rel_l2(g.vf(), o.vf) <= tol
    assert rel_l2(g.lam(), o.lam) <= lam_tol
    if mu_exact:
        assert np.array_equal(g.mu(), o.mu)


CASES = [
    dict(name="linear_m4", cp=lambda: W.small_coupled(m=4, n_coarse=20)),
    dict(name="m1", cp=lambda: W.small_coupled(m=1, n_coarse=25)),
    dict(name="cubic_m5", cp=lambda: W.small_coupled(m=5, n_coarse=12, weight_kind=2)),
    dict(name="constant_m3", cp=lambda: W.small_coupled(m=3, n_coarse=12, weight_kind=0)),
    dict(name="breaking_rebuild", cp=lambda: W.small_coupled(m=4, n_coarse=16, traction=30e6)),
]


@pytest.mark.parametrize("case", CASES, ids=[c["name"] for c in CASES])
def test_mts_fp64_matches_oracle(fresh, case):
    cp = case["cp"]()
    o = MTSOracle(cp).advance(cp.n_coarse)
    g = GpuMTS(fresh(), cp, P.PDMTS_FP64).run(cp.n_coarse)
    _compare(g, o, FP64_TOL, 1e-8)
    info = P.arlequin_info(g.arl)
    assert info["rebuilds"] == o.n_rebuilds
    assert g.residual() <= 1e-12
    if case["name"] == "breaking_rebuild":
        assert o.n_rebuilds > 1 and (o.mu == 0).sum() > 100


def test_mts_fp32_bulk_within_tolerance(fresh):
    cp = W.small_coupled(m=4, n_coarse=20)
    o = MTSOracle(cp).advance(cp.n_coarse)
    g = GpuMTS(fresh(), cp, P.PDMTS_FP32_BULK).run(cp.n_coarse)
    err = rel_l2(g.u(), o.u)
    mm = np.count_nonzero(g.mu() != o.mu) / len(o.mu)
    print(f"MTS fp32-bulk: rel-L2 u_pd {err:.2e}, u_fe {rel_l2(g.uf(), o.uf):.2e}, mismatch {mm:.2e}")
    assert err <= 1e-4
    assert rel_l2(g.uf(), o.uf) <= 1e-4
    assert mm <= 1e-3
    assert g.residual() <= 1e-5


def test_fp32_pair_multiplier_product_matches_fp64_product(fresh):
    """FP32-bulk multiplies lambda_m = (-H)^-1 y out with the inverse kept as
    FP32 pairs (error-free FP32 products, compensated sums). On the first
    coarse step everything before the product is the same in a run that takes
    the FP64 product instead, so the two lambda_m differ only by the
    product's rounding: within 1e-10 of the largest |lambda| (an FP32-only
    product, without the low parts, would miss by about 1e-7)."""
    cp = W.small_coupled(m=4, n_coarse=4)
    a = GpuMTS(fresh(), cp, P.PDMTS_FP32_BULK)
    b = GpuMTS(fresh(), cp, P.PDMTS_FP32_BULK)
    P.arlequin_set_multiplier_product(b.arl, P.PDMTS_PRODUCT_FP64)
    assert P.arlequin_info(a.arl)["n_lambda"] % 2 == 0
    a.run(1)
    b.run(1)
    la, lb = a.lam(), b.lam()
    scale = np.abs(lb).max()
    print(f"pair product vs FP64 product: max diff {np.abs(la - lb).max() / scale:.2e} of max |lambda|")
    assert scale > 0
    assert np.abs(la - lb).max() <= 1e-10 * scale
    with pytest.raises(P.PdmtsError):
        P.arlequin_set_multiplier_product(a.arl, 7)


def test_mts_uniform_velocity_patch(fresh):
    cp = W.small_coupled(m=5, n_coarse=4, crack=False, traction=0.0)
    v0 = np.array([3.0, -1.5])
    g = GpuMTS(fresh(), cp, P.PDMTS_FP64, v0=v0).run(4)
    assert np.abs(g.v() - v0.reshape(2, 1)).max() <= 1e-12 * 3.0
    assert np.abs(g.vf() - np.repeat(v0, cp.fe.n)).max() <= 1e-12 * 3.0
    force_scale = cp.pd.mat.rho * 3.0 / (cp.m * cp.dt_pd)
    assert np.abs(g.lam()).max() <= 1e-9 * force_scale


@pytest.mark.parametrize("prec", [P.PDMTS_FP64, P.PDMTS_FP32_BULK])
def test_coupled_400x64_full_size_properties(fresh, prec):
    """The 100 x 40 mm coupled plate (25,600 PD nodes, 3,030 FE nodes): the
    velocity constraint holds after every coarse step and the state stays finite."""
    cp = W.coupled_plate_400x64()
    g = GpuMTS(fresh(), cp, prec)
    for _ in range(3):
        g.run(5)
        res = g.residual()
        assert res <= (1e-11 if prec == P.PDMTS_FP64 else 1e-5), res
    assert np.isfinite(g.u()).all() and np.isfinite(g.uf()).all()
    info = P.arlequin_info(g.arl)
    print("400x64 coupling:", info)
    assert info["n_lambda"] == 2 * 606


FULL_SIZE = [dict(name="coupled_2000x400", cp=W.coupled_plate_2000x400, steps=20, n_lambda=4020),
             dict(name="coupled3d_400x64x8", cp=W.coupled_plate3d_400x64x8, steps=6, n_lambda=5454)]


@pytest.mark.parametrize("case", FULL_SIZE, ids=[c["name"] for c in FULL_SIZE])
def test_full_size_coupled_fp32_bulk_against_fp64(fresh, case):
    """The benchmark plates at full size, as bench.py runs them (FP32-bulk PD,
    autotuned lattice tiles): after every coarse step the velocity constraint
    holds, and at the end FP32-bulk agrees with the FP64 path (bit-identical
    to the oracle on the parity cases) within the stated tolerances: PD and
    FE displacement rel-L2 <= 1e-4, broken-bond mismatch <= 0.1 %, crack tip
    within one horizon."""
    cp = case["cp"]()
    runs = {}
    for prec in (P.PDMTS_FP64, P.PDMTS_FP32_BULK):
        g = GpuMTS(fresh(), cp, prec)
        for _ in range(case["steps"]):
            g.run(1)
            res = g.residual()
            assert res <= (1e-11 if prec == P.PDMTS_FP64 else 1e-5), (prec, res)
        assert P.arlequin_info(g.arl)["n_lambda"] == case["n_lambda"]
        runs[prec] = dict(u=g.u(), uf=g.uf(), mu=g.mu(), phi=P.pd_read_damage(g.pd))
    a, b = runs[P.PDMTS_FP32_BULK], runs[P.PDMTS_FP64]
    assert np.isfinite(a["u"]).all() and np.isfinite(a["uf"]).all()
    eu, ef = rel_l2(a["u"], b["u"]), rel_l2(a["uf"], b["uf"])
    mm = float(np.count_nonzero(a["mu"] != b["mu"])) / len(b["mu"])
    X = cp.pd.lat.X
    tip = D.tip_error(D.crack_tip(X, a["phi"], 1, 0.020, 0, 6e-3), D.crack_tip(X, b["phi"], 1, 0.020, 0, 6e-3))
    print(f"{case['name']}: rel-L2 u_pd {eu:.2e} u_fe {ef:.2e}, mismatch {mm:.2e}, crack-tip error {tip:.2e} m")
    assert eu <= 1e-4 and ef <= 1e-4 and mm <= 1e-3
    assert tip <= cp.pd.delta


def test_coupled_lattice_tiles_bit_identical(fresh):
    """Coupled FP32-bulk steps on the 100 x 40 mm plate with every lattice tile
    configuration (the link substeps run on windows of tile rows converted per
    tile height), and with the tuned pair of configurations (free chains, link
    chains): identical PD, FE and multiplier states."""
    cp = W.coupled_plate_400x64()
    ref = None
    for tile in [*range(P.PDMTS_LATTICE_TILES), P.PDMTS_LATTICE_TILE_AUTO]:
        g = GpuMTS(fresh(), cp, P.PDMTS_FP32_BULK)
        P.pd_set_lattice_tile(g.pd, tile)
        g.run(4)
        info = P.pd_info(g.pd)
        if tile >= 0:
            assert info["lattice_tile"] == tile and info["link_tile"] == tile
        else:  # tuned separately for the free and the link chains
            assert 0 <= info["lattice_tile"] < P.PDMTS_LATTICE_TILES
            assert 0 <= info["link_tile"] < P.PDMTS_LATTICE_TILES
            print("400x64 tuned tiles: free", info["lattice_tile"], "link", info["link_tile"])
        got = (g.u(), g.v(), g.uf(), g.lam(), g.mu())
        if ref is None:
            ref = got
            continue
        for a, b in zip(got, ref):
            assert np.array_equal(a, b)


def _batch_members():
    return [W.small_coupled(m=2, n_coarse=4, dx=0.25e-3),
            W.small_coupled(m=3, n_coarse=4, dx=0.2e-3, traction=20e6),
            W.small_coupled(m=5, n_coarse=4, dx=0.25e-3, crack=False)]


def test_batch_equals_each_member_alone(fresh):
    """A batch of coupled plates of different sizes, loads and m advanced with one
    launch per substep slot gives every member the bits of its own solo run."""
    cps = _batch_members()
    rounds = 4
    solo = [GpuMTS(fresh(), cp, P.PDMTS_FP32_BULK).run(rounds) for cp in cps]
    members = [GpuMTS(fresh(), cp, P.PDMTS_FP32_BULK) for cp in cps]
    b = P.mts_batch_create([g.ctx for g in members])
    try:
        P.mts_batch_advance(b, 2)
        P.mts_batch_advance(b, rounds - 2)
        info = P.mts_batch_info(b)
    finally:
        P.mts_batch_destroy(b)
    assert info["rounds"] == rounds and info["n_members"] == 3 and info["lattice_tile"] in (0, 1)
    # one batched launch per slot: max(m) slots in each of the free and link phases
    assert info["batched_launches"] == rounds * 2 * max(cp.m for cp in cps)
    for g, s_ in zip(members, solo):
        for a, b_ in [(g.u(), s_.u()), (g.v(), s_.v()), (g.uf(), s_.uf()), (g.vf(), s_.vf()),
                      (g.lam(), s_.lam()), (g.mu(), s_.mu())]:
            assert np.array_equal(a, b_)
        assert g.residual() <= 1e-5
        st = P.pdmts_get_stats(g.ctx)
        assert st["coarse_steps"] == rounds


def _oracle_batch_members():
    return [W.small_coupled(m=2, n_coarse=6, dx=0.25e-3),
            W.small_coupled(m=3, n_coarse=6, dx=0.2e-3, traction=20e6),
            W.small_coupled(m=5, n_coarse=6, dx=0.25e-3, crack=False),
            # m = 20; its interface operator is rebuilt inside the batch (rounds 5 and 6)
            W.small_coupled(m=20, n_coarse=6, dx=0.25e-3, traction=6e6),
            # 70 x 14 lattice: rows not a multiple of 16 bytes of FP32 (nx % 4 != 0)
            W.small_coupled(m=3, n_coarse=6, dx=0.02 / 70)]


def test_batch_members_match_the_oracle(fresh):
    """Every member of a batch of coupled plates (m = 2, 3, 5, 20; lattices of
    80 x 16, 100 x 20 and 70 x 14 nodes; with and without a crack; one member
    whose interface operator is rebuilt inside the batch) advanced by
    mts_batch_advance in FP32-bulk agrees with its own FP64 oracle run of
    Algorithm 1 within the stated FP32-bulk tolerances: PD and FE displacement
    rel-L2 <= 1e-4, broken-bond mismatch <= 0.1 %, velocity-constraint residual
    <= 1e-5."""
    cps = _oracle_batch_members()
    rounds = cps[0].n_coarse
    oracles = [MTSOracle(cp).advance(rounds) for cp in cps]
    members = [GpuMTS(fresh(), cp, P.PDMTS_FP32_BULK) for cp in cps]
    assert members[4].cp.pd.lat.shape[0] % 4 != 0
    b = P.mts_batch_create([g.ctx for g in members])
    try:
        P.mts_batch_advance(b, 2)
        P.mts_batch_advance(b, rounds - 2)
        info = P.mts_batch_info(b)
    finally:
        P.mts_batch_destroy(b)
    assert info["rounds"] == rounds
    assert oracles[3].n_rebuilds > 1 and P.arlequin_info(members[3].arl)["rebuilds"] > 1
    for g, o in zip(members, oracles):
        eu, ef = rel_l2(g.u(), o.u), rel_l2(g.uf(), o.uf)
        ev, el = rel_l2(g.v(), o.v), rel_l2(g.lam(), o.lam)
        mm = np.count_nonzero(g.mu() != o.mu) / len(o.mu)
        print(f"batch member {g.cp.pd.lat.shape} m={g.cp.m}: rel-L2 u_pd {eu:.2e} v_pd {ev:.2e} u_fe {ef:.2e} "
              f"lambda {el:.2e}, mismatch {mm:.2e}, broken {(o.mu == 0).sum()}")
        assert eu <= 1e-4 and ef <= 1e-4 and ev <= 1e-3
        assert mm <= 1e-3
        assert g.residual() <= 1e-5


def test_batch_equals_solo_with_growing_link_windows(fresh):
    """Members of the batched workload's kind (the 100 x 40 mm plate, 16 mm PD
    strip at dx = 0.28 and 0.23 mm, m = 5 and 10): a link run's early
    substeps reach only the rows near the overlap bands, so each substep
    evaluates its own window of rows. Batched, every member gets the bits of
    its solo run, and counts the same bond updates."""
    cps = [W.batch_member(20_000, 0.030, 1.0e7, 5, n_coarse=3), W.batch_member(30_000, 0.045, 1.2e7, 10, n_coarse=3)]
    rounds = 3
    solo = [GpuMTS(fresh(), cp, P.PDMTS_FP32_BULK).run(rounds) for cp in cps]
    members = [GpuMTS(fresh(), cp, P.PDMTS_FP32_BULK) for cp in cps]
    b = P.mts_batch_create([g.ctx for g in members])
    try:
        P.mts_batch_advance(b, rounds)
    finally:
        P.mts_batch_destroy(b)
    for g, s_ in zip(members, solo):
        for a, b_ in [(g.u(), s_.u()), (g.v(), s_.v()), (g.uf(), s_.uf()), (g.lam(), s_.lam()), (g.mu(), s_.mu())]:
            assert np.array_equal(a, b_)
        assert P.pdmts_get_stats(g.ctx)["bond_updates"] == P.pdmts_get_stats(s_.ctx)["bond_updates"]


def test_batch_rejects_unsupported_members(fresh):
    cp = W.small_coupled(m=2, n_coarse=2)
    g64 = GpuMTS(fresh(), cp, P.PDMTS_FP64)
    with pytest.raises(P.PdmtsError) as e:
        P.mts_batch_create([g64.ctx])
    assert e.value.code == -8  # PDMTS_ERR_UNSUPPORTED
    g = GpuMTS(fresh(), cp, P.PDMTS_FP32_BULK)
    with pytest.raises(P.PdmtsError):
        P.mts_batch_create([g.ctx, g.ctx])


def test_batch_members_alone_in_between_and_dropped(fresh):
    """A member advanced alone between batch calls, and a member whose coupling is
    destroyed while in the batch: the others still match their solo runs."""
    cps = _batch_members()
    solo = [GpuMTS(fresh(), cp, P.PDMTS_FP32_BULK) for cp in cps]
    solo[0].run(2 + 1 + 2)
    solo[1].run(2 + 2)
    members = [GpuMTS(fresh(), cp, P.PDMTS_FP32_BULK) for cp in cps]
    b = P.mts_batch_create([g.ctx for g in members])
    try:
        P.mts_batch_advance(b, 2)
        members[0].run(1)                      # alone, between batch calls
        P.arlequin_destroy(members[2].arl)     # the member leaves the batch
        P.mts_batch_advance(b, 2)
        assert P.mts_batch_info(b)["n_members"] == 2
    finally:
        P.mts_batch_destroy(b)
    for g, s_ in zip(members[:2], solo[:2]):
        assert np.array_equal(g.u(), s_.u()) and np.array_equal(g.uf(), s_.uf())
        assert np.array_equal(g.lam(), s_.lam()) and np.array_equal(g.mu(), s_.mu())


CASES3D = [
    dict(name="3d_linear_m3", cp=lambda: W.small_coupled3d(m=3, n_coarse=6)),
    dict(name="3d_cubic_m2_breaking", cp=lambda: W.small_coupled3d(m=2, n_coarse=6, weight_kind=2, traction=40e6)),
]


@pytest.mark.parametrize("case", CASES3D, ids=[c["name"] for c in CASES3D])
def test_mts3d_fp64_matches_oracle(fresh, case):
    """3D coupling (bond-based PD through the thickness, Hex8 FE): FP64 parity
    with the oracle's Algorithm 1."""
    cp = case["cp"]()
    o = MTSOracle(cp).advance(cp.n_coarse)
    g = GpuMTS(fresh(), cp, P.PDMTS_FP64).run(cp.n_coarse)
    _compare(g, o, FP64_TOL, 1e-8)
    assert P.arlequin_info(g.arl)["rebuilds"] == o.n_rebuilds
    assert g.residual() <= 1e-12


def test_mts3d_fp32_bulk_within_tolerance(fresh):
    cp = W.small_coupled3d(m=3, n_coarse=6)
    o = MTSOracle(cp).advance(cp.n_coarse)
    g = GpuMTS(fresh(), cp, P.PDMTS_FP32_BULK).run(cp.n_coarse)
    mm = np.count_nonzero(g.mu() != o.mu) / len(o.mu)
    print(f"MTS 3D fp32-bulk: rel-L2 u_pd {rel_l2(g.u(), o.u):.2e}, u_fe {rel_l2(g.uf(), o.uf):.2e}, mismatch {mm:.2e}")
    assert rel_l2(g.u(), o.u) <= 1e-4 and rel_l2(g.uf(), o.uf) <= 1e-4
    assert mm <= 1e-3
    assert g.residual() <= 1e-5


def test_mts3d_uniform_velocity_patch(fresh):
    cp = W.small_coupled3d(m=2, n_coarse=3, crack=False, traction=0.0)
    v0 = np.array([1.0, -2.0, 0.5])
    g = GpuMTS(fresh(), cp, P.PDMTS_FP64, v0=v0).run(3)
    assert np.abs(g.v() - v0.reshape(3, 1)).max() <= 1e-12 * 2.0
    assert np.abs(g.vf() - np.repeat(v0, cp.fe.n)).max() <= 1e-12 * 2.0
