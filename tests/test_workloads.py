"""The seeded batched benchmark (64 coupled plates of uneven size) as specified."""
import numpy as np

from paper_2403_03605_gb300 import workloads as W


def test_batch_draws_follow_the_stated_distributions():
    d = W.batch_plates_draws()
    assert len(d) == 64
    N = np.array([x[0] for x in d])
    crack = np.array([x[1] for x in d])
    T = np.array([x[2] for x in d])
    m = np.array([x[3] for x in d])
    assert N.min() >= 20_000 and N.max() <= 400_000
    assert crack.min() >= 0.020 and crack.max() <= 0.060
    assert T.min() >= 6e6 and T.max() <= 15e6
    assert set(m.tolist()) <= {5, 10, 20} and len(set(m.tolist())) == 3
    assert W.batch_plates_draws() == d  # seeded
    # about 13.6 million PD nodes in total
    assert 12e6 < N.sum() < 15e6


def test_batch_member_geometry():
    for N in (20_000, 400_000):
        cp = W.batch_member(N, 0.03, 1e7, 10)
        assert abs(cp.pd.n - N) / N < 0.02
        # PD strip 16 mm tall, FE bands overlapping it by 2 mm, dt below the stable bound
        y = cp.pd.lat.X[1]
        assert abs((y.max() - y.min()) + cp.pd.lat.dx - 0.016) < 1.5 * cp.pd.lat.dx
        assert cp.dt_pd <= 0.41 * W.DT_CRIT_PER_M * cp.pd.lat.dx
        assert np.allclose([b.lo for b in cp.bands], [0.012, 0.026])


def test_edge_traction_layer_carries_the_traction():
    """The traction of the pure-PD plates enters as a body force on the node rows
    within delta of each loaded face: at delta = 3.015 dx that is k = 3 rows per
    face, and each layer carries exactly T L h (2D; T L_x L_z in 3D) along the
    outward normal, with nothing elsewhere."""
    T, dx, h = 12e6, 0.5e-3, 1e-3
    lat = W.Lattice((40, 24), dx, (0.0, 0.0))
    delta = W.HORIZON_FACTOR * dx
    b = W.edge_traction_body_force(lat, T, delta)
    rows = lat.idx[1]
    V = h * dx * dx
    L = 40 * dx
    bottom, top = rows < 3, rows >= 24 - 3
    assert np.count_nonzero(b[1]) == 2 * 3 * 40 and not b[0].any()
    assert not b[1][(rows >= 3) & (rows < 21)].any()
    assert np.isclose((b[1][bottom] * V).sum(), -T * L * h, rtol=1e-13)
    assert np.isclose((b[1][top] * V).sum(), T * L * h, rtol=1e-13)
    # the fourth row's centre (3.5 dx) lies beyond delta; the third's (2.5 dx) within
    assert 2.5 * dx <= delta < 3.5 * dx
    lat3 = W.Lattice((12, 10, 4), dx, (0.0, 0.0, 0.0))
    b3 = W.edge_traction_body_force(lat3, T, delta)
    r3 = lat3.idx[1]
    assert np.isclose((b3[1][r3 >= 10 - 3] * dx ** 3).sum(), T * (12 * dx) * (4 * dx), rtol=1e-13)
    assert np.count_nonzero(b3[1]) == 2 * 3 * 12 * 4 and not b3[0].any() and not b3[2].any()
