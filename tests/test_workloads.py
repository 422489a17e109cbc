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
