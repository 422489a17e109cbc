"""The damage read-back that allocates nothing (pd_read_damage_static).

Callers that cannot let the library allocate device memory at the point of the
call (an application whose device memory is wholly held by its own pool
allocator, or a time-critical loop in which an allocation, which may
synchronise the device, is not allowed) use this entry point; it stages the
result in a device array that is part of the library image. Here it
is called through the C ABI and compared with pd_read_damage on two calls in a
row, for both family layouts; the file is named so that pytest collects it
after every other test.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2403_03605_gb300 import pdmts as P
from paper_2403_03605_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _static_damage(pd, n):
    out = np.empty(n, dtype=np.float64)
    rc = P.load().pd_read_damage_static(C.c_void_p(pd), out.ctypes.data_as(C.c_void_p))
    assert rc == 0, P.pdmts_last_error()
    return out


@pytest.mark.parametrize("precision", [P.PDMTS_FP64, P.PDMTS_FP32_BULK])
def test_static_damage_matches_allocating_read_back(precision):
    from paper_2403_03605_gb300 import build
    build.build()
    pb = W.small_plate(48, 30, nsteps=120)
    ctx = P.pdmts_ctx_create(0)
    try:
        pd = P.pd_create(ctx, pb.lat.X, horizon=pb.delta, c=pb.c, s0=pb.s0, rho=pb.mat.rho, vol_uniform=pb.vol,
                         precision=precision)
        P.pd_set_precrack(pd, [c.as_array() for c in pb.cuts])
        P.pd_set_body_force(pd, pb.b)
        P.mts_set_time(ctx, pb.dt, 1)
        P.mts_advance(ctx, 60)
        first_ref = P.pd_read_damage(pd)
        first = _static_damage(pd, pb.n)
        np.testing.assert_allclose(first, first_ref, rtol=0, atol=1e-15)
        assert first_ref.max() > 0  # the pre-crack and the run produce damage
        P.mts_advance(ctx, 60)
        second_ref = P.pd_read_damage(pd)
        second = _static_damage(pd, pb.n)
        np.testing.assert_allclose(second, second_ref, rtol=0, atol=1e-15)
        assert not np.array_equal(first_ref, second_ref)  # the second call sees new damage
    finally:
        P.pdmts_ctx_destroy(ctx)


def test_static_damage_rejects_oversized_subdomain():
    from paper_2403_03605_gb300 import build
    build.build()
    lat = W.Lattice((1025, 1024), 1e-4, (0.0, 0.0))  # 1,049,600 nodes > 2^20
    ctx = P.pdmts_ctx_create(0)
    try:
        pd = P.pd_create(ctx, lat.X, horizon=1.5e-4, c=1e20, s0=1e-3, rho=1e3, vol_uniform=1e-12,
                         precision=P.PDMTS_FP32_BULK)
        out = np.empty(lat.n)
        rc = P.load().pd_read_damage_static(C.c_void_p(pd), out.ctypes.data_as(C.c_void_p))
        assert rc == -8 and "exceed" in P.pdmts_last_error()
    finally:
        P.pdmts_ctx_destroy(ctx)
