"""Checkpoint / resume through the C ABI: a context saved after some coarse
steps and loaded into a fresh context with the same set-up continues with the
same bits as the saved context (PD, FE, multiplier and bond state), in FP64
and FP32-bulk, with bond breaking and interface rebuilds."""
import numpy as np
import pytest

from gpu_common import GpuMTS, GpuPDRun
from paper_2403_03605_gb300 import pdmts as P
from paper_2403_03605_gb300 import workloads as W

pytestmark = pytest.mark.gpu


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


def _coupled_state(g):
    return (g.u(), g.v(), P.pd_read_acceleration(g.pd), g.uf(), g.vf(), g.lam(), g.mu())


COUPLED = [dict(name="fp64_breaking_rebuilds", cp=lambda: W.small_coupled(m=4, n_coarse=12, traction=30e6),
                prec=P.PDMTS_FP64, before=5, after=6),
           dict(name="fp32_bulk_plate_25600", cp=W.coupled_plate_400x64, prec=P.PDMTS_FP32_BULK, before=3, after=4)]


@pytest.mark.parametrize("case", COUPLED, ids=[c["name"] for c in COUPLED])
def test_coupled_resume_bit_identical(fresh, case):
    cp = case["cp"]()
    a = GpuMTS(fresh(), cp, case["prec"]).run(case["before"])
    image = P.mts_state_save(a.ctx)
    a.run(case["after"])
    b = GpuMTS(fresh(), cp, case["prec"])
    P.mts_state_load(b.ctx, image)
    b.run(case["after"])
    for x, y in zip(_coupled_state(b), _coupled_state(a)):
        assert np.array_equal(x, y)
    assert P.pd_info(b.pd)["steps_done"] == P.pd_info(a.pd)["steps_done"]
    assert b.residual() <= (1e-12 if case["prec"] == P.PDMTS_FP64 else 1e-5)


@pytest.mark.parametrize("prec", [P.PDMTS_FP64, P.PDMTS_FP32_BULK])
def test_pure_pd_resume_bit_identical(fresh, prec):
    pb = W.small_plate(40, 24, nsteps=80)
    a = GpuPDRun(fresh(), pb, prec).run(40)
    image = P.mts_state_save(a.ctx)
    a.run(40)
    b = GpuPDRun(fresh(), pb, prec)
    P.mts_state_load(b.ctx, image)
    b.run(40)
    for x, y in [(b.u(), a.u()), (b.v(), a.v()), (b.a(), a.a()), (b.mu(), a.mu())]:
        assert np.array_equal(x, y)


def test_load_rejects_other_set_up(fresh):
    pb = W.small_plate(40, 24, nsteps=10)
    a = GpuPDRun(fresh(), pb, P.PDMTS_FP64).run(3)
    image = P.mts_state_save(a.ctx)
    other = GpuPDRun(fresh(), pb, P.PDMTS_FP32_BULK)
    with pytest.raises(P.PdmtsError):
        P.mts_state_load(other.ctx, image)
    with pytest.raises(P.PdmtsError):
        P.mts_state_load(a.ctx, image[:-8])
    bigger = GpuPDRun(fresh(), W.small_plate(41, 24, nsteps=10), P.PDMTS_FP64)
    with pytest.raises(P.PdmtsError):
        P.mts_state_load(bigger.ctx, image)
