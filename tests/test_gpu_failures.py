"""Failures made on the host come back as status codes and leave the library
usable (no GPU fault is provoked): a device allocator that refuses, NaN/Inf
inputs, and a body force rejected between steps without touching the state."""
import numpy as np
import pytest

from gpu_common import GpuPDRun
from paper_2403_03605_gb300 import pdmts as P
from paper_2403_03605_gb300 import workloads as W

pytestmark = pytest.mark.gpu

PDMTS_ERR_ARG, PDMTS_ERR_NOMEM = -1, -7
_KEEP = []  # allocator callbacks must outlive the contexts that call them


class BudgetAllocator:
    """Device memory from PyTorch's caching allocator until `left` runs out,
    then NULL (an out-of-memory condition made on the host)."""

    def __init__(self, left, stream):
        import torch
        self.torch = torch
        self.left = left
        self.stream = stream
        self.alloc = P.ALLOC_FN(self._alloc)
        self.free = P.FREE_FN(self._free)

    def _alloc(self, size, user):
        if self.left <= 0:
            return None
        self.left -= 1
        return self.torch.cuda.caching_allocator_alloc(int(size), 0, self.stream)

    def _free(self, ptr, user):
        self.torch.cuda.caching_allocator_delete(ptr)


@pytest.fixture
def fresh():
    from paper_2403_03605_gb300 import build
    build.build()
    made = []

    def mk(**kw):
        c = P.pdmts_ctx_create(0, **kw)
        made.append(c)
        return c
    yield mk
    for c in made:
        P.pdmts_ctx_destroy(c)


def test_allocation_failure_is_reported_and_recoverable(fresh):
    import torch
    stream = torch.cuda.current_stream(0).cuda_stream
    ctx = fresh(torch_allocator=False)
    al = BudgetAllocator(2, stream)
    _KEEP.append(al)
    assert P.load().pdmts_set_allocator(ctx, al.alloc, al.free, None) == 0
    pb = W.small_plate(40, 24, nsteps=20)
    with pytest.raises(P.PdmtsError) as e:
        P.pd_create(ctx, pb.lat.X, horizon=pb.delta, c=pb.c, s0=pb.s0, rho=pb.mat.rho, vol_uniform=pb.vol)
    assert e.value.code == PDMTS_ERR_NOMEM
    # with memory available again the same context sets the problem up and runs
    al.left = 10 ** 9
    pd = P.pd_create(ctx, pb.lat.X, horizon=pb.delta, c=pb.c, s0=pb.s0, rho=pb.mat.rho, vol_uniform=pb.vol)
    P.pd_set_precrack(pd, [c.as_array() for c in pb.cuts])
    P.pd_set_body_force(pd, pb.b)
    P.mts_set_time(ctx, pb.dt, 1)
    P.mts_advance(ctx, 20)
    ref = GpuPDRun(fresh(), pb, P.PDMTS_FP64).run(20)  # the default allocator
    assert np.array_equal(P.pd_read_displacement(pd), ref.u())


def test_non_finite_inputs_are_rejected_and_leave_the_state(fresh):
    pb = W.small_plate(40, 24, nsteps=40)
    X = pb.lat.X.copy()
    X[0, 5] = np.nan
    with pytest.raises(P.PdmtsError) as e:
        P.pd_create(fresh(), X, horizon=pb.delta, c=pb.c, s0=pb.s0, rho=pb.mat.rho, vol_uniform=pb.vol)
    assert e.value.code == PDMTS_ERR_ARG
    for prec in (P.PDMTS_FP64, P.PDMTS_FP32_BULK):
        a = GpuPDRun(fresh(), pb, prec).run(20)
        b = GpuPDRun(fresh(), pb, prec).run(20)
        bad = pb.b.copy()
        bad[1, 7] = np.inf
        with pytest.raises(P.PdmtsError) as e:
            P.pd_set_body_force(b.pd, bad)
        assert e.value.code == PDMTS_ERR_ARG
        bad[1, 7] = np.nan
        with pytest.raises(P.PdmtsError):
            P.pd_set_body_force(b.pd, bad)
        a.run(20)
        b.run(20)  # the rejected loads left the previous ones in place
        assert np.array_equal(a.u(), b.u()) and np.array_equal(a.mu(), b.mu())


PDMTS_ERR_TIMEOUT = -5


def test_bounded_tensor_copy_wait_gives_up_and_recovers(fresh):
    """A bounded wait that runs out, made without a fault: the first tensor-copy
    wait of every lattice tile gets a poll limit of 0 (a wait that nothing can
    satisfy in time), so each tile gives up, drains its copies with the full
    limit and returns without writing. The next blocking call reports
    PDMTS_ERR_TIMEOUT; advancing, the statistics and saving a checkpoint are
    refused while the state is undefined; loading the image saved before the
    give-up makes the context usable again, and it continues with the bits of
    an uninterrupted run."""
    pb = W.small_plate(48, 30, nsteps=40)  # nx % 4 == 0: the tensor-copy tile configuration applies
    ref = GpuPDRun(fresh(), pb, P.PDMTS_FP32_BULK)
    P.pd_set_lattice_tile(ref.pd, 5)
    ref.run(30)
    g = GpuPDRun(fresh(), pb, P.PDMTS_FP32_BULK)
    P.pd_set_lattice_tile(g.pd, 5)
    g.run(20)
    image = P.mts_state_save(g.ctx)
    P.pdmts_set_debug_poll_limit(g.ctx, 0)
    P.mts_advance(g.ctx, 1)  # queued; its tiles give up on the device
    with pytest.raises(P.PdmtsError) as e:
        g.u()
    assert e.value.code == PDMTS_ERR_TIMEOUT and "gave up" in str(e.value)
    for call in (lambda: P.mts_advance(g.ctx, 1), lambda: P.pdmts_get_stats(g.ctx),
                 lambda: P.mts_state_save(g.ctx), lambda: P.pd_read_damage(g.pd)):
        with pytest.raises(P.PdmtsError) as e:
            call()
        assert e.value.code == PDMTS_ERR_TIMEOUT
    P.pdmts_set_debug_poll_limit(g.ctx, -1)
    P.mts_state_load(g.ctx, image)
    g.run(10)
    assert np.array_equal(g.u(), ref.u()) and np.array_equal(g.v(), ref.v())
    assert np.array_equal(g.mu(), ref.mu())
    assert P.pd_info(g.pd)["lattice_tile"] == 5
    P.pdmts_get_stats(g.ctx)  # usable again
