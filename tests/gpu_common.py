"""Helpers shared by the GPU tests: set the same problem up on the oracle and
on the CUDA library, both from the seeded workload generators."""
import numpy as np

import oracle
from paper_2403_03605_gb300 import pdmts as P
from paper_2403_03605_gb300 import workloads as W


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    den = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / den) if den > 0 else float(np.linalg.norm(a - b))


class OracleRun:
    """A PD problem advanced by the FP64 CPU oracle."""

    def __init__(self, pb: W.PDProblem, *, alpha=None, micro=oracle.MICRO_POWER, l=0.0, c=None,
                 force=oracle.FORCE_LINEAR, breaking=True, u0=None, v0=None, body=True):
        self.pb = pb
        self.rp, self.col = oracle.family(pb.lat.X, pb.delta)
        if pb.cuts:
            self.mu, self.ncut = oracle.precrack(pb.lat.P, self.rp, self.col,
                                                 [cc.in_half_units(pb.lat) for cc in pb.cuts])
        else:
            self.mu, self.ncut = np.ones(len(self.col), np.uint8), 0
        self.pd = oracle.PD(pb.lat.X, pb.vol, pb.delta, pb.c if c is None else c, pb.s0, pb.mat.rho, pb.dt,
                            micro=micro, l=l, force=force, breaking=breaking)
        self.alpha = alpha
        self.b = pb.b if body else None
        self.u = np.zeros((pb.dim, pb.n)) if u0 is None else np.array(u0, dtype=np.float64)
        self.v = np.zeros((pb.dim, pb.n)) if v0 is None else np.array(v0, dtype=np.float64)
        self.a = np.zeros((pb.dim, pb.n))
        self.inited = False
        self.broken = 0

    def run(self, nsteps):
        self.broken += oracle.pd_run(self.pd, self.rp, self.col, self.mu, self.u, self.v, self.a, nsteps,
                                     alpha=self.alpha, b=self.b, init=not self.inited)
        self.inited = True
        return self

    def damage(self):
        return oracle.damage(self.pd, self.rp, self.col, self.mu)


class GpuPDRun:
    """The same PD problem advanced by libpdmts.so through the C ABI."""

    def __init__(self, ctx, pb: W.PDProblem, precision, *, micro=P.PDMTS_MICRO_POWER, l=0.0, c=None,
                 force=P.PDMTS_FORCE_LINEAR, breaking=True, u0=None, v0=None, body=True, alpha=None):
        self.ctx = ctx
        self.pb = pb
        self.pd = P.pd_create(ctx, pb.lat.X, horizon=pb.delta, c=pb.c if c is None else c, s0=pb.s0,
                              rho=pb.mat.rho, vol_uniform=pb.vol, micro_kind=micro, l=l, precision=precision)
        if pb.cuts:
            P.pd_set_precrack(self.pd, [cc.as_array() for cc in pb.cuts])
        if body:
            P.pd_set_body_force(self.pd, pb.b)
        if alpha is not None:
            P.pd_set_weights(self.pd, alpha)
        P.pd_set_breaking(self.pd, breaking)
        P.pd_set_force_law(self.pd, force)
        if u0 is not None or v0 is not None:
            P.pd_set_state(self.pd, u0, v0)
        P.mts_set_time(ctx, pb.dt, 1)

    def run(self, nsteps):
        P.mts_advance(self.ctx, nsteps)
        return self

    def u(self):
        return P.pd_read_displacement(self.pd)

    def v(self):
        return P.pd_read_velocity(self.pd)

    def a(self):
        return P.pd_read_acceleration(self.pd)

    def mu(self):
        return P.pd_read_bond_status(self.pd)[0]

    def damage(self):
        return P.pd_read_damage(self.pd)


class GpuMTS:
    """A coupled problem advanced by libpdmts.so (Algorithm 1) through the C ABI."""

    def __init__(self, ctx, cp, precision, v0=None):
        self.ctx, self.cp = ctx, cp
        pb = cp.pd
        mat = pb.mat
        self.pd = P.pd_create(ctx, pb.lat.X, horizon=pb.delta, c=pb.c, s0=pb.s0, rho=mat.rho, vol_uniform=pb.vol,
                              micro_kind=pb.extra.get("micro", P.PDMTS_MICRO_POWER), l=pb.extra.get("l", 0.0),
                              precision=precision)
        if pb.cuts:
            P.pd_set_precrack(self.pd, [c.as_array() for c in pb.cuts])
        self.fe = P.fem_create(ctx, cp.fe.X, cp.fe.conn, E=mat.E, nu=mat.nu, rho=mat.rho, thickness=mat.thickness)
        P.fem_set_traction(self.fe, cp.faces, cp.face_traction)
        if cp.fixed is not None:
            P.fem_set_fixed(self.fe, cp.fixed)
        self.arl = P.arlequin_bind(ctx, self.pd, self.fe, cp.weight_kind, [b.as_array() for b in cp.bands])
        dim = pb.lat.dim
        if v0 is not None:
            v0 = np.asarray(v0, dtype=np.float64)
            P.pd_set_state(self.pd, None, np.repeat(v0.reshape(dim, 1), pb.n, axis=1))
            P.fem_set_state(self.fe, None, np.repeat(v0, cp.fe.n))
        P.mts_set_time(ctx, cp.dt_pd, cp.m, cp.gamma_fe, cp.beta_fe)
        self.ndof = dim * cp.fe.n

    def run(self, n):
        P.mts_advance(self.ctx, n)
        return self

    def u(self):
        return P.pd_read_displacement(self.pd)

    def v(self):
        return P.pd_read_velocity(self.pd)

    def mu(self):
        return P.pd_read_bond_status(self.pd)[0]

    def uf(self):
        return P.fem_read_displacement(self.fe, self.ndof)

    def vf(self):
        return P.fem_read_velocity(self.fe, self.ndof)

    def lam(self):
        return P.arlequin_read_lambda(self.arl)

    def residual(self):
        r, f = P.arlequin_constraint_residual(self.arl)
        return r / f if f > 0 else r
