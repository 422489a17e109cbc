"""FP64 CPU oracle of the multi-time-step Arlequin coupling (test infrastructure only).

Follows arXiv 2403.03605 Sec. 2.2-2.5 step by step:
  * finite elements (Eq. 24 ff.): bilinear Q4 with plane stress D (Eq. 9) and
    2 x 2 Gauss points, or trilinear Hex8 with the 3D isotropic D and 2 x 2 x 2
    Gauss points; stiffness and lumped mass weighted by the Arlequin weight
    alpha and loads by alpha (Eq. 34);
  * PD subdomain weighted by 1 - alpha (Eq. 17, Eq. 34), stepped by the C oracle
    (velocity Verlet, Eq. 38 with gamma = 1/2, beta = 0);
  * velocity constraint G_FE v_FE - G_PD v_PD = 0 (Eq. 33, Eq. 41) with the
    multiplier on the finite-element nodes of the overlap;
  * Newmark for the finite elements (Eq. 39), m PD substeps per coarse step
    (Eq. 40) with the multiplier interpolated linearly (Eq. 42);
  * free / link split (Eq. 47-48), unit-load responses (Eq. unit), interface
    problem for lambda_m (Eq. 49), correction U = V + Y lambda_m and
    Algorithm 1's loop.

Readings of points the paper leaves open or garbles:
  * Signs are taken from Eq. 33: the FE equation carries +G_FE^T lambda, the PD
    equation -G_PD^T lambda, the constraint G_FE v_FE - G_PD v_PD = 0. Eq. 43-49
    are then derived from these (their printed signs disagree with Eq. 33).
  * The free-problem multiplier term is S_j = (1 - j/m) lambda_0 (the load
    bracket printed with S_j vanishes for the constant loads used here).
  * Non-matching meshes: lambda lives on the FE nodes of the overlap;
    G_FE[k, I] = int_O N_k N_I dV (Gauss), G_PD[k, p] = N_k(x_p) V_p.
  * The link problem (Eq. 48b) uses the bond state at the start of the coarse
    step and never breaks bonds; the unit responses (and H) are rebuilt after a
    step in which a bond within (m + 1) delta of an overlap band broke.
  * lambda_0 = 0 at t = 0.
  * Weights (Sec. 3.2): with t = distance to the FE boundary / overlap width,
    alpha = t (linear), t^3 (cubic) or 1/2 (constant) inside a band; 1 on the
    FE-only side, 0 on the PD-only side.
  * Dirichlet dofs (the beam's fixed end, Sec. 3.2) are eliminated: Newmark
    solves for the free dofs only and the fixed ones stay zero.

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may use it.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import (MICRO_POWER, PD, damage, family, pd_forces, pd_run, precrack)

GAUSS = np.array([-1.0, 1.0]) / np.sqrt(3.0)
NAT = np.array([[-1.0, -1.0], [1.0, -1.0], [1.0, 1.0], [-1.0, 1.0]])  # Q4 node natural coordinates
# Hex8 corners: bottom face (zeta = -1) counter-clockwise seen from +z, then the top face
NAT3 = np.array([[-1.0, -1.0, -1.0], [1.0, -1.0, -1.0], [1.0, 1.0, -1.0], [-1.0, 1.0, -1.0],
                 [-1.0, -1.0, 1.0], [1.0, -1.0, 1.0], [1.0, 1.0, 1.0], [-1.0, 1.0, 1.0]])


def band_weight(x, bands, kind, outside):
    """Arlequin weight alpha at points x (dim, n) (Sec. 3.2)."""
    x = np.asarray(x)
    a = np.full(x.shape[1], float(outside))
    for b in bands:
        c = x[b.axis]
        inside = (c >= b.lo) & (c <= b.hi)
        t = (b.hi - c) / (b.hi - b.lo) if b.fe_side < 0 else (c - b.lo) / (b.hi - b.lo)
        if kind == 0:
            w = np.full_like(t, 0.5)
        elif kind == 1:
            w = t
        else:
            w = t ** 3
        a = np.where(inside, w, a)
    return a


def q4_shape(xi, eta):
    N = 0.25 * (1 + NAT[:, 0] * xi) * (1 + NAT[:, 1] * eta)
    dxi = 0.25 * NAT[:, 0] * (1 + NAT[:, 1] * eta)
    deta = 0.25 * NAT[:, 1] * (1 + NAT[:, 0] * xi)
    return N, dxi, deta


def hex8_shape(xi, eta, zeta):
    """Trilinear shape functions and their natural derivatives (8,), (3, 8)."""
    p = 1 + NAT3[:, 0] * xi
    q = 1 + NAT3[:, 1] * eta
    r = 1 + NAT3[:, 2] * zeta
    N = p * q * r / 8
    dN = np.stack([NAT3[:, 0] * q * r, NAT3[:, 1] * p * r, NAT3[:, 2] * p * q]) / 8
    return N, dN


def hex8_gauss(xe):
    """Yield (N, physical derivatives (3, 8), detJ, point) at the 2 x 2 x 2 Gauss points of xe (3, 8)."""
    for gx in GAUSS:
        for gy in GAUSS:
            for gz in GAUSS:
                N, dN = hex8_shape(gx, gy, gz)
                J = dN @ xe.T  # J[i, j] = d x_j / d xi_i
                yield N, np.linalg.solve(J, dN), np.linalg.det(J), xe @ N


class FE:
    """Alpha-weighted discretisation of the CCM subdomain (Eq. 24 ff., Eq. 34):
    Q4 plane stress in 2D, Hex8 isotropic linear elasticity in 3D."""

    def __init__(self, mesh, E, nu, rho, thick, bands, kind, faces, face_traction):
        self.X = np.asarray(mesh.X, dtype=np.float64)
        self.conn = np.asarray(mesh.conn, dtype=np.int64)
        n = self.X.shape[1]
        self.n = n
        self.dim = self.X.shape[0]
        if self.dim == 3:
            self._init3d(E, nu, rho, bands, kind, faces, face_traction)
            return
        D = E / (1 - nu * nu) * np.array([[1, nu, 0], [nu, 1, 0], [0, 0, (1 - nu) / 2]])
        rows, cols, vals = [], [], []
        mass = np.zeros(n)
        for e, nodes in enumerate(self.conn):
            xe = self.X[:, nodes]  # (2, 4)
            ke = np.zeros((8, 8))
            for gx in GAUSS:
                for gy in GAUSS:
                    N, dxi, deta = q4_shape(gx, gy)
                    J = np.array([[dxi @ xe[0], dxi @ xe[1]], [deta @ xe[0], deta @ xe[1]]])
                    detJ = np.linalg.det(J)
                    dN = np.linalg.solve(J, np.stack([dxi, deta]))  # (2, 4): d/dx, d/dy
                    B = np.zeros((3, 8))
                    B[0, 0::2] = dN[0]
                    B[1, 1::2] = dN[1]
                    B[2, 0::2] = dN[1]
                    B[2, 1::2] = dN[0]
                    xg = xe @ N
                    al = band_weight(xg.reshape(2, 1), bands, kind, 1.0)[0]
                    ke += al * (B.T @ D @ B) * detJ * thick
                    mass[nodes] += al * rho * N * detJ * thick
            dof = np.stack([nodes, nodes + n], axis=1).reshape(-1)  # [x0, y0, x1, y1, ...] -> SoA ids
            for a in range(8):
                for b in range(8):
                    rows.append(dof[a]); cols.append(dof[b]); vals.append(ke[a, b])
        self.K = sp.csr_matrix((vals, (rows, cols)), shape=(2 * n, 2 * n))
        self.M = np.concatenate([mass, mass])  # lumped, per dof (SoA: x block, y block)
        P = np.zeros(2 * n)
        for (i, j), t in zip(np.asarray(faces), np.asarray(face_traction)):
            L = np.linalg.norm(self.X[:, j] - self.X[:, i])
            xm = 0.5 * (self.X[:, i] + self.X[:, j])
            al = band_weight(xm.reshape(2, 1), bands, kind, 1.0)[0]
            for node in (i, j):
                P[node] += al * t[0] * L * thick / 2
                P[node + n] += al * t[1] * L * thick / 2
        self.P = P

    def _init3d(self, E, nu, rho, bands, kind, faces, face_traction):
        n = self.n
        lam = E * nu / ((1 + nu) * (1 - 2 * nu))
        mu = E / (2 * (1 + nu))
        D = np.zeros((6, 6))
        D[:3, :3] = lam
        D[[0, 1, 2], [0, 1, 2]] = lam + 2 * mu
        D[[3, 4, 5], [3, 4, 5]] = mu
        rows, cols, vals = [], [], []
        mass = np.zeros(n)
        for nodes in self.conn:
            xe = self.X[:, nodes]  # (3, 8)
            ke = np.zeros((24, 24))
            for N, dNx, detJ, xg in hex8_gauss(xe):
                B = np.zeros((6, 24))  # strains xx, yy, zz, yz, xz, xy; local dof a * 3 + d
                B[0, 0::3] = dNx[0]
                B[1, 1::3] = dNx[1]
                B[2, 2::3] = dNx[2]
                B[3, 1::3] = dNx[2]; B[3, 2::3] = dNx[1]
                B[4, 0::3] = dNx[2]; B[4, 2::3] = dNx[0]
                B[5, 0::3] = dNx[1]; B[5, 1::3] = dNx[0]
                al = band_weight(xg.reshape(3, 1), bands, kind, 1.0)[0]
                ke += al * (B.T @ D @ B) * detJ
                mass[nodes] += al * rho * N * detJ
            dof = np.stack([nodes, nodes + n, nodes + 2 * n], axis=1).reshape(-1)
            for a in range(24):
                for b in range(24):
                    rows.append(dof[a]); cols.append(dof[b]); vals.append(ke[a, b])
        self.K = sp.csr_matrix((vals, (rows, cols)), shape=(3 * n, 3 * n))
        self.M = np.concatenate([mass, mass, mass])
        P = np.zeros(3 * n)
        for fn, t in zip(np.asarray(faces), np.asarray(face_traction)):
            xf = self.X[:, fn]  # (3, 4), corners in order around the face
            area = 0.5 * np.linalg.norm(np.cross(xf[:, 2] - xf[:, 0], xf[:, 3] - xf[:, 1]))
            al = band_weight(xf.mean(axis=1).reshape(3, 1), bands, kind, 1.0)[0]
            for node in fn:
                for d in range(3):
                    P[node + d * n] += al * t[d] * area / 4
        self.P = P


class Newmark:
    """K_eff = M + beta dt^2 K (Eq. 39) on the free dofs: solve() returns the
    acceleration increment of a right-hand side with the fixed dofs at zero."""

    def __init__(self, fe, dt, beta, fixed=None):
        nd = fe.dim * fe.n
        self.fixed = np.unique(np.asarray([] if fixed is None else fixed, dtype=np.int64))
        free = np.ones(nd, bool)
        free[self.fixed] = False
        self.free = np.nonzero(free)[0]
        self.nd = nd
        self.fe = fe
        Keff = (sp.diags(fe.M) + beta * dt ** 2 * fe.K).tocsr()[self.free][:, self.free]
        self.lu = spla.splu(Keff.tocsc())

    def solve(self, r):
        x = np.zeros(self.nd)
        x[self.free] = self.lu.solve(np.asarray(r)[self.free])
        return x

    def initial_acceleration(self, u):
        a = (self.fe.P - self.fe.K @ u) / self.fe.M
        a[self.fixed] = 0.0
        return a


def newmark_fe(fp, n_steps, record):
    """Undecomposed finite-element reference (Table 1, cases 1 and 2): the
    whole body as one FE subdomain (alpha = 1), Newmark with gamma, beta of
    `fp` (beta = 0 with the lumped mass is the explicit scheme), fixed dofs
    eliminated, starting at rest under the constant traction load. Returns
    u at the dof ids `record` after each step, (n_steps, len(record))."""
    mat = fp.mat
    fe = FE(fp.mesh, mat.E, mat.nu, mat.rho, mat.thickness, [], 0, fp.faces, fp.face_traction)
    dt, g_, b_ = fp.dt, fp.gamma, fp.beta
    nw = Newmark(fe, dt, b_, fp.fixed)
    u = np.zeros(fe.dim * fe.n)
    v = np.zeros_like(u)
    a = nw.initial_acceleration(u)
    out = np.zeros((n_steps, len(record)))
    for k in range(n_steps):
        ut = u + dt * v + (0.5 - b_) * dt * dt * a
        vt = v + (1 - g_) * dt * a
        a = nw.solve(fe.P - fe.K @ ut)
        u, v = ut + b_ * dt * dt * a, vt + g_ * dt * a
        out[k] = u[record]
    return out


class MTSOracle:
    """Algorithm 1 (MTS coupling of PD and CCM) in FP64 on the CPU."""

    def __init__(self, cp, breaking=True, rebuild="auto", v0=None):
        self.cp = cp
        pb = cp.pd
        mat = pb.mat
        self.m = cp.m
        self.dt_pd = cp.dt_pd
        self.dt_fe = cp.m * cp.dt_pd
        self.gamma, self.beta = cp.gamma_fe, cp.beta_fe
        self.rebuild_mode = rebuild
        # --- PD subdomain (Eq. 1-5, weighted by 1 - alpha) ---
        self.pd = PD(pb.lat.X, pb.vol, pb.delta, pb.c, pb.s0, mat.rho, cp.dt_pd, breaking=breaking,
                     micro=pb.extra.get("micro", MICRO_POWER), l=pb.extra.get("l", 0.0))
        self.rp, self.col = family(pb.lat.X, pb.delta)
        if pb.cuts:
            self.mu, _ = precrack(pb.lat.P, self.rp, self.col, [c.in_half_units(pb.lat) for c in pb.cuts])
        else:
            self.mu = np.ones(len(self.col), np.uint8)
        self.alpha = band_weight(pb.lat.X, cp.bands, cp.weight_kind, 0.0)
        npd = pb.n
        self.npd = npd
        self.dim = dim = pb.lat.dim
        self.u = np.zeros((dim, npd)); self.v = np.zeros_like(self.u); self.a = np.zeros_like(self.u)
        self.pd_inited = False
        # --- FE subdomain ---
        self.fe = FE(cp.fe, mat.E, mat.nu, mat.rho, mat.thickness, cp.bands, cp.weight_kind, cp.faces,
                     cp.face_traction)
        nfe = self.fe.n
        self.nfe = nfe
        self.uf = np.zeros(dim * nfe); self.vf = np.zeros_like(self.uf); self.af = np.zeros_like(self.uf)
        if v0 is not None:  # uniform initial velocity (patch tests)
            self.v[:] = np.asarray(v0, dtype=np.float64).reshape(dim, 1)
            self.vf[:] = np.repeat(np.asarray(v0, dtype=np.float64), nfe)
        self.solver = Newmark(self.fe, self.dt_fe, self.beta, getattr(cp, "fixed", None))
        if v0 is not None:
            self.vf[self.solver.fixed] = 0.0
        # initial acceleration from the equation of motion at t_0 with lambda_0 = 0
        self.af = self.solver.initial_acceleration(self.uf)
        # --- multiplier space and constraint matrices (Eq. 33, Eq. 41) ---
        self._build_G()
        self.lam = np.zeros(self.nlam)  # lambda_0 = 0 at t = 0
        self.mu_link = self.mu.copy()
        self.H = None
        self.n_rebuilds = 0
        self.residuals = []
        xb = pb.lat.X[1]
        reach = (cp.m + 1) * pb.delta
        near = np.zeros(npd, bool)
        for b in cp.bands:
            near |= (pb.lat.X[b.axis] >= b.lo - reach) & (pb.lat.X[b.axis] <= b.hi + reach)
        self.near = near
        del xb

    # ----------------------------------------------------------------------
    def _build_G(self):
        cp, fe = self.cp, self.fe
        X = fe.X
        dim = self.dim
        cen = X[:, fe.conn].mean(axis=2)  # (dim, ne)
        in_band = np.zeros(fe.conn.shape[0], bool)
        for b in cp.bands:
            c = cen[b.axis]
            in_band |= (c > b.lo) & (c < b.hi)
        self.ov_elems = np.nonzero(in_band)[0]
        lam_nodes = np.unique(fe.conn[self.ov_elems].reshape(-1))
        for d in range(dim):  # a fixed dof carries no multiplier force
            assert not np.isin(d * self.nfe + lam_nodes, self.solver.fixed).any(), "fixed dof in the overlap"
        self.lam_nodes = lam_nodes
        nl = len(lam_nodes)
        self.nlam_nodes = nl
        self.nlam = dim * nl
        pos = {int(k): i for i, k in enumerate(lam_nodes)}
        nfe, npd = self.nfe, self.npd
        thick = cp.pd.mat.thickness
        # G_FE[k, I] = int_O N_k N_I dV, per component (2 x 2 or 2 x 2 x 2 Gauss)
        rows, cols, vals = [], [], []
        for e in self.ov_elems:
            nodes = fe.conn[e]
            xe = X[:, nodes]
            if dim == 2:
                pts = []
                for gx in GAUSS:
                    for gy in GAUSS:
                        N, dxi, deta = q4_shape(gx, gy)
                        J = np.array([[dxi @ xe[0], dxi @ xe[1]], [deta @ xe[0], deta @ xe[1]]])
                        pts.append((N, np.linalg.det(J) * thick))
            else:
                pts = [(N, detJ) for N, _, detJ, _ in hex8_gauss(xe)]
            for N, w in pts:
                for a in range(len(nodes)):
                    for b in range(len(nodes)):
                        k = pos[int(nodes[a])]
                        for c in range(dim):
                            rows.append(c * nl + k); cols.append(c * nfe + int(nodes[b]))
                            vals.append(N[a] * N[b] * w)
        self.Gfe = sp.csr_matrix((vals, (rows, cols)), shape=(dim * nl, dim * nfe))
        # G_PD[k, p] = N_k(x_p) V_p for PD nodes inside overlap elements
        Xp = cp.pd.lat.X
        rows, cols, vals = [], [], []
        for e in self.ov_elems:
            nodes = fe.conn[e]
            xe = X[:, nodes]
            lo, hi = xe.min(axis=1), xe.max(axis=1)
            inside = np.ones(npd, bool)
            for d in range(dim):
                inside &= (Xp[d] > lo[d]) & (Xp[d] < hi[d])
            for p in np.nonzero(inside)[0]:
                xi = 2 * (Xp[:, p] - lo) / (hi - lo) - 1
                if dim == 2:
                    N, _, _ = q4_shape(xi[0], xi[1])
                else:
                    N, _ = hex8_shape(xi[0], xi[1], xi[2])
                for a in range(len(nodes)):
                    k = pos[int(nodes[a])]
                    for c in range(dim):
                        rows.append(c * nl + k); cols.append(c * npd + int(p)); vals.append(N[a] * cp.pd.vol)
        self.Gpd = sp.csr_matrix((vals, (rows, cols)), shape=(dim * nl, dim * npd))

    def interface_force_density(self, lam):
        """g = G_PD^T lambda / V per PD node (dim, npd)."""
        return (self.Gpd.T @ lam).reshape(self.dim, self.npd) / self.cp.pd.vol

    # ----------------------------------------------------------------------
    def pd_link(self, lam, mu):
        """Link problem (Eq. 48b): zero start, load (j/m) G_PD^T lambda, no breaking."""
        m = self.m
        u = np.zeros((self.dim, self.npd)); v = np.zeros_like(u); a = np.zeros_like(u)
        theta = np.arange(1, m + 1, dtype=np.float64) / m
        g = self.interface_force_density(lam)
        mu_c = mu.copy()
        pd_run(self.pd, self.rp, self.col, mu_c, u, v, a, m, alpha=self.alpha, b=None, g=g, theta=theta,
               breaking=False)
        return u, v, a

    def fe_link(self, lam):
        """FE link response (Eq. 47b with Newmark): a = -K_eff^-1 G_FE^T lambda."""
        aw = -self.solver.solve(self.Gfe.T @ lam)
        return self.beta * self.dt_fe ** 2 * aw, self.gamma * self.dt_fe * aw, aw

    def build_H(self):
        """Unit-load responses (Eq. unit) and the interface operator of Eq. 49:
        H = G_FE Ydot_FE - G_PD Ydot_PD, one column per multiplier component."""
        nl = self.nlam
        H = np.zeros((nl, nl))
        for q in range(nl):
            e = np.zeros(nl); e[q] = 1.0
            _, vf, _ = self.fe_link(e)
            _, vp, _ = self.pd_link(e, self.mu_link)
            H[:, q] = self.Gfe @ vf - self.Gpd @ vp.reshape(-1)
        self.H = H
        self.n_rebuilds += 1

    # ----------------------------------------------------------------------
    def coarse_step(self):
        """One coarse step t_0 -> t_m of Algorithm 1."""
        m, dtf, g_, b_ = self.m, self.dt_fe, self.gamma, self.beta
        if self.H is None:
            self.build_H()
        # free FE problem (Eq. 47a with Newmark, Eq. 39)
        ut = self.uf + dtf * self.vf + (0.5 - b_) * dtf * dtf * self.af
        vt = self.vf + (1 - g_) * dtf * self.af
        af = self.solver.solve(self.fe.P - self.fe.K @ ut)
        Vu, Vv, Va = ut + b_ * dtf * dtf * af, vt + g_ * dtf * af, af
        # free PD problem (Eq. 48a): m substeps, multiplier (1 - j/m) lambda_0
        mu_start = self.mu.copy()
        theta = 1.0 - np.arange(1, m + 1, dtype=np.float64) / m
        g = self.interface_force_density(self.lam)
        pd_run(self.pd, self.rp, self.col, self.mu, self.u, self.v, self.a, m, alpha=self.alpha, b=None, g=g,
               theta=theta, theta_init=1.0, init=not self.pd_inited)
        self.pd_inited = True
        # interface problem (Eq. 49): H lambda_m = -(G_FE V_FE - G_PD V_PD)
        r = -(self.Gfe @ Vv - self.Gpd @ self.v.reshape(-1))
        lam = np.linalg.solve(self.H, r)
        # correction U = V + Y lambda_m (FE exactly; PD by the link run)
        wu, wv, wa = self.fe_link(lam)
        self.uf, self.vf, self.af = Vu + wu, Vv + wv, Va + wa
        pu, pv, pa = self.pd_link(lam, self.mu_link)
        self.u += pu; self.v += pv; self.a += pa
        self.lam = lam
        res = self.Gfe @ self.vf - self.Gpd @ self.v.reshape(-1)
        self.residuals.append(np.linalg.norm(res) / max(np.linalg.norm(self.Gfe @ self.vf), 1e-300))
        # bonds broken this step near an overlap band -> rebuild the unit responses
        broke = (mu_start == 1) & (self.mu == 0)
        i_of = np.repeat(np.arange(self.npd), np.diff(self.rp))
        near_break = bool(np.any(broke & (self.near[i_of] | self.near[self.col])))
        self.mu_link = self.mu.copy()
        if self.rebuild_mode == "always" or (self.rebuild_mode == "auto" and near_break):
            self.H = None  # rebuilt at the start of the next coarse step
        return lam

    def advance(self, n):
        for _ in range(n):
            self.coarse_step()
        return self

    def damage(self):
        return damage(self.pd, self.rp, self.col, self.mu)


def monolithic_step(orc: MTSOracle, state):
    """The single-step coupled scheme of Eq. 33 for m = 1, as one KKT solve
    (no breaking): unknowns (a_FE, a_PD, lambda) at t_{n+1}."""
    uf, vf, af, u, v, a = state
    dt = orc.dt_fe
    g_, b_ = orc.gamma, orc.beta
    nfe2, npd2, nl = 2 * orc.nfe, 2 * orc.npd, orc.nlam
    utf = uf + dt * vf + (0.5 - b_) * dt * dt * af
    vtf = vf + (1 - g_) * dt * af
    utp = u + dt * v + 0.5 * dt * dt * a  # explicit PD predictor (beta = 0)
    vtp = v + 0.5 * dt * a
    f, _ = pd_forces(orc.pd, orc.rp, orc.col, orc.mu.copy(), utp, alpha=orc.alpha, breaking=False)
    V = orc.cp.pd.vol
    Mpd = np.concatenate([(1 - orc.alpha) * orc.cp.pd.mat.rho * V] * 2)
    Keff = (sp.diags(orc.fe.M) + b_ * dt * dt * orc.fe.K).toarray()
    A = np.zeros((nfe2 + npd2 + nl, nfe2 + npd2 + nl))
    A[:nfe2, :nfe2] = Keff
    A[:nfe2, nfe2 + npd2:] = orc.Gfe.T.toarray()
    A[nfe2:nfe2 + npd2, nfe2:nfe2 + npd2] = np.diag(Mpd)
    A[nfe2:nfe2 + npd2, nfe2 + npd2:] = -orc.Gpd.T.toarray()
    A[nfe2 + npd2:, :nfe2] = g_ * dt * orc.Gfe.toarray()
    A[nfe2 + npd2:, nfe2:nfe2 + npd2] = -g_ * dt * orc.Gpd.toarray()
    rhs = np.concatenate([orc.fe.P - orc.fe.K @ utf, (f * V).reshape(-1),
                          -(orc.Gfe @ vtf - orc.Gpd @ vtp.reshape(-1))])
    sol = np.linalg.solve(A, rhs)
    afn, apn, lam = sol[:nfe2], sol[nfe2:nfe2 + npd2].reshape(2, -1), sol[nfe2 + npd2:]
    return (utf + b_ * dt * dt * afn, vtf + g_ * dt * afn, afn, utp, vtp + 0.5 * dt * apn, apn), lam
