"""Seeded synthetic inputs shared by the tests, the oracle runs and the benchmark.

This module only builds problem statements: lattices of PD nodes, finite-element
meshes, pre-crack cuts, traction loads, material constants and random initial
fields. It holds none of the method's arithmetic (no bond force, no time step,
no coupling), so the oracle and the CUDA library can both take their inputs
from it without sharing any computation.

Workloads follow the benchmark plates of arXiv 2403.03605 (Sec. 3.3, Sec. 4.1):
regular lattices with nodes at cell centres, horizon 3.015 dx, glass-like
material (E = 72 GPa, nu = 1/3, rho = 2440 kg/m^3, G0 = 3.8 J/m^2), tractions
applied as a body force over a layer of width delta (Sec. 3.3) and straight
pre-cracks whose crossing bonds start broken. The paper uses no dataset; these
synthetic plates stand in for its examples.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

HORIZON_FACTOR = 3.015


@dataclass
class Material:
    E: float = 72e9
    nu: float = 1.0 / 3.0
    rho: float = 2440.0
    G0: float = 3.8
    thickness: float = 1e-3  # plane-stress thickness h of the 2D plates [m]


def pmb_constants(dim: int, mat: Material, delta: float):
    """Micromodulus constant c and critical stretch s0 of the benchmark plates.

    2D plane stress: c = 9E / (pi h delta^3), s0 = sqrt(4 pi G0 / (9 E delta)).
    3D: c = 12E / (pi delta^4), s0 = sqrt(5 G0 / (9 E delta)).
    These are the problem statement's constants, inputs to both sides.
    """
    if dim == 2:
        c = 9.0 * mat.E / (math.pi * mat.thickness * delta ** 3)
        s0 = math.sqrt(4.0 * math.pi * mat.G0 / (9.0 * mat.E * delta))
    else:
        c = 12.0 * mat.E / (math.pi * delta ** 4)
        s0 = math.sqrt(5.0 * mat.G0 / (9.0 * mat.E * delta))
    return c, s0


@dataclass
class Lattice:
    """Regular lattice of PD nodes at cell centres, x fastest.

    shape: nodes per axis; dx: spacing; origin: corner of the lattice box.
    Node (ix, iy[, iz]) has index ix + nx * (iy + ny * iz) and position
    origin + (idx + 1/2) dx. `P` holds the same position in integer half-dx
    units relative to origin (2 idx + 1), used for exact pre-crack tests.
    """
    shape: tuple
    dx: float
    origin: tuple

    @property
    def dim(self):
        return len(self.shape)

    @property
    def n(self):
        return int(np.prod(self.shape))

    def index_grid(self):
        axes = [np.arange(s, dtype=np.int64) for s in self.shape]
        grids = np.meshgrid(*axes, indexing="ij")  # grids[d][ix, iy, ...]
        # flatten with x fastest: transpose so that axis 0 (x) varies fastest
        return np.stack([g.transpose(*reversed(range(self.dim))).reshape(-1) for g in grids])

    @property
    def idx(self):
        return self.index_grid()

    @property
    def X(self):
        idx = self.index_grid().astype(np.float64)
        org = np.asarray(self.origin, dtype=np.float64).reshape(-1, 1)
        return org + (idx + 0.5) * self.dx

    @property
    def P(self):
        return 2 * self.index_grid() + 1

    def half_units(self, value: float, axis: int) -> int:
        """A coordinate on the half-dx grid, as an exact integer (asserts it is on it)."""
        q = (value - self.origin[axis]) / (0.5 * self.dx)
        k = int(round(q))
        assert abs(q - k) < 1e-6, (value, axis, q)
        return k


@dataclass
class Cut:
    """Axis-aligned straight pre-crack: plane x[normal] = level, lo <= x[along] < hi [m]."""
    normal: int
    level: float
    along: int
    lo: float
    hi: float

    def as_array(self):
        return np.array([self.normal, self.level, self.along, self.lo, self.hi], dtype=np.float64)

    def in_half_units(self, lat: Lattice):
        return (self.normal, lat.half_units(self.level, self.normal), self.along,
                lat.half_units(self.lo, self.along), lat.half_units(self.hi, self.along))


def edge_traction_body_force(lat: Lattice, traction: float, delta: float, axis: int = 1):
    """Traction on the two faces normal to `axis` as a body force (Sec. 3.3, Sec. 4.1).

    Nodes whose cell-centre distance to a face is at most delta form a layer of
    `k` rows; each gets b = +-T / (k dx) along `axis` (outward), so the layer
    carries exactly T per unit face area.
    """
    idx = lat.idx
    ncount = lat.shape[axis]
    k = 0
    while k < ncount and (k + 0.5) * lat.dx <= delta:
        k += 1
    b = np.zeros((lat.dim, lat.n))
    mag = traction / (k * lat.dx)
    b[axis, idx[axis] < k] = -mag
    b[axis, idx[axis] >= ncount - k] = +mag
    return b


@dataclass
class PDProblem:
    """A pure PD problem statement (inputs only)."""
    name: str
    lat: Lattice
    mat: Material
    delta: float
    c: float
    s0: float
    dt: float
    nsteps: int
    cuts: list
    b: np.ndarray
    vol: float
    extra: dict = field(default_factory=dict)

    @property
    def dim(self):
        return self.lat.dim

    @property
    def n(self):
        return self.lat.n


def plate2d(nx: int, ny: int, dx: float, *, cuts_mm=(), traction=12e6, dt=25e-9, nsteps=500,
            mat: Material | None = None, name="plate2d") -> PDProblem:
    mat = mat or Material()
    lat = Lattice((nx, ny), dx, (0.0, 0.0))
    delta = HORIZON_FACTOR * dx
    c, s0 = pmb_constants(2, mat, delta)
    cuts = [Cut(*cm) for cm in cuts_mm]
    b = edge_traction_body_force(lat, traction, delta, axis=1) if traction else np.zeros((2, lat.n))
    return PDProblem(name, lat, mat, delta, c, s0, dt, nsteps, cuts, b, mat.thickness * dx * dx)


def plate3d(nx: int, ny: int, nz: int, dx: float, *, cuts_mm=(), traction=12e6, dt=20e-9, nsteps=300,
            mat: Material | None = None, name="plate3d") -> PDProblem:
    mat = mat or Material(nu=0.25)
    lat = Lattice((nx, ny, nz), dx, (0.0, 0.0, 0.0))
    delta = HORIZON_FACTOR * dx
    c, s0 = pmb_constants(3, mat, delta)
    cuts = [Cut(*cm) for cm in cuts_mm]
    b = edge_traction_body_force(lat, traction, delta, axis=1) if traction else np.zeros((3, lat.n))
    return PDProblem(name, lat, mat, delta, c, s0, dt, nsteps, cuts, b, dx ** 3)


def plate_100x100() -> PDProblem:
    """Pure FP64 2D plate: 0.05 x 0.05 m, dx 0.5 mm (100 x 100 nodes), centred 10 mm
    pre-crack at mid-height, 12 MPa on top/bottom edges, dt 25 ns, 500 steps."""
    return plate2d(100, 100, 0.5e-3, cuts_mm=[(1, 0.025, 0, 0.020, 0.030)], traction=12e6,
                   dt=25e-9, nsteps=500, name="plate2d_100x100_dx0.5mm_centre_crack")


def small_plate(nx=40, ny=24, dx=0.5e-3, nsteps=200, crack=True, dt=25e-9) -> PDProblem:
    """A small plate the oracle finishes in well under a second (tests)."""
    # edge crack between the two middle node rows, tip on a lattice column boundary
    cuts = [(1, (ny // 2) * dx, 0, 0.0, round(0.4 * nx) * dx)] if crack else []
    return plate2d(nx, ny, dx, cuts_mm=cuts, traction=12e6, dt=dt, nsteps=nsteps,
                   name=f"plate2d_{nx}x{ny}")


def strip_lattice_pd(nx: int, ny: int, dx: float, crack_len: float, traction=12e6, dt=5e-9, nsteps=100,
                     name="strip") -> PDProblem:
    """The PD strip of the coupled plates used as a standalone PD lattice
    (edge pre-crack along the mid line, traction layer on the strip's faces)."""
    return plate2d(nx, ny, dx, cuts_mm=[(1, ny * dx / 2, 0, 0.0, crack_len)], traction=traction,
                   dt=dt, nsteps=nsteps, name=name)


def random_field(shape, scale, seed):
    """Seeded smooth-ish random field (used for initial displacements in tests)."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal(shape) * scale


# --------------------------------------------------------------------------
# Coupled PD / finite-element plates (Sec. 2.2-2.5, Sec. 3.3, Sec. 4.1)
# --------------------------------------------------------------------------
@dataclass
class Band:
    """Overlap band lo <= x[axis] <= hi; the finite-element-only region lies on
    `fe_side` (-1: below lo, +1: above hi)."""
    axis: int
    lo: float
    hi: float
    fe_side: int

    def as_array(self):
        return np.array([self.axis, self.lo, self.hi, self.fe_side, 0.0], dtype=np.float64)


@dataclass
class FEMesh:
    """Structured mesh: nodes (dim, n) and connectivity (ne, 4) Q4 counter-clockwise
    or (ne, 8) Hex8."""
    X: np.ndarray
    conn: np.ndarray
    h: float  # element size

    @property
    def n(self):
        return self.X.shape[1]

    @property
    def ne(self):
        return self.conn.shape[0]


def q4_block(x0, y0, nex, ney, h, node_offset=0):
    xs = x0 + h * np.arange(nex + 1)
    ys = y0 + h * np.arange(ney + 1)
    X = np.stack(np.meshgrid(xs, ys, indexing="xy")).reshape(2, -1)  # x fastest
    conn = []
    for j in range(ney):
        for i in range(nex):
            a = j * (nex + 1) + i
            conn.append([a, a + 1, a + nex + 2, a + nex + 1])
    return X, np.asarray(conn, dtype=np.int32) + node_offset


@dataclass
class CoupledProblem:
    """A coupled PD / FE problem statement (inputs only)."""
    name: str
    pd: PDProblem          # PD strip (its own body force is zero)
    fe: FEMesh
    faces: np.ndarray      # (nf, 2) FE edge node pairs carrying traction
    face_traction: np.ndarray  # (nf, 2) traction vector per face [Pa]
    bands: list
    weight_kind: int       # 0 constant, 1 linear, 2 cubic (Sec. 3.2)
    m: int                 # time-step ratio dt_FE / dt_PD
    n_coarse: int
    gamma_fe: float = 0.5
    beta_fe: float = 0.25
    fixed: np.ndarray | None = None  # FE dof ids d * n + node held at zero (Dirichlet)

    @property
    def dt_pd(self):
        return self.pd.dt


def coupled_plate(Lx, Ly, strip, dx, h_fe, overlap, *, crack=None, traction=12e6, dt=20e-9, m=10, n_coarse=200,
                  weight_kind=1, mat: Material | None = None, name="coupled_plate") -> CoupledProblem:
    """Plate [0, Lx] x [0, Ly]; PD strip strip = (y0, y1) at spacing dx; Q4
    elements of size h_fe on [0, y0 + overlap] and [y1 - overlap, Ly]; the
    overlap bands are [y0, y0 + overlap] and [y1 - overlap, y1]. Traction on
    the bottom and top edges (mode I). crack = (y_level, x_lo, x_hi)."""
    mat = mat or Material()
    y0, y1 = strip
    nx = int(round(Lx / dx))
    ny = int(round((y1 - y0) / dx))
    lat = Lattice((nx, ny), dx, (0.0, y0))
    delta = HORIZON_FACTOR * dx
    c, s0 = pmb_constants(2, mat, delta)
    cuts = [Cut(1, crack[0], 0, crack[1], crack[2])] if crack else []
    pd = PDProblem(name + "_pd", lat, mat, delta, c, s0, dt, m * n_coarse, cuts, np.zeros((2, lat.n)),
                   mat.thickness * dx * dx)
    nex = int(round(Lx / h_fe))
    neb = int(round((y0 + overlap) / h_fe))
    net = int(round((Ly - (y1 - overlap)) / h_fe))
    Xb, cb = q4_block(0.0, 0.0, nex, neb, h_fe)
    Xt, ct = q4_block(0.0, y1 - overlap, nex, net, h_fe, node_offset=Xb.shape[1])
    fe = FEMesh(np.concatenate([Xb, Xt], axis=1), np.concatenate([cb, ct]), h_fe)
    nb = Xb.shape[1]
    bot = [(i, i + 1) for i in range(nex)]
    top_row = nb + net * (nex + 1)
    top = [(top_row + i + 1, top_row + i) for i in range(nex)]
    faces = np.asarray(bot + top, dtype=np.int32)
    tr = np.zeros((len(faces), 2))
    tr[:nex, 1] = -traction
    tr[nex:, 1] = +traction
    bands = [Band(1, y0, y0 + overlap, -1), Band(1, y1 - overlap, y1, +1)]
    return CoupledProblem(name, pd, fe, faces, tr, bands, weight_kind, m, n_coarse)


def coupled_plate_400x64() -> CoupledProblem:
    """Coupled 2D plate 0.1 x 0.04 m, 50 mm edge pre-crack at mid-height; PD strip
    16 mm (400 x 64 nodes at 0.25 mm), Q4 elements of 1 mm elsewhere, 2 mm overlap
    bands with linear weights; 12 MPa; dt_PD 20 ns, m = 10, 200 coarse steps."""
    return coupled_plate(0.1, 0.04, (0.012, 0.028), 0.25e-3, 1e-3, 2e-3, crack=(0.020, 0.0, 0.050),
                         dt=20e-9, m=10, n_coarse=200, name="coupled_plate_100x40mm_pd400x64")


def coupled_plate_2000x400() -> CoupledProblem:
    """Fine coupled plate: PD strip 20 mm at 0.05 mm (2000 x 400 = 800k nodes), Q4
    0.5 mm, 2 mm overlap, 50 mm edge crack at mid-height; dt_PD 5 ns, m = 20, 500 coarse."""
    return coupled_plate(0.1, 0.04, (0.010, 0.030), 0.05e-3, 0.5e-3, 2e-3, crack=(0.020, 0.0, 0.050),
                         dt=5e-9, m=20, n_coarse=500, name="coupled_plate_100x40mm_pd2000x400")


def small_coupled(m=4, n_coarse=20, weight_kind=1, crack=True, traction=12e6, dx=0.25e-3) -> CoupledProblem:
    """A small coupled plate the oracle finishes in seconds (tests): 20 x 10 mm,
    PD strip y in [3, 7] mm, Q4 1 mm, 1 mm overlap bands."""
    return coupled_plate(0.02, 0.01, (0.003, 0.007), dx, 1e-3, 1e-3,
                         crack=(0.005, 0.0, 0.008) if crack else None, traction=traction, dt=20e-9, m=m,
                         n_coarse=n_coarse, weight_kind=weight_kind, name="coupled_small")


# Stable PD step of the coupled plates scales with the lattice spacing: the
# 0.25 mm plate's bound is 51.7 ns (a statement of the benchmark, used only to
# choose a step below it).
DT_CRIT_PER_M = 51.7e-9 / 0.25e-3


def batch_member(N: int, crack_len: float, traction: float, m: int, *, n_coarse=200, name="batch") -> CoupledProblem:
    """One specimen of the batched benchmark: the 0.1 x 0.04 m plate with a 16 mm
    PD strip at dx = sqrt(0.1 * 0.016 / N) (about N nodes), Q4 1 mm, 2 mm overlap,
    an edge crack of length crack_len at mid-height, dt_PD = 0.4 of the bound."""
    dx = math.sqrt(0.1 * 0.016 / N)
    dt = 0.4 * DT_CRIT_PER_M * dx
    return coupled_plate(0.1, 0.04, (0.012, 0.028), dx, 1e-3, 2e-3, crack=(0.020, 0.0, crack_len),
                         traction=traction, dt=dt, m=m, n_coarse=n_coarse, name=name)


def batch_plates_draws(seed: int = 3605, n: int = 64):
    """(N_PD, crack length, traction, m) of the batched benchmark's specimens,
    drawn per specimen in this order: N ~ U[20k, 400k] (integer), crack ~
    U[20, 60] mm, traction ~ U[6, 15] MPa, m ~ choice{5, 10, 20}."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        N = int(rng.integers(20_000, 400_001))
        crack = float(rng.uniform(0.020, 0.060))
        T = float(rng.uniform(6e6, 15e6))
        m = int(rng.choice([5, 10, 20]))
        out.append((N, crack, T, m))
    return out


def batch_plates(seed: int = 3605, n: int = 64, n_coarse: int = 200) -> list[CoupledProblem]:
    """Batched: n independent coupled plates of uneven size, crack, load and m."""
    return [batch_member(N, c, T, m, n_coarse=n_coarse, name=f"batch_plate_{k}")
            for k, (N, c, T, m) in enumerate(batch_plates_draws(seed, n))]


def hex8_block(x0, y0, z0, nex, ney, nez, h, node_offset=0):
    """Structured Hex8 block (nodes x fastest, then y, then z); each element's
    corners: the bottom face (z low) counter-clockwise seen from +z, then the
    top face in the same order."""
    xs = x0 + h * np.arange(nex + 1)
    ys = y0 + h * np.arange(ney + 1)
    zs = z0 + h * np.arange(nez + 1)
    Z, Y, Xg = np.meshgrid(zs, ys, xs, indexing="ij")
    X = np.stack([Xg.reshape(-1), Y.reshape(-1), Z.reshape(-1)])

    def nid(i, j, k):
        return (k * (ney + 1) + j) * (nex + 1) + i

    conn = []
    for k in range(nez):
        for j in range(ney):
            for i in range(nex):
                conn.append([nid(i, j, k), nid(i + 1, j, k), nid(i + 1, j + 1, k), nid(i, j + 1, k),
                             nid(i, j, k + 1), nid(i + 1, j, k + 1), nid(i + 1, j + 1, k + 1), nid(i, j + 1, k + 1)])
    return X, np.asarray(conn, dtype=np.int32) + node_offset


def coupled_plate3d(Lx, Ly, Lz, strip, dx, h_fe, overlap, *, crack=None, traction=12e6, dt=20e-9, m=10,
                    n_coarse=300, weight_kind=1, mat: Material | None = None, name="coupled_plate3d") -> CoupledProblem:
    """3D counterpart of coupled_plate: box [0, Lx] x [0, Ly] x [0, Lz]; PD strip
    y in strip at spacing dx (through the thickness); Hex8 elements of size h_fe
    on [0, y0 + overlap] and [y1 - overlap, Ly]; traction on the faces y = 0 and
    y = Ly; crack = (y_level, x_lo, x_hi) through the thickness."""
    mat = mat or Material(nu=0.25)
    y0, y1 = strip
    nx, ny, nz = int(round(Lx / dx)), int(round((y1 - y0) / dx)), int(round(Lz / dx))
    lat = Lattice((nx, ny, nz), dx, (0.0, y0, 0.0))
    delta = HORIZON_FACTOR * dx
    c, s0 = pmb_constants(3, mat, delta)
    cuts = [Cut(1, crack[0], 0, crack[1], crack[2])] if crack else []
    pd = PDProblem(name + "_pd", lat, mat, delta, c, s0, dt, m * n_coarse, cuts, np.zeros((3, lat.n)), dx ** 3)
    nex, nez = int(round(Lx / h_fe)), int(round(Lz / h_fe))
    neb = int(round((y0 + overlap) / h_fe))
    net = int(round((Ly - (y1 - overlap)) / h_fe))
    Xb, cb = hex8_block(0.0, 0.0, 0.0, nex, neb, nez, h_fe)
    Xt, ct = hex8_block(0.0, y1 - overlap, 0.0, nex, net, nez, h_fe, node_offset=Xb.shape[1])
    fe = FEMesh(np.concatenate([Xb, Xt], axis=1), np.concatenate([cb, ct]), h_fe)
    nb = Xb.shape[1]

    def bot(i, k):  # node on the face y = 0 of the bottom block
        return k * (neb + 1) * (nex + 1) + i

    def top(i, k):  # node on the face y = Ly of the top block
        return nb + (k * (net + 1) + net) * (nex + 1) + i

    faces, tr = [], []
    for k in range(nez):
        for i in range(nex):
            faces.append([bot(i, k), bot(i + 1, k), bot(i + 1, k + 1), bot(i, k + 1)])
            tr.append([0.0, -traction, 0.0])
            faces.append([top(i, k), top(i + 1, k), top(i + 1, k + 1), top(i, k + 1)])
            tr.append([0.0, +traction, 0.0])
    bands = [Band(1, y0, y0 + overlap, -1), Band(1, y1 - overlap, y1, +1)]
    return CoupledProblem(name, pd, fe, np.asarray(faces, dtype=np.int32), np.asarray(tr), bands, weight_kind, m,
                          n_coarse)


def coupled_plate3d_400x64x8() -> CoupledProblem:
    """3D coupled plate 0.1 x 0.04 x 0.002 m: PD strip 16 mm at 0.25 mm
    (400 x 64 x 8 nodes), Hex8 1 mm elsewhere, 2 mm overlap, 50 mm edge crack
    at mid-height, 12 MPa, dt_PD 20 ns, m = 10, 300 coarse steps, nu = 1/4."""
    return coupled_plate3d(0.1, 0.04, 0.002, (0.012, 0.028), 0.25e-3, 1e-3, 2e-3, crack=(0.020, 0.0, 0.050),
                           dt=20e-9, m=10, n_coarse=300, name="coupled_plate3d_100x40x2mm_pd400x64x8")


def small_coupled3d(m=3, n_coarse=6, weight_kind=1, crack=True, traction=12e6, dx=0.5e-3) -> CoupledProblem:
    """A small 3D coupled plate the oracle finishes in seconds (tests): 8 x 8 x 2 mm,
    PD strip y in [2, 6] mm, Hex8 1 mm, 1 mm overlap bands."""
    return coupled_plate3d(0.008, 0.008, 0.002, (0.002, 0.006), dx, 1e-3, 1e-3,
                           crack=(0.004, 0.0, 0.003) if crack else None, traction=traction, dt=20e-9, m=m,
                           n_coarse=n_coarse, weight_kind=weight_kind, name="coupled_small3d")


# ---------------------------------------------------------------------------
# 3D beam of the coupling-accuracy study (Sec. 3.2, Table 1, Figs. 4-7)
# ---------------------------------------------------------------------------
BEAM_MATERIAL = Material(E=6.5e9, nu=0.25, rho=2235.0, G0=0.0, thickness=1.0)
BEAM_HORIZON_FACTOR = 3.03   # delta = 3.03 dx
BEAM_DT = 2.5e-5             # coarse (FE) step of Table 1
BEAM_TRACTION = 4e6          # axial traction on the free end [Pa]


def exp_micromodulus_c0(E: float, delta: float, ell: float) -> float:
    """c0 of the 3D exponential micromodulus c(r) = c0 exp(-r / ell) (Sec. 3.2):
    c0 = 3E / (pi int_0^delta r^6 exp(-r/ell) dr), the integral in closed form
    ell^7 6! (1 - exp(-x) sum_{k<=6} x^k / k!) with x = delta / ell."""
    x = delta / ell
    tail = math.exp(-x) * sum(x ** k / math.factorial(k) for k in range(7))
    return 3.0 * E / (math.pi * ell ** 7 * math.factorial(6) * (1.0 - tail))


@dataclass
class FEProblem:
    """An undecomposed finite-element problem (the Table 1 reference)."""
    name: str
    mesh: FEMesh
    faces: np.ndarray
    face_traction: np.ndarray
    fixed: np.ndarray
    mat: Material
    dt: float
    n_steps: int
    gamma: float = 0.5
    beta: float = 0.25
    record: dict = field(default_factory=dict)  # tracked points -> x dof id


def _beam_block(x0, nex, ne_yz, h, node_offset=0):
    """Hex8 block [x0, x0 + nex h] x [0, ne_yz h]^2 with its end-face helpers."""
    X, conn = hex8_block(x0, 0.0, 0.0, nex, ne_yz, ne_yz, h, node_offset=node_offset)

    def nid(i, j, k):
        return node_offset + (k * (ne_yz + 1) + j) * (nex + 1) + i

    def face(i):  # quads of the face x = x0 + i h, corners in order around each quad
        return [[nid(i, j, k), nid(i, j + 1, k), nid(i, j + 1, k + 1), nid(i, j, k + 1)]
                for k in range(ne_yz) for j in range(ne_yz)]

    def face_nodes(i):
        return [nid(i, j, k) for k in range(ne_yz + 1) for j in range(ne_yz + 1)]

    return X, conn, nid, face, face_nodes


def beam3d_fe(dx=0.1, n_steps=480, beta=0.25, length=10.0, width=1.0, mat: Material | None = None) -> FEProblem:
    """Undecomposed Hex8 beam [0, length] x [0, width]^2 at element size dx,
    fixed at x = 0 (all components), axial traction 4 MPa on x = length,
    Newmark dt 2.5e-5 s; tracked points A (length, width/2, width/2) and, on
    beams longer than 6, B (6, width/2, width/2) (Sec. 3.2, cases 1 and 2 of
    Table 1)."""
    nex, ne_yz = int(round(length / dx)), int(round(width / dx))
    X, conn, nid, face, face_nodes = _beam_block(0.0, nex, ne_yz, dx)
    n = X.shape[1]
    faces = np.asarray(face(nex), dtype=np.int32)
    tr = np.tile([BEAM_TRACTION, 0.0, 0.0], (len(faces), 1))
    fixed = np.asarray([d * n + k for d in range(3) for k in face_nodes(0)], dtype=np.int64)
    c = ne_yz // 2
    ib = int(round(6.0 / dx))
    record = {"A": nid(nex, c, c)}
    if ib < nex:
        record["B"] = nid(ib, c, c)
    return FEProblem(f"beam3d_fe_dx{dx:g}", FEMesh(X, conn, dx), faces, tr, fixed, mat or BEAM_MATERIAL, BEAM_DT,
                     n_steps, 0.5, beta, record=record)


def beam3d(dx=0.1, overlap_cells=3, weight_kind=2, m=1, n_coarse=480, length=10.0, width=1.0,
           pd_range=(4.0, 6.0)) -> CoupledProblem:
    """The coupled beam of Table 1: PD on pd_range (exponential micromodulus,
    ell = delta / 16, delta = 3.03 dx, nodes at cell centres, no breaking),
    Hex8 elements of size dx on [0, x0 + l_O] and [x1 - l_O, length] with the
    overlap width l_O = overlap_cells dx, overlap bands [x0, x0 + l_O] and
    [x1 - l_O, x1], fixed end x = 0, traction on x = length, coarse step
    2.5e-5 s and dt_PD = 2.5e-5 / m. extra["record"] holds the x dof ids of
    the tracked points A and B on the right FE block."""
    mat = BEAM_MATERIAL
    x0, x1 = pd_range
    lo = overlap_cells * dx
    ne_yz = int(round(width / dx))
    lat = Lattice((int(round((x1 - x0) / dx)), ne_yz, ne_yz), dx, (x0, 0.0, 0.0))
    delta = BEAM_HORIZON_FACTOR * dx
    ell = delta / 16.0
    c0 = exp_micromodulus_c0(mat.E, delta, ell)
    pd = PDProblem(f"beam3d_pd_dx{dx:g}", lat, mat, delta, c0, 1.0, BEAM_DT / m, m * n_coarse, [],
                   np.zeros((3, lat.n)), dx ** 3, extra={"micro": 1, "l": ell})
    nl_ = int(round((x0 + lo) / dx))
    nr_ = int(round((length - (x1 - lo)) / dx))
    Xl, cl, nidl, _, face_l = _beam_block(0.0, nl_, ne_yz, dx)
    Xr, cr, nidr, face_r, _ = _beam_block(x1 - lo, nr_, ne_yz, dx, node_offset=Xl.shape[1])
    X = np.concatenate([Xl, Xr], axis=1)
    n = X.shape[1]
    faces = np.asarray(face_r(nr_), dtype=np.int32)
    tr = np.tile([BEAM_TRACTION, 0.0, 0.0], (len(faces), 1))
    fixed = np.asarray([d * n + k for d in range(3) for k in face_l(0)], dtype=np.int64)
    bands = [Band(0, x0, x0 + lo, -1), Band(0, x1 - lo, x1, +1)]
    c = ne_yz // 2
    pd.extra["record"] = {"A": nidr(nr_, c, c), "B": nidr(int(round((x1 - (x1 - lo)) / dx)), c, c)}
    return CoupledProblem(f"beam3d_dx{dx:g}_lo{overlap_cells}_w{weight_kind}_m{m}", pd,
                          FEMesh(X, np.concatenate([cl, cr]), dx), faces, tr, bands, weight_kind, m, n_coarse,
                          fixed=fixed)
