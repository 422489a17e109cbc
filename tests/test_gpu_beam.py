"""The 3D beam of the coupling-accuracy study (Sec. 3.2, Table 1): Dirichlet
dofs on the GPU, FP64 parity of the coupled beam with the oracle, and the
error of the coupled solution at the tracked point A against the
undecomposed finite-element beam."""
import os

import numpy as np
import pytest

from gpu_common import GpuMTS, rel_l2
from oracle.mts import MTSOracle, newmark_fe
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


def test_beam_fp64_matches_oracle(fresh):
    """Fixed end, exponential micromodulus, cubic weights, m = 2: FP64 parity
    with the oracle's Algorithm 1 after the reflected wave has crossed the
    PD subdomain; the fixed dofs stay exactly zero."""
    cp = W.beam3d(dx=0.25, overlap_cells=3, weight_kind=2, m=2, n_coarse=240)
    o = MTSOracle(cp).advance(cp.n_coarse)
    g = GpuMTS(fresh(), cp, P.PDMTS_FP64).run(cp.n_coarse)
    for a, b in [(g.u(), o.u), (g.v(), o.v), (g.uf(), o.uf), (g.vf(), o.vf)]:
        assert rel_l2(a, b) <= FP64_TOL
    assert rel_l2(g.lam(), o.lam) <= 1e-8
    assert np.all(g.uf()[cp.fixed] == 0.0) and np.all(g.vf()[cp.fixed] == 0.0)
    assert g.residual() <= 1e-12


def test_fixed_dofs_validation(fresh):
    cp = W.beam3d(dx=0.25, overlap_cells=1, m=1, n_coarse=1)
    ctx = fresh()
    fe = P.fem_create(ctx, cp.fe.X, cp.fe.conn, E=1e9, nu=0.25, rho=1e3, thickness=1.0)
    with pytest.raises(P.PdmtsError):
        P.fem_set_fixed(fe, [3 * cp.fe.n])  # id out of range
    # a node of an overlap element may not be fixed
    ov = int(np.argmin(np.abs(cp.fe.X[0] - 4.0) + np.abs(cp.fe.X[1]) + np.abs(cp.fe.X[2])))
    P.fem_set_fixed(fe, [ov])
    pb = cp.pd
    pd = P.pd_create(ctx, pb.lat.X, horizon=pb.delta, c=pb.c, s0=pb.s0, rho=pb.mat.rho, vol_uniform=pb.vol,
                     micro_kind=P.PDMTS_MICRO_EXP, l=pb.extra["l"])
    with pytest.raises(P.PdmtsError):
        P.arlequin_bind(ctx, pd, fe, cp.weight_kind, [b.as_array() for b in cp.bands])


# --- Table 1: u_x error at point A against the undecomposed FE beam --------
DX, N_STEPS = 0.1, 480
# (weight kind, overlap width in dx, m): cases 3-11 (m = 1) and the MTS
# cases with cubic weights over 3 dx (m = 2, 5, 10)
STUDY = [(k, c, 1) for k in (0, 1, 2) for c in (1, 3, 5)] + [(2, 3, 2), (2, 3, 5), (2, 3, 10)]
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "table1_beam_ux_error.txt")
KINDS = {"constant": 0, "linear": 1, "cubic": 2}


def _table1():
    """Table 1 rows as printed: {(weight kind, l_O / dx, m): [(case, beta_PD, error %)]}."""
    rows = {}
    with open(GOLDEN) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                case, kind, cells, _beta_fe, beta_pd, m, err = line.split()
                rows.setdefault((KINDS[kind], int(cells), int(m)), []).append(
                    (int(case), float(beta_pd), float(err)))
    return rows


def _paper(key):
    """The printed error of the case matching this library's explicit PD
    (beta_PD = 0) where Table 1 has one, else the beta_PD = 1/4 case."""
    rows = _table1()[key]
    explicit = [r for r in rows if r[1] == 0.0]
    return (explicit or rows)[0]


@pytest.fixture(scope="module")
def beam_reference():
    fp = W.beam3d_fe(dx=DX, n_steps=N_STEPS)
    return newmark_fe(fp, N_STEPS, np.array([fp.record["A"]]))[:, 0]


def _lattice_axial_modulus_ratio(pb):
    """Young's modulus along a lattice axis of the bond-based PD lattice
    (nodal quadrature, cell-centred cubic lattice), over E: the energy
    1/4 sum c (xi . eps xi)^2 V gives the cubic constants C11, C12 and
    E_x = (C11 - C12)(C11 + 2 C12) / (C11 + C12)."""
    dx = pb.lat.dx
    r = np.arange(-4, 5)
    xi = np.stack(np.meshgrid(r, r, r, indexing="ij")).reshape(3, -1) * dx
    d = np.sqrt((xi ** 2).sum(0))
    keep = (d > 0) & (d <= pb.delta)
    xi, d = xi[:, keep], d[keep]
    c = pb.c * np.exp(-d / pb.extra["l"])
    c11 = 0.5 * np.sum(c * xi[0] ** 4) * pb.vol
    c12 = 0.5 * np.sum(c * xi[0] ** 2 * xi[1] ** 2) * pb.vol
    return (c11 - c12) * (c11 + 2 * c12) / (c11 + c12) / pb.mat.E


def _coupled_history(ctx, cp):
    g = GpuMTS(ctx, cp, P.PDMTS_FP32_BULK)
    ia = cp.pd.extra["record"]["A"]
    out = np.zeros(cp.n_coarse)
    for k in range(cp.n_coarse):
        g.run(1)
        out[k] = g.uf()[ia]
    assert np.all(g.uf()[cp.fixed] == 0.0)
    return out


def test_beam_accuracy_study(fresh, beam_reference):
    """Global error of u_x at A over all coarse steps (the error measure of
    Sec. 3.2) for the weight types and overlap widths of Table 1 and for
    m = 2, 5, 10: every case within a few percent, cubic over 3 dx better
    than constant over dx, and the MTS cases as accurate as m = 1."""
    ref = beam_reference
    errs = {}
    for kind, cells, m in STUDY:
        cp = W.beam3d(dx=DX, overlap_cells=cells, weight_kind=kind, m=m, n_coarse=N_STEPS)
        got = _coupled_history(fresh(), cp)
        errs[(kind, cells, m)] = 100.0 * np.linalg.norm(got - ref) / np.linalg.norm(ref)
    names = {0: "constant", 1: "linear", 2: "cubic"}
    print("\nweight    l_O  m  u_x err at A (%)  Table 1 (%), case, beta_PD")
    for key, e in errs.items():
        case, beta_pd, pe = _paper(key)
        print(f"{names[key[0]]:9s} {key[1]}dx {key[2]:2d}  {e:8.3f}          {pe:.2f}  case {case}, beta_PD {beta_pd:g}")
    assert max(errs.values()) < 5.0
    # within 2 percentage points of the printed figure of every case
    assert all(abs(e - _paper(key)[2]) < 2.0 for key, e in errs.items())
    assert errs[(2, 3, 1)] < errs[(0, 1, 1)]
    for m in (2, 5, 10):
        assert abs(errs[(2, 3, m)] - errs[(2, 3, 1)]) < 0.5
    # The lattice with ell = delta / 16 is stiffer along its axes than the
    # continuum it is normalised to; with c0 scaled so that its axial
    # modulus is E, the remaining error is the coupling's own
    ratio = _lattice_axial_modulus_ratio(W.beam3d(dx=DX).pd)
    print(f"PD lattice axial modulus / E = {ratio:.4f}; with c0 / {ratio:.4f}:")
    cal = {}
    for kind, cells, m in STUDY[:9]:
        cp = W.beam3d(dx=DX, overlap_cells=cells, weight_kind=kind, m=m, n_coarse=N_STEPS)
        cp.pd.c /= ratio
        got = _coupled_history(fresh(), cp)
        cal[(kind, cells, m)] = e = 100.0 * np.linalg.norm(got - ref) / np.linalg.norm(ref)
        print(f"{names[kind]:9s} {cells}dx {m:2d}  {e:8.3f}          {_paper((kind, cells, m))[2]:.2f}")
    assert ratio > 1.2 and max(cal.values()) < 5.0
    assert all(abs(e - _paper(key)[2]) < 2.0 for key, e in cal.items())
