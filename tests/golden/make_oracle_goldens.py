"""Write tests/golden/oracle_plate_100x100.json: a summary of the FP64 oracle's
500-step run of the 100 x 100 pre-cracked plate (12 MPa, dt 25 ns). Calls only
oracle/ and the seeded input generators. The CPU test that reads it catches an
unintended change of the oracle's arithmetic; an intended change regenerates
it, and its commit names the passage that justifies it.

    python tests/golden/make_oracle_goldens.py
"""
import hashlib
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2403_03605_gb300 import workloads as W  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_plate_100x100.json")


def run():
    pb = W.plate_100x100()
    rp, col = oracle.family(pb.lat.X, pb.delta)
    mu, ncut = oracle.precrack(pb.lat.P, rp, col, [c.in_half_units(pb.lat) for c in pb.cuts])
    pd = oracle.PD(pb.lat.X, pb.vol, pb.delta, pb.c, pb.s0, pb.mat.rho, pb.dt)
    u = np.zeros((2, pb.n)); v = np.zeros_like(u); a = np.zeros_like(u)
    broken = oracle.pd_run(pd, rp, col, mu, u, v, a, pb.nsteps, b=pb.b, init=True)
    phi = oracle.damage(pd, rp, col, mu)
    digest = hashlib.sha256(u.tobytes() + v.tobytes() + a.tobytes() + mu.tobytes()).hexdigest()
    return {"workload": "plate_100x100 (100 x 100 nodes, dx 0.5 mm, centred 10 mm pre-crack, 12 MPa, "
                        "dt 25 ns, 500 steps)",
            "directed_bonds": int(len(col)), "precut": int(ncut), "broken_by_dynamics": int(broken),
            "intact_at_end": int(mu.sum()), "damaged_nodes_phi_ge_0.35": int(np.count_nonzero(phi >= 0.35)),
            "max_abs_u": float(np.abs(u).max()), "state_sha256": digest}


if __name__ == "__main__":
    with open(OUT, "w") as f:
        json.dump(run(), f, indent=1)
    print(open(OUT).read())
