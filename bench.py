"""Benchmark of the MTS-coupled PD hot path (bond updates/s, HBM roofline).

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                [--workload coupled|pd|coupled3d|batch] [--accuracy-steps S] [--lattice-tile T]

Default workload (coupled): the fine coupled plate, 0.1 x 0.04 m with a 50 mm
edge pre-crack, a 20 mm PD strip at 0.05 mm (2000 x 400 = 800,000 PD nodes,
22.3M directed bonds), Q4 elements of 0.5 mm elsewhere, 2 mm overlap bands,
12 MPa, FP32-bulk PD with FP64 coupling, m = 20. A step is one coarse step of
Algorithm 1: the FE free step (concurrent stream), 20 PD free substeps (one
CUDA graph), the FP64 interface solve, the FE correction and 20 PD link
substeps. `value` counts every PD bond update (free and link substeps) per
second of device time; coarse steps/s is reported beside it.

--workload pd: the same 800,000-node lattice as a pure PD plate (traction as a
body force on its faces), 20 substeps per step. --workload coupled3d: the 3D
coupled plate (400 x 64 x 8 PD nodes, Hex8 FE, m = 10). --workload batch: 64
seeded coupled plates of uneven size and m, one round per step.

Beside the timed figures the line reports the stated error of FP32-bulk
against the FP64 path on the same workload (displacement rel-L2, bond-status
mismatch, crack-tip error) and the FP64 form's rate with its FP64-ALU
roofline.

Inputs are seeded synthetic data resident in HBM before the timed region; L2
is flushed between timed steps. --impl reference times the FP64 CPU oracle
(the FP64 reference implementation) on the host cores, on bounded samples of the
same lattice. One JSON line is printed by rank 0.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

WORKLOAD = dict(name="pd_strip_2000x400_dx0.05mm_m20_fp32bulk", nx=2000, ny=400, dx=0.05e-3, crack=0.05,
                traction=12e6, dt=5e-9, m=20)
COUPLED_NAME = "coupled_plate_100x40mm_pd2000x400_fe0.5mm_m20_fp32bulk"
COUPLED3D_NAME = "coupled_plate3d_100x40x2mm_pd400x64x8_hex1mm_m10_fp32bulk"
METRIC = "PD bond updates/s"
UNIT = "bond updates/s"


def make_problem():
    from paper_2403_03605_gb300 import workloads as W
    w = WORKLOAD
    return W.strip_lattice_pd(w["nx"], w["ny"], w["dx"], w["crack"], traction=w["traction"], dt=w["dt"],
                              name=w["name"])


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def stored_counters(workload, tile):
    """Per-launch ncu figures of the lattice kernel (DRAM bytes, warp
    instructions, SM-side L2 bytes) stored in profiles/traffic.json, or {} when
    absent or measured on other kernel source; and the L2 sector bandwidth
    ncu reports as the peak of this GPU."""
    tfile = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(tfile) as f:
            tj = json.load(f)
        ent = tj.get(workload, {}).get(str(tile), {})
        return (ent if ent.get("kernel_version") == kernel_version(workload) else {}), tj.get("l2_peak_gbs")
    except Exception:
        return {}, None


def issue_and_l2(ent, launch_ms, clocks, n_sm, l2_peak):
    """Instruction-issue and L2 lines for a kernel whose chain stays in L2:
    warp instructions per launch against the issue peak (one warp instruction
    per cycle on each of the four schedulers of every SM, at the median SM
    clock sampled in the timed region), and the SM-side L2 bytes per launch
    against ncu's nominal L2 sector rate. Per-launch counts are ncu's; the
    launch time is the live CUDA-event figure. A plain device copy between two
    L2-resident 32 MB buffers reaches about 8.2 TB/s on this GPU, so the L2
    fraction reads against a nominal ceiling, not a measured one."""
    mhz = clocks.get("sm_mhz") or 2070.0
    ipeak = n_sm * 4 * mhz * 1e6
    winst = ent.get("warp_instructions_per_launch")
    iach = winst / (launch_ms * 1e-3) if winst else None
    issue = {"warp_instructions_per_launch": winst, "achieved": iach, "peak": ipeak,
             "unit": "warp instructions/s", "frac": iach / ipeak if iach else None,
             "peak_kind": f"{n_sm} SMs x 4 schedulers x {mhz:.0f} MHz (sampled)"}
    lb = ent.get("l2_bytes_per_launch")
    lach = lb / (launch_ms * 1e-3) / 1e9 if lb else None
    l2 = {"bytes_per_launch": lb, "achieved": lach, "peak": l2_peak, "unit": "GB/s",
          "frac": lach / l2_peak if lach and l2_peak else None,
          "peak_kind": "nominal: ncu's peak L2 sector rate on this GPU (188 slices x 3 sectors x 32 B per L2 cycle)",
          "source": "ncu lts__t_sectors_srcunit_tex.sum x 32 B"}
    return issue, l2


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.samples = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.samples.append(parts)

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        mx = [float(s[2]) for s in self.samples if s[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for s in self.samples for k in range(4) if s[5 + k].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples)}


def algorithmic_bytes(info, pb, with_body=True, coupled=False):
    """Bytes one FP32-bulk substep must move with the family layout in use.
    (3D: u and v 24 + 24 B each, a 16 + 16 B, loads 12 B, weight and
    interface force 16 B; the 3D lattice reads four bond words, 16 B.)

    Per node: u (16 in, 16 out), v (16 in, 16 out), a (8 in, 8 out), 1/m (4),
    plus the weighted body force (8) in the pure-PD plate, or the Arlequin
    weight (4) and the interface force (8) in the coupled plate. Lattice
    layout: the family is implicit and the node's 32-bit bond word (one bit
    per bond) is read once. Sliced-ELL layout: per directed bond a 4-byte
    family word and one status bit."""
    nb, n = info["n_bonds"], info["n"]
    if info["dim"] == 3:  # u, v: 24 B pairs (hi xyz + lo xyz); a: 16 B; loads 12 B
        per_node = 24 + 24 + 24 + 24 + 16 + 16 + 4 + (12 if with_body else 0) + (16 if coupled else 0)
        if info["layout"] == 2:  # 3D lattice: four bond words per node, no family list
            return (per_node + 16) * n, per_node + 16
        return 4 * nb + nb / 8.0 + per_node * n, per_node
    per_node = 16 + 16 + 16 + 16 + 8 + 8 + 4 + (8 if with_body else 0) + (12 if coupled else 0)
    if info["layout"] == 1:
        return (per_node + 4) * n, per_node + 4
    return 4 * nb + nb / 8.0 + per_node * n, per_node


def oracle_sample(pb, nsub, setup=None, threads=1):
    """Time `nsub` oracle substeps on this workload (FP64, plain C) on `threads`
    host threads (0: every core; the same bits for any count). Returns (rate,
    seconds, setup, threads used)."""
    import oracle
    if setup is None:
        oracle.set_threads(1)
        rp, col = oracle.family(pb.lat.X, pb.delta)
        mu, _ = oracle.precrack(pb.lat.P, rp, col, [c.in_half_units(pb.lat) for c in pb.cuts])
        opd = oracle.PD(pb.lat.X, pb.vol, pb.delta, pb.c, pb.s0, pb.mat.rho, pb.dt)
        u = np.zeros((pb.dim, pb.n)); v = np.zeros_like(u); a = np.zeros_like(u)
        oracle.pd_run(opd, rp, col, mu, u, v, a, 0, b=pb.b, init=True)
        setup = (rp, col, mu, opd, u, v, a)
    rp, col, mu, opd, u, v, a = setup
    used = oracle.set_threads(threads)
    t0 = time.perf_counter()
    oracle.pd_run(opd, rp, col, mu, u, v, a, nsub, b=pb.b)
    dt = time.perf_counter() - t0
    oracle.set_threads(1)
    return len(col) * nsub / dt, dt, setup, used


def cpu_baseline(workload, what):
    """The FP64 oracle timed on this host on a bounded sample of the workload's
    PD lattice: 20 substeps on one core, then on every core (OpenMP over nodes,
    identical bits) as many substeps as take about as long. The line's value
    is the all-core rate; the one-core rate is kept beside it."""
    _, rpb = reference_problem(workload)
    r1, dt1, setup, _ = oracle_sample(rpb, 20)
    probe, tp, setup, cores = oracle_sample(rpb, 2, setup, threads=0)
    nsub = max(2, min(400, int(round(2 * dt1 / max(tp, 1e-6)))))
    rn, dtn, setup, cores = oracle_sample(rpb, nsub, setup, threads=0)
    return {"value": rn, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{nsub} FP64 oracle PD substeps of {what} ({rpb.n} nodes) on {cores} host threads "
                      f"({dtn:.1f} s; the PD substeps only)",
            "single_core": {"value": r1, "unit": UNIT, "cores": 1,
                            "sample": f"20 substeps of the same lattice on one thread ({dt1:.1f} s)"}}


def reference_problem(workload):
    """(workload name, PD problem) whose PD substeps the oracle samples for a
    workload: the coupled plates' own PD lattices (their loads come through
    the interface, so the sampled substeps start from rest), the pure-PD
    strip for the pd and batch workloads (a batch member is a smaller plate
    of the same kind)."""
    from paper_2403_03605_gb300 import workloads as W
    if workload == "coupled":
        return COUPLED_NAME, W.coupled_plate_2000x400().pd
    if workload == "coupled3d":
        return COUPLED3D_NAME, W.coupled_plate3d_400x64x8().pd
    if workload == "batch":
        return BATCH_NAME.format(n=64), make_problem()
    return WORKLOAD["name"], make_problem()


def run_reference(args, rank, world):
    if rank != 0:
        return
    name, pb = reference_problem(args.workload)
    nsub = 2
    setup = None
    for _ in range(args.warmup):
        _, _, setup, cores = oracle_sample(pb, nsub, setup, threads=0)
    total_t, total_u = 0.0, 0
    for _ in range(args.steps):
        rate, dt, setup, cores = oracle_sample(pb, nsub, setup, threads=0)
        total_t += dt
        total_u += len(setup[1]) * nsub
    value = total_u / total_t
    sample = (f"{nsub} FP64 oracle PD substeps per step of the workload's {pb.n}-node PD lattice on {cores} "
              f"host threads (the PD substeps only: no FE step or interface solve)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total_t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": name, "pd_nodes": pb.n, "directed_bonds": len(setup[1])},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def reduce_job(total_ms, units, world, device=None):
    """Whole-job figures of N replicas (weak scaling): the slowest rank's time
    and the units all ranks processed, divided. Returns (max_ms, units_sum, rate)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(u, op=dist.ReduceOp.SUM)
    tmax, usum = float(t.item()), float(u.item())
    return tmax, usum, usum / (tmax * 1e-3)


def setup_ours(P, ctx, workload):
    """Create the workload through the C ABI; returns (pd, fe, arl, info, pb, m, cp)."""
    from paper_2403_03605_gb300 import workloads as W
    if workload == "pd":
        pb = make_problem()
        m = WORKLOAD["m"]
        pd = P.pd_create(ctx, pb.lat.X, horizon=pb.delta, c=pb.c, s0=pb.s0, rho=pb.mat.rho, vol_uniform=pb.vol,
                         precision=P.PDMTS_FP32_BULK)
        P.pd_set_precrack(pd, [c.as_array() for c in pb.cuts])
        P.pd_set_body_force(pd, pb.b)
        P.mts_set_time(ctx, pb.dt, m)
        return pd, None, None, P.pd_info(pd), pb, m, None
    cp = W.coupled_plate3d_400x64x8() if workload == "coupled3d" else W.coupled_plate_2000x400()
    pd, fe, arl = make_coupled(P, ctx, cp)
    return pd, fe, arl, P.pd_info(pd), cp.pd, cp.m, cp


def make_coupled(P, ctx, cp, precision=None):
    """Bind one coupled plate (FP32-bulk PD unless stated, Q4/Hex8 FE, Arlequin bands) in ctx."""
    pb = cp.pd
    mat = pb.mat
    pd = P.pd_create(ctx, pb.lat.X, horizon=pb.delta, c=pb.c, s0=pb.s0, rho=mat.rho, vol_uniform=pb.vol,
                     micro_kind=pb.extra.get("micro", P.PDMTS_MICRO_POWER), l=pb.extra.get("l", 0.0),
                     precision=P.PDMTS_FP32_BULK if precision is None else precision)
    P.pd_set_precrack(pd, [c.as_array() for c in pb.cuts])
    fe = P.fem_create(ctx, cp.fe.X, cp.fe.conn, E=mat.E, nu=mat.nu, rho=mat.rho, thickness=mat.thickness)
    P.fem_set_traction(fe, cp.faces, cp.face_traction)
    if cp.fixed is not None:
        P.fem_set_fixed(fe, cp.fixed)
    arl = P.arlequin_bind(ctx, pd, fe, cp.weight_kind, [b.as_array() for b in cp.bands])
    P.mts_set_time(ctx, cp.dt_pd, cp.m, cp.gamma_fe, cp.beta_fe)
    return pd, fe, arl


BATCH_NAME = "batch_{n}_coupled_plates_seed3605_pd20k-400k_m5-10-20_fp32bulk"


def shard(work, rank, world):
    """Indices of the independent members rank `rank` of `world` advances.
    `work` holds each member's work per round (PD nodes x m). Largest first,
    each member goes to the rank with the least work so far (lowest rank on a
    tie), so the shards partition the members with balanced work; the job's
    time is the slowest rank's."""
    load = [0.0] * world
    mine = []
    for i in sorted(range(len(work)), key=lambda k: (-work[k], k)):
        r = min(range(world), key=lambda q: (load[q], q))
        load[r] += work[i]
        if r == rank:
            mine.append(i)
    return sorted(mine)


def member_work(cp):
    """PD node updates of one member per round (its m free and m link substeps)."""
    return float(cp.pd.n) * 2 * cp.m


def run_batch(args, rank, world, local_rank):
    """Batched workload: independent coupled plates of uneven size, crack, load
    and m (seeded), advanced one round (one coarse step of each) at a time by
    mts_batch_advance; the per-instance loop over the same rounds is timed
    beside it. With N ranks the members are sharded over them (no collective
    on the data path; the job's rate is the summed units over the slowest
    rank's time)."""
    import torch
    import torch.distributed as dist
    from paper_2403_03605_gb300 import build as B
    from paper_2403_03605_gb300 import pdmts as P
    from paper_2403_03605_gb300 import workloads as W

    B.build()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream(dev)
    t_setup = time.perf_counter()
    all_cps = W.batch_plates(n=args.batch_members)
    cps = [all_cps[i] for i in shard([member_work(cp) for cp in all_cps], rank, world)]
    ctxs, handles = [], []
    for cp in cps:
        ctx = P.pdmts_ctx_create(local_rank, stream.cuda_stream)
        ctxs.append(ctx)
        handles.append(make_coupled(P, ctx, cp))
    batch = P.mts_batch_create(ctxs)
    flush = torch.empty(int(256e6) // 4, dtype=torch.float32, device=dev)
    for _ in range(args.warmup):
        P.mts_batch_advance(batch, 1)
    torch.cuda.synchronize(dev)
    t_setup = time.perf_counter() - t_setup

    def stats_sum():
        sts = [P.pdmts_get_stats(c) for c in ctxs]
        return {k: sum(st[k] for st in sts) for k in sts[0]}

    def timed(advance):
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        stops = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        s0 = stats_sum()
        torch.cuda.synchronize(dev)
        for k in range(args.steps):
            flush.zero_()
            starts[k].record(stream)
            advance()
            stops[k].record(stream)
        torch.cuda.synchronize(dev)
        s1 = stats_sum()
        ms = float(sum(a.elapsed_time(b) for a, b in zip(starts, stops)))
        return ms, {k: s1[k] - s0[k] for k in s1}

    def rebuilds():
        return sum(P.arlequin_info(h[2])["rebuilds"] for h in handles)

    i0 = P.mts_batch_info(batch)
    r0 = rebuilds()
    if world > 1:
        dist.barrier()
    with ClockSampler(local_rank) as clk:
        time.sleep(0.3)
        torch.cuda.nvtx.range_push("timed_steps")
        batch_ms, d = timed(lambda: P.mts_batch_advance(batch, 1))
        torch.cuda.nvtx.range_pop()
    if world > 1:
        dist.barrier()
    i1 = P.mts_batch_info(batch)
    timed_rebuilds = rebuilds() - r0
    own_ms = batch_ms  # this rank's members
    own_value = d["bond_updates"] / (own_ms * 1e-3)
    batch_ms, _, value = reduce_job(own_ms, d["bond_updates"], world, device=dev)  # the job
    _, coarse_total, _ = reduce_job(own_ms, d["coarse_steps"], world, device=dev)
    launches = i1["kernel_launches"] - i0["kernel_launches"]
    solo_ms, ds = timed(lambda: [P.mts_advance(c, 1) for c in ctxs])
    solo_value = ds["bond_updates"] / (solo_ms * 1e-3)

    # end to end: every round also reads every member's PD and FE displacement back to pinned host memory
    outs = [(torch.empty((2, cp.pd.n), dtype=torch.float64).pin_memory(),
             torch.empty(2 * cp.fe.n, dtype=torch.float64).pin_memory()) for cp in cps]
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    s0 = stats_sum()
    e2e_rounds = max(3, min(args.steps, 10))
    for _ in range(e2e_rounds):
        P.mts_batch_advance(batch, 1)
        for (pd, fe, arl), (u, uf) in zip(handles, outs):
            P.pd_read_displacement(pd, u.numpy())
            P.fem_read_displacement(fe, uf.shape[0], uf.numpy())
    torch.cuda.synchronize(dev)
    e2e_s = time.perf_counter() - t0
    _, _, e2e_value = reduce_job(1e3 * e2e_s, stats_sum()["bond_updates"] - s0["bond_updates"], world, device=dev)
    d2h = sum(u.numel() * 8 + uf.numel() * 8 for u, uf in outs)
    info = P.mts_batch_info(batch)
    P.mts_batch_destroy(batch)
    for c in ctxs:
        P.pdmts_ctx_destroy(c)
    if rank != 0:
        return
    accuracy = None
    if args.accuracy_steps != 0 and world == 1:
        accuracy = run_batch_accuracy(P, dev, stream, all_cps, 20 if args.accuracy_steps < 0 else args.accuracy_steps,
                                      args.batch_accuracy_members, args.accuracy_budget_s)
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline("batch", "a plate of the same kind")
    nodes = sum(cp.pd.n for cp in all_cps)
    ms_mix = sorted({cp.m for cp in all_cps})
    # algorithmic bytes of rank 0's PD substeps of the timed rounds (100 B per node and
    # substep, FP32-bulk coupled), over its whole round time: a lower bound on the
    # substeps' own rate
    sub_bytes = 100.0 * sum(2 * cp.m * cp.pd.n for cp in cps) * args.steps
    achieved = sub_bytes / (own_ms * 1e-3) / 1e9
    peak, peak_kind = peaks()
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": batch_ms / args.steps, "higher_is_better": True,
        "scaling": "strong", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": BATCH_NAME.format(n=len(all_cps)), "members": len(all_cps),
                   "members_per_rank": "balanced by PD nodes x m" if world > 1 else len(cps), "pd_nodes_total": nodes,
                   "m_values": ms_mix, "step": "one round = one coarse step of every member",
                   "lattice_tile": info["lattice_tile"], "batched_launches_per_round":
                   (i1["batched_launches"] - i0["batched_launches"]) // max(args.steps, 1),
                   "work_items_per_round": (i1["work_items"] - i0["work_items"]) // max(args.steps, 1),
                   "setup_s": round(t_setup, 2), "l2": "flushed between timed rounds (256 MB write)",
                   "last_round_phase_ms": dict(zip(["lambda0_forces", "free_substeps", "lambda_m", "link_substeps",
                                                    "corrections"], [round(x, 3) for x in i1["last_round_ms"]])),
                   "interface_rebuilds_in_timed_rounds": timed_rebuilds,
                   "per_instance_loop_value": solo_value, "batch_over_loop": own_value / solo_value},
        "coarse_steps_per_s": coarse_total / (batch_ms * 1e-3),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": None, "peak_kind": peak_kind, "kernel": "k_pd_step_lattice2d_batch (whole round)",
                     "algorithmic_bytes_per_step": sub_bytes / args.steps},
        "cpu_baseline": cpu,
        "accuracy": accuracy,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": d2h},
        "gpu_launches": int(launches),
        "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)


def run_ours(args, rank, world, local_rank):
    import torch
    import torch.distributed as dist
    from paper_2403_03605_gb300 import build as B
    from paper_2403_03605_gb300 import pdmts as P

    B.build()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    coupled = args.workload in ("coupled", "coupled3d")
    stream = torch.cuda.current_stream(dev)
    ctx = P.pdmts_ctx_create(local_rank, stream.cuda_stream)
    t_setup = time.perf_counter()
    pd, fe, arl, info, pb, m, cp = setup_ours(P, ctx, args.workload)
    P.pd_set_lattice_tile(pd, args.lattice_tile)
    flush = torch.empty(int(256e6) // 4, dtype=torch.float32, device=dev)  # > L2 (129 MiB)

    for _ in range(args.warmup):  # the first coarse step also builds the interface operator
        P.mts_advance(ctx, 1)
    torch.cuda.synchronize(dev)
    t_setup = time.perf_counter() - t_setup

    # ---- device-timed region: K steps, L2 flushed between steps ----------
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    stops = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    st0 = P.pdmts_get_stats(ctx)
    P.pdmts_get_timing(ctx)
    P.pdmts_set_timing(ctx, True)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    with ClockSampler(local_rank) as clk:
        time.sleep(0.3)
        torch.cuda.nvtx.range_push("timed_steps")  # lets a profiler select the timed launches
        for k in range(args.steps):
            flush.zero_()
            starts[k].record(stream)
            P.mts_advance(ctx, 1)
            stops[k].record(stream)
        torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize(dev)
    P.pdmts_set_timing(ctx, False)
    if world > 1:
        dist.barrier()
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, stops)]
    total_ms = float(sum(step_ms))
    chain_ms, chain_sub = P.pdmts_get_timing(ctx)
    phases, nph = P.mts_get_phase_timing(ctx) if coupled else ({}, 0)
    st1 = P.pdmts_get_stats(ctx)
    launches = st1["kernel_launches"] - st0["kernel_launches"]
    substeps = st1["pd_substeps"] - st0["pd_substeps"]
    units = st1["bond_updates"] - st0["bond_updates"]  # link substeps count only the rows they evaluate
    total_ms, _, value = reduce_job(total_ms, units, world, device=dev)
    coarse_per_s = args.steps * world / (total_ms * 1e-3)

    # ---- roofline of the dominant kernel (the FP32-bulk substep) ----------
    abytes, per_node = algorithmic_bytes(info, pb, with_body=not coupled, coupled=coupled)
    launch_ms = chain_ms / max(chain_sub, 1)
    achieved = abytes / (launch_ms * 1e-3) / 1e9
    peak, peak_kind = peaks()
    tile = P.pd_info(pd)["lattice_tile"]
    # lattice kernel of each tile configuration, as listed at pd_set_lattice_tile
    lat_kernels = ["k_pd_step_lattice2d<false,2,3,false>", "k_pd_step_lattice2d<false,2,4,false>",
                   "k_pd_step_lattice2d_pipe<false,2,2>", "k_pd_step_lattice2d_pipe<false,1,4>",
                   "k_pd_step_lattice2d<false,2,3,true>", "k_pd_step_lattice2d_tma<false,2,4>",
                   "k_pd_step_lattice2d_tma<false,2,3>", "k_pd_step_lattice2d_tpipe<false,2,2>",
                   "k_pd_step_lattice2d_tpipe<false,1,4>", "k_pd_step_lattice2d_tma<false,4,2>"]
    kname = (lat_kernels[tile] if info["layout"] == 1 and tile >= 0 else
             f"k_pd_step_lattice3d<{8 if tile == 1 else 4},{int(coupled)},0>" if info["layout"] == 2
             else f"k_pd_step_f32<{info['dim']}>")
    ent, l2_peak = stored_counters(args.workload, tile)
    traffic = ent.get("dram_bytes_per_launch")
    issue, l2 = issue_and_l2(ent, launch_ms, clk.summary(),
                             torch.cuda.get_device_properties(dev).multi_processor_count, l2_peak)

    # ---- end to end through the C ABI with host buffers ------------------
    # each step: upload a PD body-force field from pinned host memory, advance
    # one coarse step, read the PD (and FE) displacement back into pinned memory
    b_np = np.zeros((pb.dim, pb.n)) if coupled else np.ascontiguousarray(pb.b)
    b_host = torch.from_numpy(b_np).pin_memory()
    u_host = torch.empty((pb.dim, pb.n), dtype=torch.float64).pin_memory()
    nfe_dof = pb.dim * cp.fe.n if coupled else 0
    uf_host = torch.empty(max(nfe_dof, 1), dtype=torch.float64).pin_memory()
    P.pd_set_body_force(pd, b_host)  # first upload allocates the load arrays (outside the timing)
    e2e_steps = max(3, min(args.steps, 10))
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    st2 = P.pdmts_get_stats(ctx)
    for _ in range(e2e_steps):
        P.pd_set_body_force(pd, b_host)
        P.mts_advance(ctx, 1)
        P.pd_read_displacement(pd, u_host.numpy())
        if coupled:
            P.fem_read_displacement(fe, nfe_dof, uf_host.numpy())
    torch.cuda.synchronize(dev)
    e2e_s = time.perf_counter() - t0
    e2e_units = P.pdmts_get_stats(ctx)["bond_updates"] - st2["bond_updates"]
    e2e_value = e2e_units * world / e2e_s
    assert np.isfinite(u_host.numpy()).all()

    # ---- stated error of FP32-bulk and the plain FP64 form's rate ---------
    accuracy, fp64_form = (None, None)
    if args.accuracy_steps != 0:
        accuracy, fp64_form = run_accuracy(P, dev, stream, args.workload, args.accuracy_steps,
                                           args.accuracy_budget_s)
        if args.workload == "coupled":
            from paper_2403_03605_gb300 import workloads as W
            accuracy["full_length"] = run_accuracy_full_length(P, dev, stream, W.coupled_plate_400x64(),
                                                               args.accuracy_budget_s)

    # ---- CPU baseline: the FP64 oracle on a bounded sample ----------------
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args.workload, "the workload's PD lattice")

    if rank == 0:
        cfg = {"workload": (COUPLED3D_NAME if args.workload == "coupled3d" else COUPLED_NAME) if coupled
               else WORKLOAD["name"], "pd_nodes": pb.n,
               "directed_bonds": info["n_bonds"], "m": m,
               "family_layout": {0: "sliced ELL", 1: "lattice bond words", 2: "3D lattice bond words"}[info["layout"]],
               "lattice_tile": tile,
               "link_tile": P.pd_info(pd)["link_tile"] if coupled else None,
               "graph": "one captured graph per PD substep chain",
               "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
               "l2": "flushed between timed steps (256 MB write)",
               "l2_bytes": getattr(torch.cuda.get_device_properties(dev), "L2_cache_size", None)}
        if coupled:
            ai = P.arlequin_info(arl)
            cfg.update({"phase_us_per_step": {k: round(v * 1e3 / max(nph, 1), 1) for k, v in phases.items()}})
            cfg.update({"fe_dofs": ai["fe_dofs"], "n_lambda": ai["n_lambda"],
                        "pd_substeps_per_step": substeps // args.steps, "setup_s": round(t_setup, 2),
                        "interface_builds": ai["rebuilds"]})
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": cfg,
            "coarse_steps_per_s": coarse_per_s if coupled else None,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic, "peak_kind": peak_kind, "kernel": kname,
                         "algorithmic_bytes_per_launch": abytes, "launch_us": launch_ms * 1e3},
            "issue_rate": issue,
            "l2_bandwidth": l2,
            "cpu_baseline": cpu,
            "accuracy": accuracy,
            "fp64_form": fp64_form,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(b_host.numel() * 8),
                    "d2h_bytes_per_step": int(u_host.numel() * 8 + nfe_dof * 8)},
            "gpu_launches": int(launches),
            "clocks": clk.summary(),
        }
        print(json.dumps(line), flush=True)
    P.pdmts_ctx_destroy(ctx)


# crack plane (normal axis, level, along axis) and the half-width of the band
# searched for the crack tip: up to the inner edges of the overlap bands
# (coupled plates) or a quarter of the strip's height (pure-PD strip)
ACCURACY_CRACK = {"coupled": ((1, 0.020, 0), 8e-3), "coupled3d": ((1, 0.020, 0), 6e-3),
                  "pd": ((1, 0.010, 0), 5e-3)}


def run_accuracy(P, dev, stream, workload, n_steps, budget_s):
    """The stated error of the FP32-bulk path and the rate of the plain FP64
    form: the same workload advanced from rest by a fresh FP64 context and a
    fresh FP32-bulk context (the FP64 path is bit-identical to the FP64 oracle
    in the parity tests), coarse step by coarse step (pure PD: chains of m
    substeps). The FP64 run stops after n_steps or once it has used budget_s
    seconds of wall time, and the FP32-bulk run takes the same number of
    steps. Reports displacement rel-L2, bond-status mismatch and crack-tip
    error of FP32-bulk against FP64 at the end, and both forms' bond
    updates/s over steps 2.. (device time, CUDA events on the caller's
    stream; the first step also builds the interface operator)."""
    import torch
    from paper_2403_03605_gb300 import diagnostics as D
    from paper_2403_03605_gb300 import workloads as W
    coupled = workload in ("coupled", "coupled3d")
    cp = (W.coupled_plate3d_400x64x8() if workload == "coupled3d" else W.coupled_plate_2000x400()) if coupled else None
    if n_steps < 0:
        n_steps = {"coupled": 60, "coupled3d": 30, "pd": 100}[workload]
    n_steps = max(n_steps, 2)
    res = {}
    for name, prec in (("fp64", P.PDMTS_FP64), ("fp32_bulk", P.PDMTS_FP32_BULK)):
        ctx = P.pdmts_ctx_create(dev.index, stream.cuda_stream)
        try:
            if coupled:
                pd, fe, arl = make_coupled(P, ctx, cp, precision=prec)
                pb = cp.pd
            else:
                pb = make_problem()
                pd = P.pd_create(ctx, pb.lat.X, horizon=pb.delta, c=pb.c, s0=pb.s0, rho=pb.mat.rho,
                                 vol_uniform=pb.vol, precision=prec)
                P.pd_set_precrack(pd, [c.as_array() for c in pb.cuts])
                P.pd_set_body_force(pd, pb.b)
                P.mts_set_time(ctx, pb.dt, WORKLOAD["m"])
            t0 = time.perf_counter()
            P.mts_advance(ctx, 1)  # the first coarse step also builds the interface operator
            torch.cuda.synchronize(dev)
            st0 = P.pdmts_get_stats(ctx)
            P.pdmts_get_timing(ctx)
            P.pdmts_set_timing(ctx, True)
            ms, done = 0.0, 1
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            while done < n_steps:
                e0.record(stream)
                P.mts_advance(ctx, 1)
                e1.record(stream)
                torch.cuda.synchronize(dev)
                ms += e0.elapsed_time(e1)
                done += 1
                if name == "fp64" and time.perf_counter() - t0 > budget_s:
                    n_steps = done  # the FP32-bulk run takes as many steps
            P.pdmts_set_timing(ctx, False)
            chain_ms, chain_sub = P.pdmts_get_timing(ctx)
            st1 = P.pdmts_get_stats(ctx)
            units = st1["bond_updates"] - st0["bond_updates"]
            out = {"u": P.pd_read_displacement(pd), "mu": P.pd_read_bond_status(pd)[0],
                   "phi": P.pd_read_damage(pd), "ms": ms, "steps": done, "value": units / (ms * 1e-3),
                   "chain_ms": chain_ms, "chain_sub": chain_sub, "units": units}
            if coupled:
                out["uf"] = P.fem_read_displacement(fe, pb.dim * cp.fe.n)
                out["rebuilds"] = P.arlequin_info(arl)["rebuilds"]
            res[name] = out
        finally:
            P.pdmts_ctx_destroy(ctx)
    crack, band = ACCURACY_CRACK[workload]
    acc = D.compare(res["fp32_bulk"], res["fp64"], pb.lat.X, crack, band)
    acc = {k: (round(v, 12) if isinstance(v, float) else v) for k, v in acc.items()}
    steps = res["fp64"]["steps"]
    acc.update({"vs": "FP64 GPU path (bit-identical to the FP64 oracle in the parity tests)",
                "coarse_steps" if coupled else "chains": steps,
                "physical_time_s": steps * (cp.m * cp.dt_pd if coupled else WORKLOAD["m"] * WORKLOAD["dt"]),
                "crack_tip_rule": f"extreme x of nodes with damage >= 0.35 within {band * 1e3:g} mm of the crack plane",
                "tolerance": {"u_pd_rel_l2": 1e-4, "broken_mismatch_frac": 1e-3}})
    if coupled:
        acc["interface_builds"] = {k: res[k]["rebuilds"] for k in res}
    r64 = res["fp64"]
    # the FP64 parity kernel evaluates each intact bond with 26 FP64 adds,
    # multiplies and compares in 2D (30 with Arlequin weights; 3D: 37 and 41),
    # each taking one FMA slot of the FP64 pipe: peak = the nominal 1.25
    # TFLOP/s (152 SMs x 2 FP64 FMA per clock x 2.07 GHz x 2 flops) / 2
    # the timed chains are the free chains (every substep evaluates every
    # intact bond of the subdomain; link chains are not timed)
    ops = {2: 26, 3: 37}[pb.dim] + (4 if coupled else 0)
    # the method's own minimum per bond (no per-bond micromodulus: 2 sub xi,
    # 2 sub eta, 2 xi.eta, 4 |xi+eta|^2, 2 |xi|^2, 2 compare/scale, 4 force
    # and accumulate in 2D; 26 in 3D)
    ops_min = {2: 18, 3: 26}[pb.dim]
    chain_s = r64["chain_ms"] * 1e-3
    intact = int(np.count_nonzero(r64["mu"]))
    achieved = ops * intact * r64["chain_sub"] / chain_s / 1e9 if chain_s > 0 else None
    achieved_min = ops_min * intact * r64["chain_sub"] / chain_s / 1e9 if chain_s > 0 else None
    peak = 1250.0 / 2
    fp64 = {"value": r64["value"], "unit": UNIT, "ms_per_step": r64["ms"] / (steps - 1),
            "fp32_bulk_value_same_steps": res["fp32_bulk"]["value"],
            "fp32_bulk_over_fp64": res["fp32_bulk"]["value"] / r64["value"],
            "steps_timed": steps - 1,
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "G FP64 ops/s",
                         "frac": achieved / peak if achieved else None, "traffic": None,
                         "peak_kind": "nominal FP64 rate 1.25 TFLOP/s (FMA = 2 flops) / 2: each non-fused op "
                                      "takes one FMA slot",
                         "kernel": f"k_pd_step_f64<{pb.dim}>", "ops_per_bond": ops,
                         "ops_per_bond_method_minimum": ops_min,
                         "frac_at_method_minimum": achieved_min / peak if achieved_min else None,
                         "launch_us": 1e3 * r64["chain_ms"] / max(r64["chain_sub"], 1),
                         "time_basis": "free substep chains (CUDA events around each chain) x the bonds "
                                       "intact at the end of the run"}}
    return acc, fp64


def run_accuracy_full_length(P, dev, stream, cp, budget_s):
    """FP32-bulk against FP64 over a coupled configuration's whole length
    (cp.n_coarse coarse steps) on the 100 x 40 mm plate at dx = 0.25 mm (25,600
    PD nodes, m = 10, 200 coarse steps), where the FP64 run and its interface
    rebuilds fit a bench; the FP64 run stops early only past budget_s."""
    from paper_2403_03605_gb300 import diagnostics as D
    res = {}
    n_steps = cp.n_coarse
    for name, prec in (("fp64", P.PDMTS_FP64), ("fp32_bulk", P.PDMTS_FP32_BULK)):
        ctx = P.pdmts_ctx_create(dev.index, stream.cuda_stream)
        try:
            pd, fe, arl = make_coupled(P, ctx, cp, precision=prec)
            t0, done = time.perf_counter(), 0
            while done < n_steps:
                P.mts_advance(ctx, 1)
                done += 1
                if name == "fp64" and done % 10 == 0:
                    P.pdmts_get_stats(ctx)  # synchronises: the budget counts device time
                    if time.perf_counter() - t0 > budget_s:
                        n_steps = done
            res[name] = {"u": P.pd_read_displacement(pd), "mu": P.pd_read_bond_status(pd)[0],
                         "phi": P.pd_read_damage(pd), "uf": P.fem_read_displacement(fe, cp.pd.dim * cp.fe.n),
                         "steps": done, "rebuilds": P.arlequin_info(arl)["rebuilds"],
                         "wall_s": time.perf_counter() - t0}
        finally:
            P.pdmts_ctx_destroy(ctx)
    crack, band = ACCURACY_CRACK["coupled"]
    acc = D.compare(res["fp32_bulk"], res["fp64"], cp.pd.lat.X, crack, band)
    acc = {k: (round(v, 12) if isinstance(v, float) else v) for k, v in acc.items()}
    acc.update({"workload": "coupled_plate_100x40mm_pd400x64_fe1mm_m10", "coarse_steps": res["fp64"]["steps"],
                "configuration_length": cp.n_coarse, "physical_time_s": res["fp64"]["steps"] * cp.m * cp.dt_pd,
                "interface_builds": {k: res[k]["rebuilds"] for k in res},
                "wall_s": {k: round(res[k]["wall_s"], 1) for k in res},
                "tolerance": {"u_pd_rel_l2": 1e-4, "broken_mismatch_frac": 1e-3}})
    return acc


def run_batch_accuracy(P, dev, stream, all_cps, n_rounds, n_members, budget_s):
    """The stated error of the batched FP32-bulk path: a spread of members of
    the batched workload (every len/n-th, so sizes and m vary) advanced as one
    FP32-bulk batch from rest for n_rounds rounds, each compared with its own
    FP64 solo run of the same coarse steps (the FP64 path is bit-identical to
    the FP64 oracle in the parity tests). Members are added while the FP64
    runs stay within budget_s of wall time. Reports the worst member and each
    member's figures."""
    import torch
    from paper_2403_03605_gb300 import diagnostics as D
    n_rounds = max(n_rounds, 1)
    stride = max(1, len(all_cps) // max(n_members, 1))
    pick = list(range(0, len(all_cps), stride))[:n_members]
    t0 = time.perf_counter()
    ref = {}
    for k in pick:  # FP64 solo runs, within the budget
        if ref and time.perf_counter() - t0 > budget_s:
            break
        cp = all_cps[k]
        ctx = P.pdmts_ctx_create(dev.index, stream.cuda_stream)
        try:
            pd, fe, arl = make_coupled(P, ctx, cp, precision=P.PDMTS_FP64)
            P.mts_advance(ctx, n_rounds)
            ref[k] = {"u": P.pd_read_displacement(pd), "mu": P.pd_read_bond_status(pd)[0],
                      "phi": P.pd_read_damage(pd), "uf": P.fem_read_displacement(fe, cp.pd.dim * cp.fe.n),
                      "rebuilds": P.arlequin_info(arl)["rebuilds"]}
        finally:
            P.pdmts_ctx_destroy(ctx)
    fp64_s = time.perf_counter() - t0
    members = sorted(ref)
    ctxs, handles = [], []
    for k in members:
        ctx = P.pdmts_ctx_create(dev.index, stream.cuda_stream)
        ctxs.append(ctx)
        handles.append(make_coupled(P, ctx, all_cps[k]))
    batch = P.mts_batch_create(ctxs)
    rows = []
    try:
        P.mts_batch_advance(batch, n_rounds)
        torch.cuda.synchronize(dev)
        crack, band = ACCURACY_CRACK["coupled"]
        for k, (pd, fe, arl) in zip(members, handles):
            cp = all_cps[k]
            got = {"u": P.pd_read_displacement(pd), "mu": P.pd_read_bond_status(pd)[0],
                   "phi": P.pd_read_damage(pd), "uf": P.fem_read_displacement(fe, cp.pd.dim * cp.fe.n)}
            acc = D.compare(got, ref[k], cp.pd.lat.X, crack, band)
            rows.append({"member": k, "pd_nodes": cp.pd.n, "m": cp.m, "u_pd_rel_l2": acc["u_pd_rel_l2"],
                         "u_fe_rel_l2": acc.get("u_fe_rel_l2"), "broken_mismatch_frac": acc["broken_mismatch_frac"],
                         "n_broken_ref": acc["n_broken_ref"], "crack_tip_error_m": acc["crack_tip_error_m"],
                         "interface_builds": {"fp64": ref[k]["rebuilds"], "fp32_bulk": P.arlequin_info(arl)["rebuilds"]}})
    finally:
        P.mts_batch_destroy(batch)
        for c in ctxs:
            P.pdmts_ctx_destroy(c)
    def worst(key):
        vals = [r[key] for r in rows if r.get(key) is not None and not (isinstance(r[key], float) and np.isnan(r[key]))]
        return max(vals) if vals else None
    return {"vs": "each member's FP64 solo GPU run (bit-identical to the FP64 oracle in the parity tests)",
            "members_compared": len(rows), "members_in_batch": len(all_cps), "coarse_steps": n_rounds,
            "u_pd_rel_l2": worst("u_pd_rel_l2"), "u_fe_rel_l2": worst("u_fe_rel_l2"),
            "broken_mismatch_frac": worst("broken_mismatch_frac"), "crack_tip_error_m": worst("crack_tip_error_m"),
            "tolerance": {"u_pd_rel_l2": 1e-4, "broken_mismatch_frac": 1e-3},
            "fp64_wall_s": round(fp64_s, 1), "per_member": rows}


def kernel_version(workload="coupled"):
    """Hash of the source of the lattice kernel a workload runs (2D: the 2D
    kernel files; 3D: the 3D kernel and the headers it includes): a stored
    ncu figure is only reported while that kernel is unchanged."""
    import hashlib
    names = (("lattice3d.cu", "lattice2d.cuh", "f32_device.cuh") if workload == "coupled3d"
             else ("lattice2d.cuh", "f32_device.cuh", "lattice2d_tma.cu"))
    h = hashlib.sha256()
    for name in names:
        with open(os.path.join(ROOT, "paper_2403_03605_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", choices=["coupled", "pd", "batch", "coupled3d"], default="coupled")
    ap.add_argument("--batch-members", type=int, default=64, help="members of the batched workload")
    ap.add_argument("--batch-accuracy-members", type=int, default=8,
                    help="batch members compared with their FP64 solo runs (a spread over the list)")
    ap.add_argument("--accuracy-steps", type=int, default=-1,
                    help="coarse steps (pure PD: chains) of the FP32-bulk vs FP64 accuracy run; "
                         "-1: 60 (coupled), 30 (coupled3d), 100 (pd); 0: skip")
    ap.add_argument("--accuracy-budget-s", type=float, default=60.0,
                    help="wall-time budget of the FP64 accuracy run (it stops early past it)")
    ap.add_argument("--lattice-tile", type=int, default=-1,
                    help="fix the lattice kernel tile configuration (default: autotune)")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    try:
        if args.workload == "batch":
            run_batch(args, rank, world, local_rank)
        else:
            run_ours(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
