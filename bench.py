#!/usr/bin/env python3
"""Benchmark of the fragment-kMC hot path (arXiv:2004.09081) on GB300.

Workload (default): 256 uneven BaTiO(3-x)H_x replicas (16^3..48^3 cells,
x ~ U[0,0.3], vacancies ~ U[0.1,1]%, T ~ U[300,1000] K, barriers 0.70/0.35 eV)
in one batch, mixed precision.  One step = `--windows` synchronisation
windows over the whole batch (8 colour phases each: rates, BKL selection,
exchange, hand-off) followed by the batch-wide displacement-moment reduction
that D comes from.  The lattice state stays resident; L2 is flushed (256 MiB
write) between timed steps.

Prints one JSON line.  `--impl reference` times the CPU oracle instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "hops/s on 1 GB300 (batched mixed vs plain FP64) at D within 1%; HBM roofline frac"
UNIT = "hops/s"
# algorithmic bytes per hop at 32-byte sector granularity: the 8 neighbour words of
# the vacancy's site (one sector each), the two site words written and its record
B_ALG_PER_HOP = 160
# site-energy path: + the energy field, 4-byte words: 9 reads (the vacancy's site and
# its 8 targets) and a read-modify-write of the 2 x 58 V-V partners moved with the hop
B_ALG_PER_HOP_SITE = 160 + 4 * (9 + 2 * 2 * 58)
# electrostatics alone: the 9 energy-field reads, no partners to move
B_ALG_PER_HOP_ELEC = 160 + 4 * 9


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--windows", type=int, default=0, help="windows per step (0: the workload's default)")
    p.add_argument("--seed", type=int, default=0)
    p.add_argument("--no-plain", action="store_true", help="skip the plain FP64 comparison leg")
    p.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    p.add_argument("--workload", default="batched",
                   choices=["batched", "sweep", "bulk", "um", "fe", "null", "htrend", "umgrains", "elec"],
                   help="batched: 256 uneven replicas (the headline); sweep: SrTiO(3-x)H_x 32^3 at "
                        "300..700 K; bulk: BaTiO(3-x)H_x 128^3; um: BaTiO3 L^3 under bias; fe: Fe-doped "
                        "SrTiO3 96^3 with vacancy-vacancy and vacancy-Fe site energies at 600..1000 K; null: "
                        "the bulk lattice with the paper's atom-based null-event kMC, one pick per vacancy; "
                        "htrend: the paper's 24 hydride runs (Table 2 trend), 32^3 each; umgrains: the paper's "
                        "1600x400x2400-cell BaTiO3 model with Voronoi grains under bias; elec: BaTiO3 128^3 with "
                        "the multigrid potential of the vacancy charges")
    p.add_argument("--um-cells", type=int, default=2500, help="edge of the um-scale cube (cells)")
    p.add_argument("--no-autotune", action="store_true", help="use the workload's default edge")
    p.add_argument("--profile-run", action="store_true",
                   help="timed steps only (no e2e, physics, comparison or CPU legs): for profiler launch lists")
    return p.parse_args()


def dist_setup(want_cuda: bool):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if want_cuda else "gloo")
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def allreduce_max(v: float, ws: int, device) -> float:
    if ws == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def allreduce_sum(v: float, ws: int, device) -> float:
    if ws == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader",
                                       "-i", str(gpu_index), "-lms", "200"], stdout=self.f,
                                      stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1].split()[0]))
                smax.append(float(parts[2].split()[0]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.f.name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ helpers
def make_batch(fk, wl, seed, precision, replicas=None, edge=None, tracer=None, site=True, **opts):
    reps = wl.replicas if replicas is None else [wl.replicas[i] for i in replicas]
    nf = reps[0].nfrag if (len(reps) == 1 and reps[0].nfrag) else None
    opts.setdefault("n_tau", wl.n_tau)
    b = fk.Batch([(*r.cells, r.a) for r in reps], [(r.n_vac, r.n_H, r.n_Fe) for r in reps], seed,
                 edge=wl.edge if edge is None else edge, nfrag=nf, precision=precision,
                 tracer=wl.tracer if tracer is None else tracer, **opts)
    if wl.site and site:
        b.set_site_energy(wl.site["vv"], wl.site["fe"])
    if "grains" in wl.notes:
        b.set_grains(*wl.notes["grains"])
    b.set_barriers([r.Ea_O for r in reps], [r.Ea_H for r in reps], [r.T for r in reps],
                   field_z=[r.field_z for r in reps])
    if "elec" in wl.notes and precision == 0:
        b.set_electrostatics(**wl.notes["elec"])
    return b


def D_from_moments(m, t, a):
    """D = <|d|^2>/(6t) (m^2/s) from the integer moments of one replica."""
    h = 0.5 * a * 1e-10
    return (m[4] + m[5] + m[6]) / max(m[0], 1) * h * h / (6 * t)


def cpu_oracle_null_rate(wl, seed, steps, budget_s):
    """The oracle's null-event form on the workload's lattice, `steps` at a time,
    until the budget is spent; returns (hops/s, hops, seconds)."""
    import oracle
    oracle.build()
    rep = wl.replicas[0]
    L = oracle.Lattice(rep.cells, rep.nfrag, rep.n_vac, rep.n_H, seed=seed)
    L.set_rates(rep.Ea_O, rep.Ea_H, rep.T, a_ang=rep.a, precision=wl.precision)
    secs = 0.0
    while secs < budget_s:
        t0 = time.perf_counter()
        L.null_run(steps, wl.notes["n_frg"])
        secs += time.perf_counter() - t0
    hops = L.counters()["hops"]
    return hops / secs, hops, secs


def cpu_oracle_rate(wl, seed, windows, budget_s, replicas=None):
    """Time the CPU oracle (one core, as written) on replicas of the workload,
    `windows` at a time, until the budget is spent; returns (hops/s, hops,
    seconds, replica-runs done)."""
    import oracle
    oracle.build()
    order = list(range(len(wl.replicas))) if replicas is None else list(replicas)
    hops, secs, done = 0, 0.0, 0
    cap = _auto_cap(wl)
    while secs < budget_s:
        for r in order:
            rep = wl.replicas[r]
            nf = rep.nfrag or oracle.partition(rep.cells, wl.edge)
            L = oracle.Lattice(rep.cells, nf, rep.n_vac, rep.n_H, seed=seed, replica=r, n_Fe=rep.n_Fe)
            if wl.site:
                L.set_site_energy(vv=wl.site["vv"], fe=wl.site["fe"])
            L.set_rates(rep.Ea_O, rep.Ea_H, rep.T, Ez=rep.field_z, a_ang=rep.a, cap_v=cap,
                        n_tau=wl.n_tau, precision=wl.precision)
            if "grains" in wl.notes:
                L.set_grains(*wl.notes["grains"])
            refresh = None
            if "elec" in wl.notes:  # the oracle's own potential (exact FFT solve), re-solved like the GPU's
                from oracle import poisson as ps
                el = wl.notes["elec"]
                g = ps.self_table(rep.cells, rep.a, el["eps_r"], oracle.neighbour_table(), q=el["q_vac"])

                def refresh(lat=L, el=el, g=g, rep=rep, ps=ps):
                    phi = ps.solve(ps.node_charge(rep.cells, lat.records()[:, 1], q=el["q_vac"]), rep.a, el["eps_r"])
                    lat.set_elec(ps.energy_units(ps.site_potential(phi), q=el["q_vac"]).astype(np.int32), g)
            while True:  # single lattices keep running until the budget is spent
                t0 = time.perf_counter()
                if refresh is None:
                    L.run(windows)
                else:
                    for _ in range(max(1, windows // wl.notes["elec"]["refresh_windows"])):
                        refresh()
                        L.run(wl.notes["elec"]["refresh_windows"])
                secs += time.perf_counter() - t0
                if len(order) > 1 or secs >= budget_s:
                    break
            hops += L.counters()["hops"]
            done += 1
            if secs >= budget_s:
                break
    return hops / secs if secs > 0 else 0.0, hops, secs, done


def oracle_jobs(wl, seed):
    """Every replica of the workload as a job for the parallel oracle timing."""
    import oracle
    from oracle import timing
    cap = _auto_cap(wl)
    return [timing.replica_job(r, rep.cells, rep.nfrag or oracle.partition(rep.cells, wl.edge), rep.n_vac,
                               rep.n_H, rep.T, rep.Ea_O, rep.Ea_H, rep.field_z, rep.a, cap, wl.precision, seed,
                               rep.n_Fe, wl.site or None, wl.n_tau)
            for r, rep in enumerate(wl.replicas)]


def _auto_cap(wl):
    """The library's default vacancy slots per fragment (kmc_opts.cap_v = 0)
    for the oracle legs, from the oracle's own partition."""
    import oracle
    worst = 0.0
    for r in wl.replicas:
        nf = r.nfrag or oracle.partition(r.cells, wl.edge)
        worst = max(worst, r.n_vac / (nf[0] * nf[1] * nf[2]))
    cap = int(math.ceil(worst + 10.0 * math.sqrt(worst + 1.0) + 8.0))
    cap = ((cap + 7) // 8) * 8
    return min(256, max(8, cap))


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def kernel_source_hash(names=None) -> str:
    """sha256 over the named CUDA sources (default: all of them); a traffic figure
    taken on other sources is stale."""
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2004_09081_gb300", "csrc")
    for name in sorted(names or os.listdir(csrc)):
        if name.endswith((".cu", ".cuh", ".h")):
            with open(os.path.join(csrc, name), "rb") as f:
                h.update(name.encode() + b"\0" + f.read())
    return h.hexdigest()


def load_counters(kernel_tag):
    """The committed ncu figures of a kernel (profiles/traffic.json), or None when
    absent or taken on different kernel sources."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    e = d.get(kernel_tag)
    if e is None or e.get("source_sha256") != kernel_source_hash(e.get("sources")):
        return None
    return e


def load_traffic(kernel_tag):
    """dram__bytes_read.sum + dram__bytes_write.sum per launch from the committed
    ncu summary, or None when absent or stale."""
    e = load_counters(kernel_tag)
    return e.get("bytes_per_launch") if e else None


# ------------------------------------------------------------------ reference arm
def run_reference(args):
    from paper_2004_09081_gb300 import workloads
    ws, rank, _ = dist_setup(False)
    if rank != 0:
        return
    from oracle import timing
    wl = workloads.batched_batio3(args.seed)
    nrep = len(wl.replicas)
    args.windows = args.windows or wl.windows
    per_step_budget = 8.0
    times, hops_all, reps_done = [], 0, 0
    jobs = oracle_jobs(wl, args.seed)
    cores = 1
    for k in range(args.warmup + args.steps):
        # the replicas are independent: one serial oracle per host core, each step
        # starting further along the replica list
        shift = (k * 37) % nrep
        rate, hops, secs, done, cores = timing.parallel_rate(jobs[shift:] + jobs[:shift], args.windows,
                                                             per_step_budget)
        if k >= args.warmup:
            times.append(secs)
            hops_all += hops
            reps_done += done
    total = sum(times)
    value = hops_all / total if total > 0 else 0.0
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / max(args.steps, 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64+u64",
        "data": "synthetic",
        "config": {"workload": wl.name, "replicas": nrep, "windows_per_step": args.windows,
                   "precision": "mixed", "edge": wl.edge, "n_tau": wl.n_tau},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{reps_done} replica runs of {args.windows} windows each over "
                                   f"{args.steps} steps, one serial C oracle per process on {cores} "
                                   f"processes (~{per_step_budget:.0f} s each per step)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


# ------------------------------------------------------------------ our arm
def physics_report(fkmc, b, wl):
    """The observables each workload is quoted with (Sec. Computational details):
    D of V (and O, H- with tracer), drift and the Arrhenius fit of the T sweep."""
    out = []
    if wl.name.startswith("h_trend"):
        return h_trend_report(fkmc, b, wl)
    if len(wl.replicas) > 8:
        return {"replicas": None, "note": "per-replica D in D_mixed_vs_plain; not listed for large batches"}
    for r, rep in enumerate(wl.replicas):
        row = {"T": rep.T, "cells": rep.cells[0], "n_vac": rep.n_vac, "n_H": rep.n_H}
        Dx, D, Dxy, v = b.D(r, fkmc.FKMC_V)
        row.update({"D_V": D, "D_V_z": Dx[2], "D_V_xy": Dxy, "v_z_V": float(v[2]),
                    "D_V_z_definition": "(<dz^2> - <dz>^2) / (2t), drift removed"})
        if wl.tracer:
            for sp, nm in ((fkmc.FKMC_O, "O"), (fkmc.FKMC_H, "H")):
                if nm == "H" and rep.n_H == 0:
                    continue
                row["D_" + nm] = b.D(r, sp)[1]
        out.append(row)
    rep = {"replicas": out}
    if wl.name.startswith("srtio3h_32c_Tsweep"):
        kB = 8.617333262e-5
        for nm in ("D_V", "D_O", "D_H"):
            pts = [(1.0 / o["T"], math.log(o[nm])) for o in out if o.get(nm, 0) > 0]
            if len(pts) >= 2:
                x, y = np.array(pts).T
                rep["Ea_apparent_" + nm[2:] + "_eV"] = float(-np.polyfit(x, y, 1)[0] * kB)
    return rep


def h_trend_report(fkmc, b, wl):
    """Apparent barriers of the hydride runs: Arrhenius fits of D_H and D_O over
    550..700 K for each material and H- fraction, beside the paper's Table 2."""
    from paper_2004_09081_gb300 import workloads
    kB = 8.617333262e-5
    rows, k = [], 0
    for mi, mat in enumerate(wl.notes["materials"]):
        for x in wl.notes["x"]:
            pts = {"H": [], "O": [], "V": []}
            Ds = []
            for T in wl.notes["T"]:
                d = {nm: b.D(k, sp)[1] for sp, nm in ((fkmc.FKMC_H, "H"), (fkmc.FKMC_O, "O"), (fkmc.FKMC_V, "V"))}
                for nm, v in d.items():
                    if v > 0:
                        pts[nm].append((1.0 / T, math.log(v)))
                Ds.append({"T": T, "D_H": d["H"], "D_O": d["O"], "D_V": d["V"]})
                k += 1
            row = {"material": mat, "x": x, "paper_Ea_H_eV": workloads.PAPER_TABLE2[x][mi], "D": Ds}
            for nm in ("H", "O", "V"):
                if len(pts[nm]) >= 2:
                    xs, ys = np.array(pts[nm]).T
                    row["Ea_app_" + nm + "_eV"] = float(-np.polyfit(xs, ys, 1)[0] * kB)
            rows.append(row)
    return {"h_trend": rows, "note": "apparent barriers from D = MSD/(6t) of the tracked ions after the run; "
                                     "the paper's Table 2 gives the H- values"}


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import torch
    ws, rank, local = dist_setup(True)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2004_09081_gb300 import autotune, fkmc, workloads
    fkmc.load()
    seed = args.seed + rank  # each rank simulates its own independent batch (weak scaling)
    makers = {"batched": workloads.batched_batio3, "sweep": workloads.srtio3_h_sweep,
              "bulk": workloads.bulk_batio3, "um": lambda sd: workloads.um_batio3_bias(sd, args.um_cells),
              "fe": workloads.fe_srtio3, "null": workloads.null_batio3, "htrend": workloads.h_trend,
              "umgrains": workloads.um_grains, "elec": workloads.elec_batio3}
    wl = makers[args.workload](seed)
    nrep = len(wl.replicas)
    default_windows = {"batched": 1024, "sweep": 64, "bulk": 16, "um": 2, "fe": 32, "null": 100, "htrend": 20000,
                       "umgrains": 2, "elec": 32}
    null = args.workload == "null"
    if null or args.workload in ("htrend", "elec"):
        args.no_plain = True  # null: one (integer) arithmetic; htrend: physics runs, mixed only
    W = args.windows if args.windows else default_windows[args.workload]
    stream = torch.cuda.current_stream()
    reps = wl.replicas
    precision = wl.precision

    # K7: fragment edge, window length and launch options, subject to the
    # windowing-accuracy bound (batched workload; single lattices keep their
    # stated partition)
    tuned, deficit = None, None
    if args.workload == "batched" and not args.no_autotune:
        best, res = autotune.autotune([(*r.cells, r.a) for r in reps], [(r.n_vac, r.n_H) for r in reps], seed,
                                      [r.Ea_O for r in reps], [r.Ea_H for r in reps], [r.T for r in reps],
                                      precision=precision)
        wl.edge, wl.n_tau = best["edge"], best["n_tau"]
        tuned_opts = {"schedule": best["schedule"], "cluster_top": best["cluster_top"]}
        tuned = [dict(r["candidate"], deficit=r["deficit"]["vacancies_only"]["deficit"], at_edge=r["at_edge"],
                      accepted=r["accepted"], hops_per_s=r["hops_per_s"]) for r in res]
    else:
        tuned_opts = dict(wl.notes.get("launch_opts", {}))
    if args.workload == "batched":
        table = autotune.deficit_table()
        worst, e_min, est = autotune.batch_deficit(table, [r.cells for r in reps], wl.edge, wl.n_tau)
        deficit = {"at_fragment_edge": e_min, "accepted": autotune.accepted(est, 0.01),
                   "by_composition": {k: {"deficit": v[0], "se": v[1]} for k, v in est.items()},
                   "bound": 0.01, "what": "hop-rate deficit of the windowed scheme against the serial BKL "
                                          "(Sec. II.A) at the shortest fragment edge of the batch; oracle table "
                                          "paper_2004_09081_gb300/window_deficit.json (se from the seed scatter; "
                                          "a row is binding where deficit > 2 se)"}
    edge = wl.edge

    b = make_batch(fkmc, wl, seed, precision, edge=edge, **tuned_opts)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def step():
        s = b.run_null(W, wl.notes["n_frg"]) if null else b.run(W)
        b.moments_all()
        return s

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    clocks = ClockSampler(local)
    barrier(ws)
    torch.cuda.synchronize()
    hops = 0
    kernel_ms = 0.0
    launches = 0
    n_launch = 0
    wall0 = time.perf_counter()
    for k in range(args.steps):
        flush.fill_(k & 0xff)
        ev[k][0].record(stream)
        s = step()
        ev[k][1].record(stream)
        hops += s.hops
        kernel_ms += s.gpu_ms
        launches += s.launches + 1  # + the moment reduction
        n_launch += s.launches
    torch.cuda.synchronize()
    barrier(ws)
    wall = time.perf_counter() - wall0
    clk = clocks.stop()
    step_ms = [a.elapsed_time(c) for a, c in ev]
    t_dev = sum(step_ms) / 1e3
    t_max = allreduce_max(t_dev, ws, dev)
    hops_all = allreduce_sum(float(hops), ws, dev)
    value = hops_all / t_max

    peak, peak_kind = load_peaks()
    all_resident = (not null) and n_launch <= args.steps * 5  # class launches only, no per-phase launches
    kinds = [b.info(r).kernel for r in range(nrep)]
    on_cluster = all_resident and all(k == 2 for k in kinds)
    if null:
        # one unit = one null-event step (rates, propose, apply + clock: three launches)
        units = args.steps * W
        tag, kname = "k_null_step_" + args.workload, "k_null_* (null-event step: rates, propose, apply + clock)"
        note = ("algorithmic bytes per step, 4-byte words: every vacancy's record and 8 neighbour words "
                "(rates), every pick's record, 8 words, proposal and 2 claims (propose), its proposal and "
                "claims plus 2 words and a record per applied hop (apply)")
    elif all_resident:
        # the resident kernels: one launch per class per call (the classes run concurrently),
        # so a "launch" here is one call's concurrent set
        units = args.steps
        if on_cluster:
            tag = "k_cluster_" + args.workload
            kname = "k_cluster (cluster-resident window kernel, %d CTAs per replica)" % b.info(0).ctas
        else:
            tag, kname = "k_resident_" + args.workload, "k_resident (replica-resident window kernel)"
        note = ("lattice state lives in shared memory for the whole launch: DRAM traffic is the stage-in/out "
                "of the state, not per hop; the kernel is bound by instruction issue and dependent latency "
                "(see profiles/)")
    else:
        units = args.steps * W * 8  # one colour phase = one screen and one run launch
        tag = "k_phase_" + ("mixed_" if precision else "plain_") + args.workload
        kname = "k_phase<%s%s> (colour-phase kernel)" % (
            "mixed" if precision else "plain",
            ", site energies" if wl.site else (", electrostatic site energies" if "elec" in wl.notes else ""))
        note = ("a launch here is one colour phase (screen + run pass); neighbour words read from L2/HBM "
                "with ld.global.cg; algorithmic bytes = 160 B per hop at 32-byte sectors" +
                (" + the energy-field words of the site-energy path" if wl.site or "elec" in wl.notes else ""))
    b_alg = B_ALG_PER_HOP_SITE if wl.site else (B_ALG_PER_HOP_ELEC if "elec" in wl.notes else B_ALG_PER_HOP)
    avg_launch_s = kernel_ms / 1e3 / units
    bytes_per_launch = hops / units * b_alg
    if null:
        nv, nfr = wl.replicas[0].n_vac, wl.notes["n_frg"]
        bytes_per_launch = nv * (24 + 8 * 4) + nfr * (24 + 8 * 4 + 16 + 2 * 8) + nfr * (16 + 2 * 8) + \
            hops / units * (2 * 4 + 24)
        b_alg = bytes_per_launch / max(hops / units, 1e-9)
    achieved = bytes_per_launch / avg_launch_s / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": load_traffic(tag), "peak_kind": f"{peak_kind} hbm_gbs",
                "kernel": kname, "bytes_per_hop": b_alg, "hops_per_launch": hops / units,
                "avg_launch_us": avg_launch_s * 1e6, "note": note}
    if roofline["traffic"]:
        # the measured side: ncu's DRAM bytes per launch over the live launch time,
        # and per hop (against the algorithmic bytes_per_hop)
        gbs = roofline["traffic"] / avg_launch_s / 1e9
        roofline["measured_dram"] = {"GBps": gbs, "frac": gbs / peak,
                                     "bytes_per_hop": roofline["traffic"] / max(hops / units, 1e-9)}
    cnt = load_counters(tag) if all_resident else None
    if cnt and cnt.get("smem_wavefronts_per_launch") and clk.get("sm_mhz"):
        # the replica-resident kernel works out of shared memory and is bound by
        # its dependent instruction chains: its warp instructions and shared-memory
        # wavefronts (ncu, per window) over the live launch time, against four warp
        # instructions and one wavefront per SM per cycle at the sampled SM clock;
        # the HBM figures stay beside them
        nsm = torch.cuda.get_device_properties(dev).multi_processor_count
        hz = clk["sm_mhz"] * 1e6
        per_w = W / cnt["counters_windows"]
        wf = cnt["smem_wavefronts_per_launch"] * per_w
        wi = cnt["warp_inst_per_launch"] * per_w
        hbm = {k: roofline[k] for k in ("achieved", "peak", "unit", "frac", "peak_kind", "bytes_per_hop")}
        if "measured_dram" in roofline:
            hbm["measured_dram"] = roofline.pop("measured_dram")
        issue_peak = 4 * nsm * hz / 1e9
        roofline.update({
            "bound": "alu", "achieved": wi / avg_launch_s / 1e9, "peak": issue_peak, "unit": "Gwarp-inst/s",
            "frac": wi / avg_launch_s / 1e9 / issue_peak,
            "peak_kind": "instruction issue: 4 warp instructions per SM per cycle x %d SMs x sampled %.0f MHz" % (
                nsm, clk["sm_mhz"]),
            "warp_inst_per_launch": wi, "hbm": hbm,
            "smem": {"frac": wf / avg_launch_s / (nsm * hz), "wavefronts_per_launch": wf,
                     "peak_wavefronts_per_s": nsm * hz},
            "counters_note": ("warp instructions and shared-memory wavefronts: ncu counts per window "
                              "(profiles/traffic.json) x windows per launch / CUDA-event launch time")})

    extra = {}
    if rank == 0 and args.profile_run:
        extra["note"] = "profile run: timed steps only"
    if rank == 0 and not args.profile_run:
        extra["physics"] = physics_report(fkmc, b, wl)
        # end to end through the public API: host state blob -> GPU, run, moments -> host
        nbytes = fkmc.kmc_state_bytes(b.h)
        if nbytes <= (4 << 30):
            host = torch.empty(nbytes, dtype=torch.uint8).pin_memory()
            fkmc.kmc_download_state(b.h, host.data_ptr(), nbytes)
            e2e_steps = max(3, min(args.steps, 5))
            e2e_hops = 0
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(e2e_steps):
                fkmc.kmc_upload_state(b.h, host.data_ptr(), nbytes)
                e2e_hops += b.run(W).hops
                m = b.moments_all()
            e2e_t = time.perf_counter() - t0
            extra["e2e"] = {"value": e2e_hops / e2e_t, "unit": UNIT, "h2d_bytes_per_step": nbytes,
                            "d2h_bytes_per_step": int(m.nbytes), "steps": e2e_steps}
            del host
        else:
            extra["e2e"] = {"value": None, "unit": UNIT, "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": 0,
                            "note": "state larger than 4 GiB: not re-uploaded every step"}

        if args.workload == "htrend":
            # the same runs stopped after a tenth of the windows: short runs see H- hopping
            # inside H- clusters before O migration sets the long-time D_H
            short_w = max(1, (args.warmup + args.steps) * W // 10)
            bsh = make_batch(fkmc, wl, seed, precision)
            bsh.run(short_w)
            extra["physics_short_run"] = dict(h_trend_report(fkmc, bsh, wl), windows=short_w)
            bsh.close()
            extra["physics"]["windows"] = (args.warmup + args.steps) * W
        if "elec" in wl.notes:
            # the multigrid solve alone: V-cycles per second and bytes moved against HBM
            # (algorithmic: 165 B per fine node per V-cycle -- 4 smoothing sweeps, the
            # residual, restriction and prolongation each touch the level's arrays
            # once -- x 8/7 for the coarser levels)
            rep = wl.replicas[0]
            nodes = rep.cells[0] * rep.cells[1] * rep.cells[2]
            cyc = wl.notes["elec"]["cycles"]
            for _ in range(2):
                b.solve_potential(0)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            nsolve = 10
            e0.record(stream)
            for _ in range(nsolve):
                _, res = b.solve_potential(0)
            e1.record(stream)
            torch.cuda.synchronize()
            t_solve = e0.elapsed_time(e1) / 1e3 / nsolve
            mg_bytes = 165.0 * 8.0 / 7.0 * nodes * cyc
            mg_gbs = mg_bytes / t_solve / 1e9
            extra["multigrid"] = {"nodes": nodes, "cycles": cyc, "warm_cycles": wl.notes["elec"].get("warm_cycles"),
                                  "ms_per_solve": 1e3 * t_solve,
                                  "rel_residual": res, "achieved_GBps": mg_gbs, "peak_GBps": peak,
                                  "frac": mg_gbs / peak,
                                  "note": "a cold solve (deposit + right-hand side + V-cycles + mean + residual "
                                          "check, with its host read-back of the residual); the refreshes inside "
                                          "the step start from the last potential and take warm_cycles V-cycles; "
                                          "all levels (~55 MB) stay in L2, so HBM is a loose bound"}
        if null:
            # cross-check of the spatial windowed scheme against the paper's own
            # formulation: D of V, O and H over the same simulated time
            bn = make_batch(fkmc, wl, seed, fkmc.FKMC_MIXED, tracer=True)
            bn.run_null(20 * W, wl.notes["n_frg"])
            t_null = bn.info(0).null_time_s
            bs = make_batch(fkmc, wl, seed, fkmc.FKMC_MIXED, tracer=True)
            Ws = max(1, int(round(t_null / bs.info(0).tau)))
            ss = bs.run(Ws)
            cmp = {"t_s": t_null, "null_steps": 20 * W, "spatial_windows": Ws,
                   "hops_null": bn.info(0).hops, "hops_spatial": ss.hops,
                   "spatial_hops_per_s": ss.hops / (ss.gpu_ms / 1e3) if ss.gpu_ms > 0 else None}
            for sp, nm in ((fkmc.FKMC_V, "V"), (fkmc.FKMC_O, "O"), (fkmc.FKMC_H, "H")):
                cmp["D_" + nm + "_null"] = bn.D(0, sp)[1]
                cmp["D_" + nm + "_spatial"] = bs.D(0, sp)[1]
            bn.close()
            bs.close()
            extra["null_vs_spatial"] = cmp
        if wl.site:
            # the paper's dopant comparison: D of the vacancies with the full model, without
            # the V-V term, without the dopant term and without interactions, same draws
            trend = {}
            variants = {"vv_and_fe": (wl.site["vv"], wl.site["fe"]), "fe_only": ((), wl.site["fe"]),
                        "vv_only": (wl.site["vv"], ()), "none": ((), ())}
            rates = {}
            for nm, (vv, fe) in variants.items():
                bv = make_batch(fkmc, wl, seed, precision, edge=edge, site=False)
                if vv or fe:
                    bv.set_site_energy(vv, fe)
                bv.run(2)
                sv = bv.run(64 * W)  # long enough for the vacancies to meet the dopants
                rates[nm] = sv.hops / (sv.gpu_ms / 1e3) if sv.gpu_ms > 0 else None
                trend[nm] = [bv.D(r, fkmc.FKMC_V)[1] for r in range(nrep)]
                bv.close()
            extra["site_energy"] = {
                "T": [r.T for r in reps], "D_V": trend, "windows": 64 * W + 2,
                "hops_per_s": rates,
                "note": "D_V (m^2/s) per temperature; the paper reports that the dopant term lowers D_V "
                        "strongly and the V-V term raises it again",
            }
        W_cmp = min(W, 64)  # the comparison legs: rates and D do not need the timed step's length
        if not args.no_plain and not wl.site:
            # accuracy: mixed vs plain FP64 from the same initial state, same draws
            Wacc = 4 * W_cmp
            bm = make_batch(fkmc, wl, seed, fkmc.FKMC_MIXED, edge=edge)
            bp = make_batch(fkmc, wl, seed, fkmc.FKMC_PLAIN, edge=edge)
            hm, hp = bm.run(Wacc).hops, bp.run(Wacc).hops
            mm, mp = bm.moments_all(), bp.moments_all()
            rel, zs = [], []
            for r in range(nrep):
                tr = bp.info(r).window * bp.info(r).tau
                Dm = D_from_moments(mm[r], tr, reps[r].a)
                Dp = D_from_moments(mp[r], tr, reps[r].a)
                if Dp > 0:
                    rel.append(abs(Dm - Dp) / Dp)
                    # sigma_D: the statistical error of D from the replica's vacancies
                    # (squared displacements of the plain run's records)
                    d2 = (bp.records(r)[:, 2:5].astype(np.float64) ** 2).sum(1)
                    h = 0.5 * reps[r].a * 1e-10
                    sd = d2.std(ddof=1) / math.sqrt(len(d2)) * h * h / (6 * tr) if len(d2) > 1 else 0.0
                    if sd > 0:
                        zs.append(abs(Dm - Dp) / sd)
            agg_m = float(mm[:, 4:7].sum()) / max(float(mm[:, 0].sum()), 1.0)
            agg_p = float(mp[:, 4:7].sum()) / max(float(mp[:, 0].sum()), 1.0)
            same = sum(int(np.array_equal(mm[r], mp[r])) for r in range(nrep))
            bm.close()
            bp.close()
            plain = {}
            if nrep > 1:
                # plain FP64, replicas one at a time (the comparison the method is quoted on)
                p_hops, p_ms = 0, 0.0
                t0 = time.perf_counter()
                for r in range(nrep):
                    # a batch of one is keyed as replica 0: its own stream, throughput comparison only
                    b1 = make_batch(fkmc, wl, seed, fkmc.FKMC_PLAIN, replicas=[r], edge=edge)
                    s1 = b1.run(W_cmp)
                    p_hops += s1.hops
                    p_ms += s1.gpu_ms
                    b1.close()
                plain["one_at_a_time"] = {"value": p_hops / (p_ms / 1e3), "unit": UNIT, "hops": p_hops,
                                          "kernel_s": p_ms / 1e3, "wall_s": time.perf_counter() - t0}
                plain["mixed_over_plain_one_at_a_time"] = value / plain["one_at_a_time"]["value"]
            bpb = make_batch(fkmc, wl, seed, fkmc.FKMC_PLAIN, edge=edge)
            bpb.run(2)
            spb = bpb.run(W_cmp)
            bpb.close()
            plain["batched"] = {"value": spb.hops / (spb.gpu_ms / 1e3), "unit": UNIT}
            plain["mixed_over_plain_batched"] = value / plain["batched"]["value"] if spb.hops else None
            extra["plain_fp64"] = plain
            extra["D_mixed_vs_plain"] = {
                "windows": Wacc, "hops_mixed": hm, "hops_plain": hp,
                "aggregate_msd_rel_err": abs(agg_m - agg_p) / agg_p if agg_p else None,
                "per_replica_rel_err_median": float(np.median(rel)) if rel else None,
                "per_replica_rel_err_max": float(np.max(rel)) if rel else None,
                "per_replica_err_over_sigma_D_max": float(np.max(zs)) if zs else None,
                "per_replica_err_over_sigma_D_median": float(np.median(zs)) if zs else None,
                "replicas_beyond_2_sigma_D": int(sum(z > 2.0 for z in zs)),
                "sigma_D_note": "sigma_D = std(|d|^2)/sqrt(N) h^2/(6t) over each replica's vacancies (plain "
                                "run): the two forms draw the same numbers and part only at a rare "
                                "rounding-induced divergence, after which they are independent samples",
                "replicas_bit_identical": same, "replicas": nrep,
            }
        if not args.no_cpu:
            if null:
                rate, ch, cs = cpu_oracle_null_rate(wl, seed, 2, 12.0)
                extra["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
                                         "sample": f"the same lattice, null-event steps of {wl.notes['n_frg']} "
                                                   f"picks, serial C oracle ({ch} hops in {cs:.1f} s)"}
            elif args.workload in ("um", "umgrains"):
                # the oracle holds one byte per site: time it on a 120^3 cube with the same
                # density, field and temperature (and grains), and quote hops/s
                small = workloads.um_batio3_bias(seed, 120)
                if args.workload == "umgrains":
                    small.notes["grains"] = wl.notes["grains"]
                rate, ch, cs, cd = cpu_oracle_rate(small, seed, 2, 12.0)
                smp = f"120^3-cell cube with the same density, field and T ({ch} hops in {cs:.1f} s)"
            else:
                rate, ch, cs, cd = cpu_oracle_rate(wl, seed, min(W, 8) if nrep == 1 else W, 12.0)
                smp = (f"{cd} replica runs of {W} windows" if nrep > 1 else "the same lattice") + \
                    f", serial C oracle ({ch} hops in {cs:.1f} s)"
            if not null:
                extra["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": smp}
            if not null and nrep > 1 and "grains" not in wl.notes and "elec" not in wl.notes:
                # independent replicas: the same oracle on every host core at once
                from oracle import timing
                prate, ph, ps_, pd, pc = timing.parallel_rate(oracle_jobs(wl, seed), W, 12.0)
                extra["cpu_baseline"] = {
                    "value": prate, "unit": UNIT, "cores": pc, "kind": "oracle",
                    "sample": f"{pd} replica runs of {W} windows, one serial C oracle per process on {pc} "
                              f"processes ({ph} hops, longest worker {ps_:.1f} s)",
                    "single_core": {"value": rate, "sample": smp}}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64+f32+f64" if precision else "f64",
            "data": "synthetic",
            "config": {"workload": wl.name, "replicas": nrep, "windows_per_step": W,
                       "precision": ("mixed (fp32 rates -> u64 fixed point, fp32 variate, fp64 clock)"
                                     if precision else "plain fp64"),
                       "n_tau": wl.n_tau, "edge": edge, "launch_opts": tuned_opts, "autotune": tuned,
                       "window_deficit": deficit,
                       "l2": "flushed between timed steps (256 MiB write)",
                       "schedule": ("null-event steps (Sec. II.B), one pick per vacancy, %d steps per "
                                    "benchmark step" % W if null else
                                    ("cluster-resident kernel: one thread-block cluster per replica, a z-slab "
                                     "of fragment layers per CTA" if on_cluster else
                                     "replica-resident kernel per shared-memory size class") if all_resident
                                    else "colour-phase kernel, one launch per phase"),
                       "seed": args.seed},
            "roofline": roofline,
            "clocks": clk,
            "gpu_launches": launches,
            "hops_per_step": hops / args.steps,
            "wall_s": wall,
        }
        line.update(extra)
        print(json.dumps(line))
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
