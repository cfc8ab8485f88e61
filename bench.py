"""Benchmark of the coupled LBM-PSM-DEM step (one JSON line on rank 0).

Workload: particle-laden Couette flow, D3Q19 PSM lattice 256^3, walls at z moving at
-/+0.05, periodic x and y, 4000 spheres of radius 6 (solid fraction ~0.22) at seeded RSA
positions, density ratio 1, distance-based solid fractions, 10 DEM substeps per fluid
step, linear contacts. A step is one coupled fluid step (all DEM substeps, tile binning,
the fused PSM collide-stream and the final corrector). Metric: coupled-step MLUPS (cells
x steps / time), with the PSM kernel's fraction of the measured HBM bandwidth.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--storage f32|f16|bf16]
  python bench.py --impl reference      # the FP64 CPU oracle on the host cores

With N > 1 (torchrun) every rank runs an independent replica of the workload on its own
GPU (the step does not shard; no collective on the data path) and the value is the
aggregate over ranks (weak scaling).
"""
import argparse
import hashlib
import json
import math
import os
import signal
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "coupled-step MLUPS & % HBM roofline, FP32 vs FP16-stored f at stated error"
BYTES_PER_CELL = {"f32": 152, "f16": 76, "bf16": 76}   # 2 x 19 populations per update
STAGES = ["neighbour_rebuild", "dem_substeps", "tile_binning", "psm_collide_stream", "final_corrector"]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--storage", default="f32", choices=["f32", "f16", "bf16"])
    ap.add_argument("--pattern", default="ab", choices=["ab", "aa"],
                    help="population arrays of the main line: two (ab) or one in place (aa)")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--ensemble-only", action="store_true",
                    help="time only the batched 64-simulation ensemble (one JSON line)")
    ap.add_argument("--ellipsoid-only", type=int, default=0, metavar="NX",
                    help="time only the sheared ellipsoid suspension, shrunk to NX x NX x NX/2 at "
                         "its particle density (384: the full workload; one JSON line)")
    ap.add_argument("--long", type=int, default=500,
                    help="steps of each of the three runs whose median the line also reports")
    ap.add_argument("--edge", type=int, default=256,
                    help="lattice edge of the Couette workload (spheres scaled to keep the "
                         "solid fraction); smaller than 256 only for profiler captures")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(x, dist):
    """Largest value of x over all ranks (x itself without a process group). The
    reduction runs on the GPU under NCCL and on the host under gloo."""
    if dist is None:
        return float(x)
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def psm_source_hash():
    h = hashlib.sha256()
    for f in ("lbm.cu", "psm.cuh", "psm_aa.cu", "psm_wide.cu", "internal.cuh"):
        h.update(open(os.path.join(ROOT, "paper_2512_04997_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def traffic_per_cell(storage, pattern="ab"):
    """DRAM bytes per cell update of the PSM kernel from the committed ncu summary, if it
    was taken on the current kernel source; else None (AA pattern: key "<storage>_aa",
    the mean of its two step forms)."""
    path = os.path.join(ROOT, "profiles", "psm_traffic.json")
    if not os.path.exists(path):
        return None
    d = json.load(open(path))
    if d.get("source_hash") != psm_source_hash():
        return None
    v = d.get("bytes_per_cell", {}).get(storage if pattern == "ab" else storage + "_aa")
    return float(v) if v is not None else None


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    def __init__(self, index):
        self.file = tempfile.NamedTemporaryFile(prefix="clocks", suffix=".csv", delete=False)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.file, stderr=subprocess.DEVNULL,
                                         start_new_session=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        os.killpg(self.proc.pid, signal.SIGTERM)
        self.proc.wait()
        self.file.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.file.name):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for k, name in enumerate(names):
                if f[5 + k].lower() == "active":
                    reasons.add(name)
        os.unlink(self.file.name)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(mx)) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def ensemble_measure(args, device, stream):
    """The batched ensemble (64 independent settling/shear simulations, edges U{24..96},
    1-64 spheres, FP16-stored populations) advanced in one batch, timed with CUDA events;
    beside it the same members stepped one after another as separate simulations."""
    import torch
    from paper_2512_04997_gb300 import ledds, workloads as W
    ws = W.batched_ensemble(nsim=64, seed_index=5, storage="f16")
    cells = sum(w.ncell for w in ws)
    b = ledds.batch_from_workloads(ws, device=device)
    b.step(args.warmup)
    choice = b.autotune(steps_per_trial=2)
    cfg = b.config()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    b.step(args.steps)
    e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    bad = {k: 0 for k in ("tile_overflow", "cand_overflow", "nan_detected", "solids_overflow")}
    for m in b.members:
        st = m.status()
        for k in bad:
            bad[k] += st[k]
    b.close()
    del b
    serial_ms = 0.0
    for w in ws:
        s = ledds.from_workload(w, device=device)
        s.step(args.warmup)
        torch.cuda.synchronize()
        e0.record(stream)
        s.step(args.steps)
        e1.record(stream)
        e1.synchronize()
        serial_ms += e0.elapsed_time(e1)
        s.close()
        del s
    torch.cuda.empty_cache()
    return {"workload": "ensemble of 64 settling/shear simulations, edges U{24..96}, 1-64 spheres R 3-8, "
                        "tau U[0.6,1.2], FP16-stored f, one batch",
            "value": cells * args.steps / (ms * 1e-3) / 1e6, "unit": "MLUPS",
            "per_sim_latency_ms_per_step": ms / args.steps,
            "sims": len(ws), "cells": cells, "particles": int(sum(w.n for w in ws)),
            "separate_sims_MLUPS": cells * args.steps / (serial_ms * 1e-3) / 1e6,
            "speedup_vs_separate_sims": serial_ms / ms,
            "launches_per_step": 4,
            "autotune_choice": {"index": choice, "tile": f"32x8x{cfg['tile_depth']}",
                                "psm_ctas_per_sm": cfg["ctas_per_sm"],
                                "order": ["member", "largest_first"][cfg["order"]]},
            # the whole step against the 16-bit algorithmic bytes of every member's cells
            "roofline": {"achieved": cells * 76 / (ms / args.steps * 1e-3) / 1e9, "unit": "GB/s",
                         "frac": cells * 76 / (ms / args.steps * 1e-3) / 1e9 / peaks()[0],
                         "note": "coupled step time (DEM, binning, PSM), not the PSM kernel alone"},
            "status": bad}


def settling_measure(device, stream):
    """The single settling sphere (32x32x64, walls, subdivision fractions) over its 2000
    steps: microseconds per coupled step (65,536 cells: L2-resident, latency-bound)."""
    import torch
    from paper_2512_04997_gb300 import ledds, workloads as W
    w = W.settling_sphere(steps=2000)
    s = ledds.from_workload(w, device=device)
    s.step(200)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    s.step(w.steps)
    e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    st = s.status()
    s.close()
    return {"workload": "settling sphere 32x32x64, R 4, density ratio 2.5, subdivision fractions, n_sub 1",
            "steps": w.steps, "us_per_step": 1e3 * ms / w.steps,
            "value": w.ncell * w.steps / (ms * 1e-3) / 1e6, "unit": "MLUPS", "launches_per_step": st["launches_per_step"]}


def granular_measure(device, stream, steps=10000, sample=100):
    """DEM only: 1e5 spheres (radii U[0.8, 1.2]) settling under gravity in a walled
    120x120x240 box over 10,000 steps, all timed. Contacts per second = sum over steps of
    the contact count / time; the counts come from a replay of the same (deterministic)
    run, read every `sample` steps."""
    import torch
    from paper_2512_04997_gb300 import ledds, workloads as W
    w = W.granular_box(steps=steps)
    s = ledds.from_workload(w, device=device)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    s.step(steps)
    e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    st = s.status()
    s.close()
    r = ledds.from_workload(w, device=device)
    total = 0
    counts = []
    for k in range(steps // sample):
        r.step(sample)
        c = len(r.pairs())
        counts.append(c)
        total += c * sample
    r.close()
    return {"workload": "granular box, 1e5 spheres R U[0.8,1.2], 120x120x240 walled box, linear law, "
                        "mu 0.4, e 0.7, g 2e-6, 10,000 steps from a jittered lattice",
            "steps": steps, "ms_per_step": ms / steps, "value": total / (ms * 1e-3), "unit": "contacts/s",
            "contacts_final": counts[-1] if counts else 0, "contacts_mean": total / steps,
            "status": {k: st[k] for k in ("cand_overflow", "skin_violation", "nan_detected")}}


def ellipsoid_measure(args, device, stream, nx=384, storages=("f32", "bf16")):
    """Prolate ellipsoids (semi-axes 6, 2, 2) in shear, 384x384x192, 2e4 particles at
    random orientations, subdivision solid fractions, common-normal contacts, n_sub 10:
    MLUPS with FP32 and BF16 storage on the same workload, BF16 field error against FP32,
    and the event-timed stage split of each. nx < 384: the box nx x nx x nx/2 at the same
    particle density."""
    import torch
    from paper_2512_04997_gb300 import ledds, workloads as W
    t0 = time.perf_counter()
    if nx == 384:
        w = W.ellipsoid_shear()
    else:
        w = W.ellipsoid_shear(nx=nx, ny=nx, nz=nx // 2, n_particles=int(round(20000 * (nx / 384.0) ** 3)))
    gen_s = time.perf_counter() - t0
    out = {"workload": f"{w.name}: semi-axes (6,2,2), random orientations, shear rate 1e-4, "
                       "subdivision fractions, common-normal contacts, n_sub 10",
           "generate_s": gen_s, "cells": w.ncell, "particles": w.n}
    u_ref = None
    for sto in storages:
        s = ledds.from_workload(w, device=device, storage=sto)
        s.step(args.warmup)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s.step(args.steps)
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        _, u = s.fields()
        s.set_profiling(True)
        s.step(min(args.steps, 10))
        sm_, ps_, _ = s.read_profile()
        st = s.status()
        rec = {"value": w.ncell * args.steps / (ms * 1e-3) / 1e6, "unit": "MLUPS",
               "ms_per_step": ms / args.steps,
               "stages_ms_per_step": {k: v / ps_ for k, v in zip(STAGES, sm_)},
               "status": {k: st[k] for k in ("tile_overflow", "cand_overflow", "skin_violation",
                                             "ell_nonconverged", "nan_detected", "solids_overflow")}}
        if u_ref is None:
            u_ref = u
        else:
            rec["field_error_vs_f32"] = float((u - u_ref).abs().max() / u_ref.abs().max())
        out[sto] = rec
        s.close()
        del s
        torch.cuda.empty_cache()
    if "bf16" in out and "f32" in out:
        out["bf16_speedup_vs_f32"] = out["bf16"]["value"] / out["f32"]["value"]
    return out


def fluidised_sweep(device, stream, phis=(0.0, 0.1, 0.2, 0.3, 0.41), steps=10, warmup=3):
    """The paper's performance workload shape (500x200x800, spheres of diameter 20, n_sub 10,
    distance fractions, FP32 storage) at increasing solid fraction: MLUPS and stage split."""
    import torch
    from paper_2512_04997_gb300 import ledds, workloads as W
    rows = []
    for phi in phis:
        w = W.fluidised_bed(phi)
        s = ledds.from_workload(w, device=device)
        s.step(warmup)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s.step(steps)
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        s.set_profiling(True)
        s.step(3)
        sm_, ps_, _ = s.read_profile()
        st = s.status()
        rows.append({"phi": round(w.n * 4.0 / 3.0 * math.pi * 1000.0 / w.ncell, 3), "spheres": w.n,
                     "value": w.ncell * steps / (ms * 1e-3) / 1e6, "unit": "MLUPS",
                     "psm_ms": sm_[3] / ps_, "dem_ms": (sm_[0] + sm_[1] + sm_[4]) / ps_,
                     "overflow": st["tile_overflow"] + st["cand_overflow"] + st["solids_overflow"]})
        s.close()
        del s
        torch.cuda.empty_cache()
    return {"workload": "fluidised bed 500x200x800 (80 M cells), spheres of diameter 20, density ratio "
                        "1.1, periodic x and z, walls on y, n_sub 10, distance fractions, FP32",
            "steps": steps, "sweep": rows,
            "mlups_ratio_phi0_to_max": rows[0]["value"] / rows[-1]["value"] if rows else None}


def rheology_measure(device, stream, phis=(0.0, 0.1, 0.2, 0.3), steps=60000, every=250, blocks=4):
    """Effective viscosity of the sheared suspension at reduced size (96^3, spheres of
    diameter 10, walls at -/+0.05): the x-y averaged u_x profile sampled every `every` steps
    over the second half of the run, the wall shear rate from the parabola through the wall
    value and the first two nodes, eta/eta0 = wall shear rate / nominal shear rate 2U/H,
    beside the Krieger-Dougherty law (1 - phi/0.64)^(-2.5 * 0.64). The second half is also
    cut into `blocks` equal blocks, each with its own estimate: their spread and the change
    from the first to the last block show whether the estimate is stationary."""
    import torch
    from paper_2512_04997_gb300 import ledds, workloads as W
    rows = []
    t0 = time.perf_counter()
    per_block = steps // 2 // every // blocks
    for phi in phis:
        w = W.rheology_suspension(phi)
        n, U = w.nz, w.u_wall[2, 1, 0]
        s = ledds.from_workload(w, device=device)
        s.step(steps // 2)
        block_prof = []
        for _ in range(blocks):
            prof = torch.zeros(n, dtype=torch.float64, device=device)
            for _ in range(per_block):
                s.step(every)
                _, u = s.fields()
                prof += u[0].view(n, -1).double().mean(1)
            block_prof.append((prof / per_block).cpu().numpy())
        st = s.status()
        s.close()
        prof = np.mean(block_prof, axis=0)
        phi_real = w.n * 4.0 / 3.0 * math.pi * 125.0 / n ** 3
        shear0 = 2.0 * U / n
        eta = W.wall_shear_rate(prof, U) / shear0
        beta = [W.wall_shear_rate(p, U) / shear0 for p in block_prof]
        kd = (1.0 - phi_real / 0.64) ** (-2.5 * 0.64)
        rows.append({"phi": round(phi_real, 3), "spheres": w.n, "eta_rel": eta, "krieger_dougherty": kd,
                     "rel_diff": eta / kd - 1.0, "block_eta": beta,
                     "block_drift": (beta[-1] - beta[0]) / eta,
                     "block_std_rel": float(np.std(beta) / eta),
                     "status": {k: st[k] for k in ("skin_violation", "nan_detected", "cand_overflow")}})
        torch.cuda.empty_cache()
    return {"workload": "sheared suspension 96^3, spheres of diameter 10, walls at -/+0.05 (nominal shear rate "
                        "1.04e-3), tau 0.8, n_sub 10, friction 0.45, restitution 0.95, "
                        f"{steps} steps (strain {steps * 2.0 * 0.05 / 96:.0f}), profiles averaged over the "
                        f"second half in {blocks} blocks",
            "seconds": time.perf_counter() - t0, "points": rows}


SLAB = dict(nx=256, ny=256, nz=32, n_particles=500)


def oracle_sample(steps, keep=False, parallel=True):
    """The oracle (FP64 C, as it stands) on a bounded sample of the workload: a 256x256x32
    slab of the same Couette suspension (same solid fraction, 500 spheres), `steps` steps
    after one untimed step. parallel: its OpenMP build on every host core (the timed CPU
    baseline), else the serial parity build. keep: also the oracle simulation and the
    workload (the serial build, for the error check)."""
    from oracle import oracle as O
    from paper_2512_04997_gb300 import workloads as W
    w = W.couette_suspension(**SLAB)
    par = parallel and not keep
    o = O.from_workload(w, parallel=par)
    o.step(1)   # warm
    t0 = time.perf_counter()
    o.step(steps)
    dt = time.perf_counter() - t0
    mlups = w.ncell * steps / dt / 1e6
    cores = O.threads(par)
    res = {"value": mlups, "unit": "MLUPS", "cores": cores, "kind": "oracle",
           "host_cores": os.cpu_count(),
           "sample": f"{steps} coupled steps of a 256x256x32 slab of the workload "
                     f"({w.ncell} cells, 500 spheres, same solid fraction), FP64, "
                     + (f"OpenMP build of the oracle source, {cores} threads" if par else "single thread"),
           "seconds": dt}
    return (res, o, w) if keep else res


def main_workload(args):
    """The Couette suspension the main line is measured on (edge E, spheres scaled with E^3)."""
    from paper_2512_04997_gb300 import workloads as W
    E = args.edge
    w = W.couette_suspension(nx=E, ny=E, nz=E, n_particles=int(round(4000 * (E / 256) ** 3)),
                             storage=args.storage)
    w.params["pattern"] = args.pattern
    return w


def main_config(w, storage, world):
    N = w.ncell
    return {"workload": w.name, "cells": N, "particles": w.n, "storage": storage,
            "pattern": w.params.get("pattern", "ab"),
            "n_sub": w.params["n_sub"], "tau": w.params["tau"], "voxel": w.params["voxel"],
            "l2": f"inputs larger than L2 (populations 2 x 19 x {N / 1e6:.1f}M values)",
            "parallelism": f"replicas x{world}"}


def run_reference(args):
    rank, world, _ = dist_env()
    if world > 1 and rank != 0:
        return
    steps = max(1, min(args.steps, 8))
    warm = max(0, min(args.warmup, 1))
    if warm:
        oracle_sample(1)
    res = oracle_sample(steps)
    config = main_config(main_workload(args), args.storage, args.gpus)
    # the timed sample is a slab of the workload: its own cell count
    config["cells"] = SLAB["nx"] * SLAB["ny"] * SLAB["nz"]
    config["particles"] = SLAB["n_particles"]
    config.pop("l2", None)
    config["timed_sample"] = (f"{SLAB['nx']}x{SLAB['ny']}x{SLAB['nz']} slab of the "
                              f"{config['workload']} workload, same solid fraction")
    line = {"metric": METRIC, "value": res["value"], "unit": "MLUPS", "n_gpus": args.gpus,
            "steps": steps, "warmup": warm, "ms_per_step": 1e3 * res["seconds"] / steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": config,
            "cpu_baseline": {"kind": "oracle", "cores": res["cores"], "sample": res["sample"],
                             "value": res["value"], "unit": "MLUPS"},
            "e2e": {"value": res["value"], "unit": "MLUPS", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import torch
    from paper_2512_04997_gb300 import ledds, workloads as W

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as td
        td.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
        dist = td
    hbm, peak_kind = peaks()
    if args.ensemble_only:
        ens = ensemble_measure(args, f"cuda:{local}", torch.cuda.current_stream())
        if rank == 0:
            print(json.dumps({"ensemble": ens, "steps": args.steps, "warmup": args.warmup}), flush=True)
        return
    if args.ellipsoid_only:
        ell = ellipsoid_measure(args, f"cuda:{local}", torch.cuda.current_stream(), nx=args.ellipsoid_only,
                                storages=(args.storage,))
        if rank == 0:
            print(json.dumps({"ellipsoid_shear": ell, "steps": args.steps, "warmup": args.warmup}), flush=True)
        return
    w = main_workload(args)
    N = w.ncell
    sim = ledds.from_workload(w, device=f"cuda:{local}")
    stream = torch.cuda.current_stream()

    def barrier():
        if dist:
            dist.barrier()
        torch.cuda.synchronize()

    # warm-up (graph capture happens here)
    sim.step(args.warmup)
    barrier()
    clocks = Clocks(local)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    e0.record(stream)
    sim.step(args.steps)
    e1.record(stream)
    e1.synchronize()
    barrier()
    clk = clocks.stop()
    ms = max_over_ranks(e0.elapsed_time(e1), dist)
    value = N * args.steps * world / (ms * 1e-3) / 1e6
    st = sim.status()
    # the protocol's longer form: three runs of LONG steps each, their median
    long_runs = []
    for _ in range(3 if args.long > 0 else 0):
        barrier()
        e0.record(stream)
        sim.step(args.long)
        e1.record(stream)
        e1.synchronize()
        barrier()
        long_runs.append(max_over_ranks(e0.elapsed_time(e1), dist))
    median3 = None
    if long_runs:
        lm = float(np.median(long_runs))
        median3 = {"steps_per_run": args.long, "runs_ms": long_runs,
                   "value": N * args.long * world / (lm * 1e-3) / 1e6, "unit": "MLUPS",
                   "ms_per_step": lm / args.long}

    # profiled pass: CUDA events around every stage of each step (eager launches)
    sim.set_profiling(True)
    sim.step(args.steps)
    stage_ms, psteps, plaunch = sim.read_profile()
    sim.set_profiling(False)
    psm_ms = stage_ms[3] / psteps
    bpc = BYTES_PER_CELL[args.storage]
    achieved = N * bpc / (psm_ms * 1e-3) / 1e9
    tpc = traffic_per_cell(args.storage, args.pattern)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                "frac": achieved / hbm, "traffic": (tpc * N if tpc is not None else None),
                "kernel": "k_psm (fused PSM collide-stream, solid fractions, force reduction)",
                "algorithmic_bytes_per_launch": N * bpc, "peak_kind": peak_kind,
                "avg_launch_ms": psm_ms}

    # end to end through the C-ABI: particle kinematics in from pinned host memory, one
    # step, kinematics out to pinned host memory, every step
    n = w.n
    h_in = torch.empty(18 * n, dtype=torch.float64, pin_memory=True)
    h_out = torch.empty(18 * n, dtype=torch.float64, pin_memory=True)
    sim.step(1)
    ledds.check("ledds_read_particles", ledds.lib().ledds_read_particles(sim.h, h_in.data_ptr(), 0))
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        ledds.check("ledds_write_kinematics", ledds.lib().ledds_write_kinematics(sim.h, h_in.data_ptr(), 0))
        sim.step(1)
        ledds.check("ledds_read_particles", ledds.lib().ledds_read_particles(sim.h, h_out.data_ptr(), 0))
    barrier()
    e2e_s = max_over_ranks(time.perf_counter() - t0, dist)
    e2e = {"value": N * args.steps * world / e2e_s / 1e6, "unit": "MLUPS",
           "h2d_bytes_per_step": 18 * 8 * n, "d2h_bytes_per_step": 18 * 8 * n,
           "api": "ledds_write_kinematics(host) + ledds_step(1) + ledds_read_particles(host)"}

    variants = {}
    if not args.no_variants and args.storage == "f32":
        # reduced-precision storage: same workload and steps; field error against FP32
        ref = ledds.from_workload(w, device=f"cuda:{local}")
        ref.step(args.warmup + args.steps)
        _, u_ref = ref.fields()
        del ref
        # AA: one population array stepped in place (half the population memory)
        for key, sto, pat in (("f16", "f16", "ab"), ("bf16", "bf16", "ab"), ("aa_f32", "f32", "aa"),
                              ("aa_f16", "f16", "aa")):
            v = ledds.from_workload(w, device=f"cuda:{local}", storage=sto, pattern=pat)
            v.step(args.warmup)
            torch.cuda.synchronize()
            a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a0.record(stream)
            v.step(args.steps)
            a1.record(stream)
            a1.synchronize()
            vms = a0.elapsed_time(a1)
            _, u_v = v.fields()
            err = float((u_v - u_ref).abs().max() / u_ref.abs().max())
            v.set_profiling(True)
            v.step(args.steps)
            sm_, ps_, _ = v.read_profile()
            pms = sm_[3] / ps_
            ach = N * BYTES_PER_CELL[sto] / (pms * 1e-3) / 1e9
            variants[key] = {"value": N * args.steps / (vms * 1e-3) / 1e6, "unit": "MLUPS",
                             "storage": sto, "pattern": pat,
                             "speedup_vs_f32": (N * args.steps / (vms * 1e-3) / 1e6) / value * world,
                             "field_error_vs_f32": err, "psm_ms": pms,
                             "workspace_gb": v.workspace.numel() / 1e9,
                             "roofline": {"achieved": ach, "frac": ach / hbm, "unit": "GB/s"}}
            del v
            torch.cuda.empty_cache()

    if not args.no_variants:
        variants["ensemble"] = ensemble_measure(args, f"cuda:{local}", stream)
        variants["settling_sphere"] = settling_measure(f"cuda:{local}", stream)
        variants["granular_dem"] = granular_measure(f"cuda:{local}", stream)
        variants["ellipsoid_shear"] = ellipsoid_measure(args, f"cuda:{local}", stream)
        variants["fluidised_bed"] = fluidised_sweep(f"cuda:{local}", stream)
        variants["rheology"] = rheology_measure(f"cuda:{local}", stream)

    cpu = None
    oracle_err = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = oracle_sample(4)
        cpu.pop("seconds", None)
        _, o, ws = oracle_sample(2, keep=True)
        # the CUDA path on the same slab and steps: its error against the oracle
        gs = ledds.from_workload(ws, device=f"cuda:{local}")
        gs.step(3)
        _, ug = gs.fields()
        _, uo = o.moments()
        pg = gs.particles()[0]
        po = o.particles()[0]
        ugn = ug.cpu().numpy()
        oracle_err = {"sample": "the oracle's slab, 3 coupled steps",
                      "velocity_normwise": float(np.abs(ugn - uo).max() / np.abs(uo).max()),
                      "positions_max_abs": float(np.abs(pg - po).max()),
                      "tolerance": {"velocity_normwise": 1e-5, "positions_max_abs": 1e-6}}
        del gs

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic",
                "config": main_config(w, args.storage, world),
                "median_of_3": median3,
                "roofline": roofline, "cpu_baseline": cpu, "error_vs_oracle": oracle_err, "e2e": e2e,
                "gpu_launches": st["launches_per_step"] * args.steps,
                "clocks": clk, "stages_ms_per_step": {k: v / psteps for k, v in zip(STAGES, stage_ms)},
                "status": {k: st[k] for k in ("tile_overflow", "cand_overflow", "skin_violation",
                                              "nan_detected", "solids_overflow")},
                "variants": variants}
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
