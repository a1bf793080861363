#!/usr/bin/env python3
"""Benchmark: full permeability tensor of a 256^3 consolidated sphere pack.

Workload (one "step"): the whole hot path on one synthetic geometry -- mask upload
and neighbourhood evaluation, percolation check, the three drive directions batched in
every sweep launch, FP32 pseudo-time sweeps with FP64 reductions, then the FP64 defect
correction (FP64 residual, FP32 correction sweeps, FP64 update) until the window
criterion holds, Darcy evaluation of the nine k_ij and symmetrisation.  Geometry: 256^3
periodic random sequential addition pack of spheres with lognormal radii (median 10
voxels, sigma 0.3), dilated to porosity 0.38 (seed 2).

Metric: fluid-voxel updates per second = pore voxels x pseudo-time iterations x
drives / time, whole job (all ranks).  Also reported: seconds to the full k tensor in
this form and in the plain form (three unbatched FP32 solves with FP64 reductions, no
graphs, no correction), the error of every k_ij of both against the FP64 oracle's
converged tensor, the sweep kernel's achieved HBM bandwidth against the measured peak,
the CPU oracle on the host cores, and the end-to-end rate through the C ABI with host
buffers.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Multi-GPU: one process per GPU under torch.distributed.run; every rank solves its own
replica (independent problems, no collective on the data path), value = sum over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

WORKLOAD = "kxyz_256c_rsa_lognormal_phi038"
SHAPE = (256, 256, 256)
SEED = 2
# window criterion (relative change of the mean velocity over one window, Sec. 7.1 form):
# the off-diagonal k_ij are ~1e-3 of the diagonal, so 1e-5 on each of them needs the
# change held well below 1e-8 of the driven component
TOL = 1e-8
PRECISION = "dc64"
PLAIN_TOL = 1e-6  # the paper's criterion for the plain FP32 form
METRIC = "fluid-voxel updates/s"
UNIT = "voxel-updates/s"


def make_mask():
    from paper_2407_19868_gb300 import geometry as G
    m, info = G.rsa_sphere_pack(SHAPE, 10.0, 0.3, 4.0, 25.0, 0.38, seed=SEED)
    return m, info


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clock / throttle samples while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.samples = []
        self._stop = threading.Event()
        self._t = None

    def _run(self):
        while not self._stop.is_set():
            try:
                out = subprocess.run(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}",
                                      "--format=csv,noheader,nounits"], capture_output=True, text=True,
                                     timeout=5).stdout.strip()
                if out:
                    self.samples.append([v.strip() for v in out.split(",")])
            except Exception:
                pass
            self._stop.wait(0.2)

    def __enter__(self):
        self._t = threading.Thread(target=self._run, daemon=True)
        self._t.start()
        return self

    def __exit__(self, *a):
        self._stop.set()
        if self._t:
            self._t.join(timeout=6)

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        mx = [float(s[2]) for s in self.samples if s[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for s in self.samples:
            for k, v in zip(names, s[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(k)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.samples)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def cpu_oracle_rate(mask, n_iter: int):
    """The oracle as it stands, one drive, n_iter iterations of the same workload."""
    import oracle
    dom = oracle.Domain(mask)
    U, p = dom.zeros()
    t = time.perf_counter()
    dom.iterate(U, p, n_iter, drive_dir=0)
    dt = time.perf_counter() - t
    n_fluid = int(np.count_nonzero(mask == 0))
    return n_fluid * n_iter / dt, oracle.num_threads(), dt


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    mask, _ = make_mask()
    import oracle
    oracle.build()
    n_fluid = int(np.count_nonzero(mask == 0))
    n_iter = args.ref_iters
    dom = oracle.Domain(mask)
    rates = []
    total_t = 0.0
    for step in range(args.warmup + args.steps):
        U, p = dom.zeros()
        t = time.perf_counter()
        dom.iterate(U, p, n_iter, drive_dir=step % 3)
        dt = time.perf_counter() - t
        if step >= args.warmup:
            rates.append(n_fluid * n_iter / dt)
            total_t += dt
    value = n_fluid * n_iter * args.steps / total_t
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * total_t / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": WORKLOAD, "shape": list(SHAPE), "porosity": 0.38, "seed": SEED,
                       "step": f"{n_iter} oracle iterations of one drive (bounded sample)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                             "sample": f"{n_iter} FP64 oracle iterations per step on the 256^3 mask"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def aggregate_ranks(seconds: float, updates: float, device="cpu"):
    """Whole-job figures over replicas: the slowest rank's time and the sum of the voxel
    updates of all ranks (no collective on the data path; only this one at the end)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return seconds, updates
    t = torch.tensor([seconds], dtype=torch.float64, device=device)
    u = torch.tensor([updates], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def reference_k():
    """The FP64 oracle's converged raw tensor of the benchmark mask (written by
    tests/golden/make_reference.py, which calls only the oracle), or None if the stored
    mask hash differs."""
    from paper_2407_19868_gb300 import geometry as G
    try:
        with open(os.path.join(ROOT, "tests", "golden", "reference_k.json")) as f:
            ref = json.load(f)["config2"]
    except Exception:
        return None, None
    kref = np.zeros((3, 3))
    for j in range(3):
        kref[:, j] = ref["columns"][str(j)]["k_col"]
    return kref, ref


def k_errors(k_raw, kref):
    """|k_ij - k_ij(oracle)| / |k_ij(oracle)| for every component (raw, unsymmetrised)."""
    k = np.asarray(k_raw, dtype=np.float64)
    return np.abs(k - kref) / np.abs(kref)


def run_ours(args):
    import torch

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    from paper_2407_19868_gb300 import api, geometry as G

    api.load()
    mask, info = make_mask()
    n_fluid = int(np.count_nonzero(mask == 0))
    N = mask.size
    dmask = torch.from_numpy(mask).cuda()
    opts = dict(tol=args.tol, precision=args.precision, check_every=args.check_every, autotune=args.autotune,
                schedule=args.schedule, tile=args.tile, dc_switch_tol=args.dc_switch_tol,
                dc_extrapolate=args.dc_extrapolate)

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    # warm-up (untimed; the first solve of the shape also tunes the sweep schedule)
    for _ in range(args.warmup):
        r = api.permeability_tensor(dmask, **opts)
    barrier()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    results = []
    with ClockSampler(local) as clk:
        barrier()
        e0.record(stream)
        for _ in range(args.steps):
            results.append(api.permeability_tensor(dmask, **opts))
        e1.record(stream)
        barrier()
    dev_ms = e0.elapsed_time(e1)
    iters = [r["stats"][0]["iters"] for r in results]
    updates = sum(n_fluid * it * 3 for it in iters)
    t_max, updates = aggregate_ranks(dev_ms / 1e3, float(updates), device="cuda")
    value = updates / t_max

    # end to end through the C ABI with host buffers (mask in host memory, k back to host)
    e2e_value = None
    if args.e2e_steps > 0:
        barrier()
        t = time.perf_counter()
        e2e_upd = 0
        for _ in range(args.e2e_steps):
            r = api.permeability_tensor(mask, **opts)
            e2e_upd += n_fluid * r["stats"][0]["iters"] * 3
        torch.cuda.synchronize()
        e2e_t = time.perf_counter() - t
        e2e_value = e2e_upd * ws / e2e_t

    # accuracy of every k_ij against the oracle, and the plain form for comparison: three
    # unbatched single-drive FP32 solves with FP64 reductions, no graphs, no correction
    kref, ref = reference_k()
    accuracy = None
    plain = None
    if rank == 0 and args.plain:
        torch.cuda.synchronize()
        t = time.perf_counter()
        cols = [api.solve_direction(dmask, j, fields=False, tol=PLAIN_TOL, precision="fp32", use_graph=0,
                                    check_every=args.check_every) for j in range(3)]
        torch.cuda.synchronize()
        plain_s = time.perf_counter() - t
        k_plain = np.stack([c["k_col"] for c in cols], axis=1)
        plain = {"form": "three unbatched FP32 solves, FP64 reductions, no graphs, no correction",
                 "tol": PLAIN_TOL, "seconds_to_k_tensor": plain_s,
                 "iters": [c["stats"]["iters"] for c in cols]}
        if kref is not None and ref["sha256"] == G.mask_sha256(mask):
            ep = k_errors(k_plain, kref)
            plain["k_err_per_component"] = ep.tolist()
            plain["k_err_max"] = float(ep.max())
    # the adjoint form: the forward solve of drive x and the transposed solve along x, then
    # dk_xx/d alpha for every voxel (FP32 fields on the tiled kernels, the plain criterion);
    # the second of two runs, so that the tuning of the shapes is excluded
    adjoint = None
    if rank == 0 and args.adjoint:
        w = np.zeros((3, 3))
        w[0, 0] = 1.0
        for _ in range(2):
            torch.cuda.synchronize()
            t = time.perf_counter()
            ra = api.sensitivity(dmask, w, precision="fp32", tol=PLAIN_TOL, check_every=args.check_every)
            torch.cuda.synchronize()
            adj_s = time.perf_counter() - t
        adjoint = {"form": "forward drive x + transposed solve along x, dk_xx/d alpha per voxel (FP32, tiled)",
                   "tol": PLAIN_TOL, "seconds": adj_s, "k_xx": float(ra["k_raw"][0, 0]),
                   "vs_plain_tensor": adj_s / plain["seconds_to_k_tensor"] if plain else None}
    # the same form with another artificial speed of sound: the fixed point (k) does not
    # depend on c^2, only the number of iterations does (the paper's 1.5e6 is the headline)
    c2_form = None
    if rank == 0 and args.c2_alt > 0:
        o2 = dict(opts, c2=args.c2_alt)
        for _ in range(2):
            torch.cuda.synchronize()
            t = time.perf_counter()
            rc2 = api.permeability_tensor(dmask, **o2)
            torch.cuda.synchronize()
            c2_s = time.perf_counter() - t
        c2_form = {"c2": args.c2_alt, "seconds_to_k_tensor": c2_s, "iters": rc2["stats"][0]["iters"]}
        if kref is not None and ref["sha256"] == G.mask_sha256(mask):
            c2_form["k_err_max"] = float(k_errors(rc2["k_raw"], kref).max())
    if kref is not None and ref["sha256"] == G.mask_sha256(mask):
        err = k_errors(results[-1]["k_raw"], kref)
        accuracy = {"reference": "FP64 CPU oracle, window criterion %g (tests/golden/reference_k.json)" % ref["tol"],
                    "k_err_per_component": err.tolist(), "k_err_max": float(err.max()),
                    "meets_1e-5_each": bool(err.max() <= 1e-5)}

    # roofline of the dominant kernel: the fused sweep over the 3 drives; the plain FP32
    # phase moves 32 B per cell and drive, the correction sweeps also read their FP32
    # source (48 B); both come from CUDA events around the window graphs of the timed
    # steps, and the one with the larger share of the step time is reported first
    st0 = [r["stats"][0] for r in results]
    plain_sweeps = sum(s["sweeps_timed"] for s in st0)
    src_sweeps = sum(s["sweeps_timed_src"] for s in st0)
    sweep_ms = sum(s["sweep_ms"] * s["sweeps_timed"] for s in st0) / max(plain_sweeps, 1)
    sweep_ms_src = sum(s["sweep_ms_src"] * s["sweeps_timed_src"] for s in st0) / max(src_sweeps, 1)
    peak, peak_kind = measured_peaks()
    kernels = [{"kernel": "fused pseudo-time sweep, 3 drives per launch (FP32 phase)", "sweep_ms": sweep_ms,
                "alg_bytes_per_launch": 3 * 32 * N + N / 8, "launches_timed": plain_sweeps,
                "time_share": plain_sweeps * sweep_ms / dev_ms},
               {"kernel": "fused pseudo-time sweep with the correction source, 3 drives per launch",
                "sweep_ms": sweep_ms_src, "alg_bytes_per_launch": 3 * 48 * N + N / 8, "launches_timed": src_sweeps,
                "time_share": src_sweeps * sweep_ms_src / dev_ms}]
    kernels = [k for k in kernels if k["launches_timed"] > 0]
    kernels.sort(key=lambda k: -k["time_share"])
    for k in kernels:
        k["achieved"] = k["alg_bytes_per_launch"] / (k["sweep_ms"] * 1e-3) / 1e9
        k["frac"] = k["achieved"] / peak
        k["traffic"] = stored_traffic(k["alg_bytes_per_launch"])
    top = kernels[0]
    kernel_launches = sum(r["stats"][0]["kernel_launches"] for r in results)

    cpu = None
    if rank == 0 and ws == 1 and args.cpu_iters > 0:
        rate, cores, secs = cpu_oracle_rate(mask, args.cpu_iters)
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{args.cpu_iters} FP64 oracle iterations of drive x on the same 256^3 mask "
                         f"({secs:.1f} s)"}
    k = results[-1]["k"]
    last = results[-1]["stats"][0]
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": dev_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32" if args.precision != "fp64" else "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "shape": list(SHAPE), "porosity": round(1 - mask.mean(), 6),
                   "seed": SEED, "drives": 3, "precision": {"fp32": "fp32", "dc64": "fp32_dc64",
                                                            "fp64": "fp64"}[args.precision],
                   "tol": args.tol, "check_every": args.check_every, "iters_per_step": iters,
                   "dc_rounds": last["dc_rounds"], "schedule": last["schedule"], "tile": last["tile"],
                   "dc_switch_tol": args.dc_switch_tol, "dc_extrapolate": args.dc_extrapolate,
                   "seconds_to_k_tensor": dev_ms / 1e3 / args.steps,
                   "setup_seconds_per_step": statistics.mean(s["setup_seconds"] for s in st0),
                   "l2": "working set 1.6 GB of fields per sweep > 129 MB L2 (no flush needed)",
                   "parallelism": f"replicas x{ws}"},
        "k_tensor": [[float(v) for v in row] for row in k],
        "accuracy": accuracy,
        "plain_form": plain,
        "adjoint_form": adjoint,
        "other_c2_form": c2_form,
        "roofline": {"bound": "hbm", "achieved": top["achieved"], "peak": peak, "unit": "GB/s",
                     "frac": top["frac"], "traffic": stored_traffic(top["alg_bytes_per_launch"]),
                     "peak_kind": peak_kind, "kernel": top["kernel"], "sweep_ms": top["sweep_ms"],
                     "alg_bytes_per_launch": top["alg_bytes_per_launch"], "launches_timed": top["launches_timed"],
                     "time_share": top["time_share"], "other_kernels": kernels[1:]},
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(N), "d2h_bytes_per_step": 9 * 8 * 2},
        "gpu_launches": kernel_launches,
        "clocks": clk.summary(),
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def run_profile_case(args):
    """A short run in the benchmark's launch configuration for ncu captures: the same
    mask, three drives batched per sweep launch, FP32 fields, stopped after
    ``--profile-iters`` iterations (windows of 2 sweeps); with --profile-precision dc64
    one correction round of as many sweeps follows (the source-carrying sweeps)."""
    import torch
    from paper_2407_19868_gb300 import api
    api.load()
    mask, _ = make_mask()
    r = api.permeability_tensor(torch.from_numpy(mask).cuda(), tol=1e-12, check_every=2,
                                max_iter=args.profile_iters, precision=args.profile_precision,
                                autotune=args.autotune, schedule=args.schedule, tile=args.tile, dc_max_rounds=1)
    torch.cuda.synchronize()
    print(json.dumps({"profile_case": "pm_permeability_tensor", "iters": r["stats"][0]["iters"],
                      "schedule": r["stats"][0]["schedule"], "status": r["status"]}))
    return 0


def run_large(args):
    """Large-domain measurement: n^3 periodic Boolean model of spheres (radius 20 +- 5
    voxels, porosity 0.35, seed 5) generated on the GPU, one drive (x), FP32 fields with
    FP64 reductions, window criterion 1e-6; reports the sweep rate and the time to k_xx."""
    import torch
    from paper_2407_19868_gb300 import api, geometry as G
    api.load()
    n = args.large
    t = time.perf_counter()
    mask, info = G.boolean_spheres_gpu(n, 15.0, 25.0, 0.35, seed=5)
    torch.cuda.synchronize()
    gen_s = time.perf_counter() - t
    N = n ** 3
    n_fluid = int(round(info["porosity"] * N))
    t = time.perf_counter()
    r = api.solve_direction(mask, 0, fields=False, tol=1e-6, check_every=args.check_every,
                            max_iter=args.large_max_iter, check_percolation=0, precision="fp32",
                            field_memory=args.field_memory)
    torch.cuda.synchronize()
    solve_s = time.perf_counter() - t
    st = r["stats"]
    sweep_s = st["sweep_ms"] * 1e-3
    alg = 32 * N + N / 8
    peak, kind = measured_peaks()
    line = {"workload": f"boolean_spheres_{n}c_r20pm5_phi035", "n": n, "cells": N, "porosity": info["porosity"],
            "field_memory": ["device", "host (one buffer)", "host (both buffers)"][args.field_memory],
            "spheres": info["spheres"], "generate_s": gen_s, "status": r["status"], "iters": st["iters"],
            "k_xx_vx2": float(r["k_col"][0]), "k_col": [float(v) for v in r["k_col"]], "delta": st["delta"],
            "err_est": st["err_est"], "seconds_to_k": solve_s, "sweep_ms": st["sweep_ms"],
            "glups": N / sweep_s / 1e9, "fluid_voxel_updates_per_s": n_fluid / sweep_s,
            "hbm_gbs": alg / sweep_s / 1e9, "hbm_frac": alg / sweep_s / 1e9 / peak, "peak_kind": kind,
            "tile": st["tile"], "schedule": st["schedule"], "schedule_split": st["schedule_split"]}
    print(json.dumps(line), flush=True)
    return 0


def run_ellipsoid(args):
    """Anisotropy benchmark of Sec. 6: a 100^3 periodic box with one solid ellipsoid
    (semi-axes 35, 10, 35 voxels along e1, e2, e3) rotated about e1 in 5 degree steps from 0
    to 90 degrees; full k tensor per angle (three drives batched, FP32 fields with FP64
    reductions, the paper's criterion tol 1e-6 of Sec. 7.1), principal permeabilities of the
    (e2, e3) block and the inclination of the major principal axis against e3.  dx = 10 um
    as in the paper."""
    import torch
    from paper_2407_19868_gb300 import api, geometry as G
    api.load()
    dx = 1e-5
    rows = []
    t_all = time.perf_counter()
    for alpha in range(0, 91, 5):
        m = torch.from_numpy(G.rotated_ellipsoid(100, (35.0, 10.0, 35.0), float(alpha))).cuda()
        t = time.perf_counter()
        r = api.permeability_tensor(m, dx=dx, precision="fp32", tol=1e-6)
        torch.cuda.synchronize()
        secs = time.perf_counter() - t
        k = np.asarray(r["k"])
        k2 = np.zeros((3, 3))
        k2[1:, 1:] = k[1:, 1:]
        lam, R = api.principal_axes(k2)
        j = int(np.argmax(lam))
        phi = float(np.degrees(np.arctan2(abs(R[1, j]), abs(R[2, j]))))
        rows.append({"alpha_deg": alpha, "k22_m2": k[1, 1], "k33_m2": k[2, 2], "k23_m2": k[1, 2],
                     "k_II_m2": float(lam[1]), "k_III_m2": float(lam[2]), "ratio_III_II": float(lam[2] / lam[1]),
                     "phi_deg": phi, "k11_m2": k[0, 0], "status": r["status"], "seconds": secs,
                     "iters": r["stats"][0]["iters"]})
        print(json.dumps(rows[-1]), flush=True)
    ratios = [row["ratio_III_II"] for row in rows]
    dev = [abs(row["phi_deg"] - row["alpha_deg"]) for row in rows if 0 < row["alpha_deg"] <= 45]
    print(json.dumps({"workload": "ellipsoid_100c_35x10x35_rotated_e1", "angles": len(rows),
                      "ratio_III_II_mean": float(np.mean(ratios)), "ratio_III_II_range": [min(ratios), max(ratios)],
                      "max_abs_phi_minus_alpha_deg_5_to_45": max(dev), "seconds_all": time.perf_counter() - t_all}),
          flush=True)
    return 0


def run_thin(args):
    """Regular thin porous media of Sec. 6 (Table sfb_domain_comparison): one cylinder per
    1 mm x 1 mm periodic cell, dx = 4 um (250 x 250 voxels), radii 0.35 .. 0.49 mm; k_11
    for a uniform (2-D) cell 4 voxels thick, and for the 27-voxel-thick cell with a 2-voxel
    solid frame at both ends of e2; FP32 fields, the paper's criterion 1e-6."""
    import torch
    from paper_2407_19868_gb300 import api, geometry as G
    api.load()
    dx = 4e-6
    paper = {0.35: 26.1, 0.40: 17.5, 0.45: 8.08, 0.47: 3.83, 0.49: 0.39}  # 1e-10 m^2
    for rad_mm, kp in paper.items():
        row = {"radius_mm": rad_mm, "paper_k11_1e-10m2": kp}
        for name, ny, frame in (("2d", 4, 0), ("frame27", 27, 2)):
            m = G.cylinder_cell(250, rad_mm * 1e-3 / dx, ny, frame)
            t = time.perf_counter()
            r = api.solve_direction(torch.from_numpy(m).cuda(), 0, dx=dx, fields=False, tol=1e-6,
                                    precision="fp32")
            torch.cuda.synchronize()
            row[name] = {"k11_1e-10m2": float(r["k_col"][0]) * 1e10, "porosity": float(1 - m.mean()),
                         "iters": r["stats"]["iters"], "status": r["status"], "seconds": time.perf_counter() - t}
        print(json.dumps(row), flush=True)
    return 0


def run_packs(args):
    """Regular sphere packings of Sec. 6: SC, BCC and FCC unit cells of 100 voxels at
    porosities 0.2 .. 0.9; full k tensor (FP32 fields, the paper's criterion 1e-6),
    k_11 against the Kozeny-Carman estimate D^2 phi^3 / (180 (1 - phi)^2) (D = sphere
    diameter) and the cubic isotropy of the computed tensor."""
    import torch
    from paper_2407_19868_gb300 import api, geometry as G
    api.load()
    for kind in ("sc", "bcc", "fcc"):
        for phi in (0.2, 0.3, 0.4, 0.5, 0.6, 0.7, 0.8, 0.9):
            m, r = G.regular_pack(100, kind, phi)
            t = time.perf_counter()
            res = api.permeability_tensor(torch.from_numpy(m).cuda(), precision="fp32", tol=1e-6)
            torch.cuda.synchronize()
            k = np.asarray(res["k"])
            ph = float(1 - m.mean())
            kc = (2 * r) ** 2 / 180.0 * ph ** 3 / (1 - ph) ** 2
            kd = float(np.mean(np.diag(k)))
            print(json.dumps({"lattice": kind, "porosity": ph, "radius_vox": r, "k11_vx2": float(k[0, 0]),
                              "k_over_kc": float(k[0, 0]) / kc,
                              "isotropy_max_rel": float(np.max(np.abs(np.diag(k) - kd)) / kd),
                              "offdiag_max_rel": float(np.max(np.abs(k - np.diag(np.diag(k)))) / kd),
                              "status": res["status"], "iters": res["stats"][0]["iters"],
                              "seconds": time.perf_counter() - t}), flush=True)
    return 0


def run_compare(args):
    """The forms of the solver against the plain GPU path on the benchmark geometry (256^3
    pack), each timed to a full k tensor (second of two runs, so tuning is excluded) and its
    error per k_ij against the FP64 oracle reference (tests/golden/reference_k.json, written
    by the oracle): plain = three unbatched single-drive solves, FP32 fields + FP64
    reductions, no graph, tol 1e-6; batched = the three drives in each launch with window
    graphs; dc64 = batched with FP64 defect correction to 1e-8; fp64 = FP64 fields to 1e-8;
    adjoint = forward + transposed solves and dk_xx/d alpha for J = k_xx."""
    import torch
    from paper_2407_19868_gb300 import api, geometry as G
    api.load()
    mask, _ = make_mask()
    with open(os.path.join(ROOT, "tests", "golden", "reference_k.json")) as f:
        ref = json.load(f)["config2"]
    if ref["sha256"] != G.mask_sha256(mask):
        print(json.dumps({"compare": "unavailable", "reason": "reference mask differs"}))
        return 0
    kref = np.zeros((3, 3))
    for j in range(3):
        kref[:, j] = ref["columns"][str(j)]["k_col"]
    d = torch.from_numpy(mask).cuda()
    kd = np.max(np.abs(np.diag(kref)))

    def errors(k):
        e = k_errors(k, kref)
        diag = float(max(e[i, i] for i in range(3)))
        off = float(max(e[i, j] for i in range(3) for j in range(3) if i != j))
        off_kd = max(abs(k[i, j] - kref[i, j]) / kd for i in range(3) for j in range(3) if i != j)
        return diag, off, off_kd

    def plain():
        cols = [api.solve_direction(d, j, fields=False, tol=1e-6, precision="fp32", use_graph=0) for j in range(3)]
        return np.stack([c["k_col"] for c in cols], axis=1), sum(c["stats"]["iters"] for c in cols)

    def tensor(**kw):
        r = api.permeability_tensor(d, **kw)
        return np.asarray(r["k_raw"]), sum(st["iters"] for st in r["stats"])

    def adjoint():
        w = np.zeros((3, 3))
        w[0, 0] = 1.0
        r = api.sensitivity(d, w=w, tol=1e-6, precision="fp32")
        k = kref.copy()
        k[:, 0] = np.asarray(r["k_raw"])[:, 0]  # only the drive-x column is solved for J = k_xx
        return k, 0

    modes = [("plain", plain), ("batched", lambda: tensor(tol=1e-6, precision="fp32")),
             ("dc64", lambda: tensor(tol=1e-8, precision="dc64")),
             ("fp64", lambda: tensor(tol=1e-8, precision="fp64")), ("adjoint_kxx", adjoint)]
    base = None
    for name, fn in modes:
        for rep in range(2):
            torch.cuda.synchronize()
            t = time.perf_counter()
            k, iters = fn()
            torch.cuda.synchronize()
            secs = time.perf_counter() - t
        base = secs if base is None else base
        ed, eo, eok = errors(k)
        print(json.dumps({"mode": name, "seconds": secs, "vs_plain": secs / base, "iters_total": iters,
                          "max_rel_err_diag": ed, "max_rel_err_offdiag": eo, "max_err_offdiag_rel_kii": eok,
                          "meets_1e-5_each": bool(ed <= 1e-5 and eo <= 1e-5)}), flush=True)
    # fixed-pressure inlet/outlet along x on the same mask (another problem: no reference
    # k): sweep time of the tiled kernel's reservoir variant and of the simple kernel
    line = {"mode": "fixed_pressure_x_sweep", "iters": 2001}
    for kernel, key in ((0, "tiled"), (1, "simple")):
        r = api.solve_direction(d, 0, fields=False, bc=(2, 0, 0), tol=1e-12, check_every=200, max_iter=2001,
                                precision="fp32", kernel=kernel)
        line[f"sweep_ms_{key}"] = r["stats"]["sweep_ms"]
        line[f"k_xx_{key}"] = float(r["k_col"][0])
    print(json.dumps(line), flush=True)
    return 0


def run_sequence(args):
    """Precipitation-sequence measurement: a 1536 x 768 disk image (radii 12..30, porosity
    0.55), 24 states of random solid growth to porosity 0.30, extruded to 4 fluid layers
    between solid walls, plus 8 crops of uneven sizes; drives x and y of every domain
    (pm_batch_ktensor, FP32 fields, the paper's criterion 1e-6).  Mode "batch": every
    (domain, drive) problem in each sweep launch, cold start; mode "sequence": the 24 states
    in order, each from the converged fields of the one before.  Iterations are capped
    (--seq-max-iter per problem); the line reports which problems converged."""
    import torch
    from paper_2407_19868_gb300 import api, geometry as G
    api.load()
    t = time.perf_counter()
    states = G.clogging_sequence()
    doms = states + G.crops(states)
    gen_s = time.perf_counter() - t
    modes = ["batch", "sequence"] if args.seq_mode == "both" else [args.seq_mode]
    for mode in modes:
        ds = doms if mode == "batch" else states
        dmasks = [torch.from_numpy(m).cuda() for m in ds]
        # a short solve first: the tile autotuner runs once per shape outside the timing
        api.batch_ktensor(dmasks[:1], drives=[3], tol=args.seq_tol, precision="fp32", max_iter=401, c2=args.seq_c2)
        torch.cuda.synchronize()
        t = time.perf_counter()
        r = api.batch_ktensor(dmasks, drives=[3] * len(ds), tol=args.seq_tol, precision="fp32",
                              max_iter=args.seq_max_iter, sequence=1 if mode == "sequence" else 0, c2=args.seq_c2)
        torch.cuda.synchronize()
        secs = time.perf_counter() - t
        fluid = [int(np.count_nonzero(m == 0)) for m in ds]
        prob = [(d, j) for d in range(len(ds)) for j in range(2) if r["stats"][d][j]["percolates"]]
        upd = sum(fluid[d] * r["stats"][d][j]["iters"] for d, j in prob)
        line = {"workload": "clogging_sequence_1536x768x6_24states" + ("_8crops" if mode == "batch" else ""),
                "mode": mode, "domains": len(ds), "cells": int(sum(m.size for m in ds)), "generate_s": gen_s,
                "status": r["status"], "seconds_all_k": secs, "fluid_voxel_updates_per_s": upd / secs,
                "problems": len(prob),
                "converged": sum(1 for d, j in prob if r["stats"][d][j]["status"] == 0),
                "max_iter": args.seq_max_iter, "tol": args.seq_tol, "c2": args.seq_c2,
                "iters": [[r["stats"][d][j]["iters"] for j in range(2)] for d in range(len(ds))],
                "percolates": [[bool(r["stats"][d][j]["percolates"]) for j in range(2)] for d in range(len(ds))],
                "delta": [[r["stats"][d][j]["delta"] for j in range(2)] for d in range(len(ds))],
                "sweep_ms": r["stats"][0][0]["sweep_ms"], "tile": r["stats"][0][0]["tile"],
                "k_xx": [float(r["k"][d][0, 0]) for d in range(len(ds))],
                "k_yy": [float(r["k"][d][1, 1]) for d in range(len(ds))],
                "shape": [list(m.shape) for m in ds],
                "porosity_2d": [float(np.count_nonzero(m[1:-1] == 0)) / m[1:-1].size for m in ds]}
        print(json.dumps(line), flush=True)
    return 0


def kernel_source_sha():
    """SHA-256 of the sweep kernel's source, to tie stored ncu counters to a version."""
    import hashlib
    h = hashlib.sha256()
    for f in ("pm_sweep_tiled.cuh", "pm_sweep_pair.cuh", "pm_common.cuh"):
        with open(os.path.join(ROOT, "paper_2407_19868_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def stored_traffic(alg_bytes=None):
    """DRAM bytes per sweep launch from the committed ncu summary, if it was taken on
    the current kernel source and for the same kind of launch (algorithmic bytes); else
    None."""
    try:
        with open(os.path.join(ROOT, "profiles", "sweep_tiled_traffic.json")) as f:
            d = json.load(f)
        if d.get("kernel_source_sha256") != kernel_source_sha():
            return None
        for rec in d.get("launches", [d]):
            if alg_bytes is None or abs(rec.get("alg_bytes_per_launch", alg_bytes) - alg_bytes) < 1:
                return float(rec["dram_bytes_per_launch"])
    except Exception:
        pass
    return None


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--tol", type=float, default=TOL)
    ap.add_argument("--precision", default=PRECISION, choices=["fp32", "dc64", "fp64"])
    ap.add_argument("--plain", type=int, default=1, help="also time the plain FP32 form once (rank 0)")
    ap.add_argument("--adjoint", type=int, default=1, help="also time the adjoint form once (rank 0)")
    ap.add_argument("--c2-alt", type=float, default=3.75e5,
                    help="also time the headline form with this c^2 (rank 0; 0 = skip)")
    ap.add_argument("--check-every", type=int, default=200)
    ap.add_argument("--e2e-steps", type=int, default=1)
    ap.add_argument("--cpu-iters", type=int, default=300)
    ap.add_argument("--ref-iters", type=int, default=20)
    ap.add_argument("--autotune", type=int, default=1, help="tune the sweep schedule in the first warm-up solve")
    ap.add_argument("--schedule", type=int, default=0,
                    help="sweep schedule: 0 automatic, -1 persistent CTAs, n > 0 chunks of n planes")
    ap.add_argument("--tile", type=int, default=0, help="sweep tile shape: 0 automatic, 1..3 pinned")
    ap.add_argument("--dc-switch-tol", type=float, default=1e-6,
                    help="defect correction: window change at which the plain FP32 phase ends")
    ap.add_argument("--dc-extrapolate", type=int, default=0,
                    help="defect correction: start the first correction solve from the FP32 phase's "
                         "geometric-tail error estimate (1) or from zero (0)")
    ap.add_argument("--large", type=int, default=0, help="large-domain measurement on an n^3 Boolean pack, then exit")
    ap.add_argument("--large-max-iter", type=int, default=40000)
    ap.add_argument("--field-memory", type=int, default=0,
                    help="large mode: field buffers in device memory (0) or pinned host memory (1: one, 2: both)")
    ap.add_argument("--sequence", action="store_true", help="batched precipitation-sequence measurement, then exit")
    ap.add_argument("--ellipsoid", action="store_true", help="rotated-ellipsoid anisotropy benchmark, then exit")
    ap.add_argument("--thin", action="store_true", help="thin porous media (cylinder cells) benchmark, then exit")
    ap.add_argument("--packs", action="store_true", help="regular SC / BCC / FCC packings benchmark, then exit")
    ap.add_argument("--compare", action="store_true",
                    help="plain / batched / defect-corrected / FP64 / adjoint forms against the oracle, then exit")
    ap.add_argument("--seq-max-iter", type=int, default=400001)
    ap.add_argument("--seq-mode", default="both", choices=["batch", "sequence", "both"])
    ap.add_argument("--seq-tol", type=float, default=1e-6, help="sequence: the paper's window criterion")
    ap.add_argument("--seq-c2", type=float, default=1.5e6,
                    help="sequence: artificial speed of sound squared (the paper's 1.5e6; k does not depend on it)")
    ap.add_argument("--profile-precision", default="fp32", choices=["fp32", "dc64"])
    ap.add_argument("--profile-iters", type=int, default=0,
                    help="profiling case: this many iterations of the benchmark solve, then exit")
    args = ap.parse_args()
    if args.profile_iters > 0:
        return run_profile_case(args)
    if args.large > 0:
        return run_large(args)
    if args.sequence:
        return run_sequence(args)
    if args.ellipsoid:
        return run_ellipsoid(args)
    if args.thin:
        return run_thin(args)
    if args.packs:
        return run_packs(args)
    if args.compare:
        return run_compare(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
