#!/usr/bin/env python3
"""Throughput of the tactile sensor step on GB300: taxel-queries/s.

Workload (default ``metric_run``): 20,480 envs x 20 capsule links x 50
taxels (1,000 per env, 20.48M active taxel queries per step), 64 procedural
objects (superquadrics and convex hulls, 3k-6k faces) as 96^3 FP16 SDF grids
baked on the GPU from the exact meshes, the full noise model (dead taxels,
hysteresis, 3x3 crosstalk, drift).  One step = one replay of the step's CUDA
graph: the pose prologue, the object-sorted work order, the fused sensor
kernel over every env (schedule picked by the autotuner) and the step-counter
advance; a taxel query is one active (env, taxel) pair of one step.  Further
measurements on the same workload add proximity rays and marker pads
("full_sensor_set"), the point-cloud ProximityTaxel ("point_cloud_proximity"),
the elastomer markers with shear anchors ("elastomer_shear") and learned-SDF
objects ("neural_sdf").

  python bench.py [--gpus N --steps K --warmup W] [--impl tg|reference]

``--impl reference`` times the FP64 CPU oracle on the host cores on a bounded
sample of the same workload (the reference arm of this build).  Under torchrun
(N > 1) every rank runs its own shard of envs with no collective on the data
path (weak scaling); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "taxel-queries/s at 20,480 envs×1,000 taxels; neural-SDF vs plain at ≤0.2 mm"
UNIT = "taxel-queries/s"

# Algorithmic HBM bytes per taxel query of the fused step kernel: taxel
# geometry (position, normal, radius) 28 + a link byte, flag byte r/w 2,
# hysteresis x_{t-1} and xi for 7 channels r/w 112, drift for 6 channels r/w
# 48, outputs 58 (contact, clean/noisy depth, clean/noisy force/torque),
# per-env poses and link outputs amortised ~2: 251 B, the per-query figure the
# roofline is taken against.  The SDF cells a query reads are not counted (the
# grids are read from L2 where the object-sorted schedule keeps them).
BYTES_PER_QUERY = 251.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["tg", "reference"], default="tg")
    ap.add_argument("--workload", choices=["metric_run", "config2"], default="metric_run")
    ap.add_argument("--envs", type=int, default=20480)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-full-sensors", action="store_true", help="skip the proximity + markers line")
    ap.add_argument("--no-pc-prox", action="store_true", help="skip the point-cloud proximity line")
    ap.add_argument("--pc-points", type=int, default=5000, help="tracked surface points per object")
    ap.add_argument("--no-shear", action="store_true", help="skip the elastomer shear-anchor line")
    ap.add_argument("--shear-points", type=int, default=1000, help="tracked points per object for the shear anchors")
    ap.add_argument("--no-temperature", action="store_true", help="skip the TemperatureGrid line")
    ap.add_argument("--no-raycast", action="store_true", help="skip the raycast depth backend line")
    ap.add_argument("--no-config2", action="store_true", help="skip the configuration-2 line")
    ap.add_argument("--no-read-delay", action="store_true", help="skip the read-delay line")
    ap.add_argument("--config2-steps", type=int, default=200, help="graph-replayed steps of the configuration-2 line")
    ap.add_argument("--clocks-csv", default=None,
                    help="where to keep the nvidia-smi clock samples of the timed region ({rank} is replaced; "
                         "default: a temporary file)")
    ap.add_argument("--no-config4", action="store_true", help="skip the configuration-4 line")
    ap.add_argument("--config4-objects", type=int, default=256, help="distinct objects of the configuration-4 line")
    ap.add_argument("--config4-steps", type=int, default=500, help="graph-replayed steps of the configuration-4 line")
    ap.add_argument("--config4-points", type=int, default=1_000_000, help="labelled training points per object")
    ap.add_argument("--config4-train-steps", type=int, default=3000, help="Adam steps per object")
    ap.add_argument("--config4-streams", type=int, default=8, help="networks trained at once, one stream each")
    ap.add_argument("--neural-objects", type=int, default=64, help="objects given a learned SDF (0: skip the line)")
    ap.add_argument("--neural-points", type=int, default=2_000_000, help="labelled training points per object")
    ap.add_argument("--neural-steps", type=int, default=3000, help="Adam steps per object")
    ap.add_argument("--neural-check-envs", type=int, default=256, help="envs compared against the exact mesh")
    ap.add_argument("--neural-max-err-mm", type=float, default=0.2,
                    help="probe error (mm) above which an object falls back to its grid")
    ap.add_argument("--oracle-envs", type=int, default=800, help="env sample of the CPU oracle legs")
    ap.add_argument("--oracle-objects", type=int, default=2, help="objects whose envs form the oracle sample")
    ap.add_argument("--oracle-steps", type=int, default=300, help="steps of the cpu_baseline leg")
    ap.add_argument("--schedule", default="auto",
                    choices=["auto"] + [f"{k}{s}" for k in ("grid", "persistent", "pipe1024", "pipe768", "pipe512",
                                                            "grid384", "persistent384")
                                        for s in ("", "-sorted")],
                    help="step-kernel schedule: picked by the autotuner (auto) or fixed")
    return ap.parse_args()


def dist_env():
    from paper_2606_22332_gb300.dist import rank_env

    return rank_env()


def make_workload(args, rank=0):
    from paper_2606_22332_gb300 import workload as W

    if args.workload == "metric_run":
        return W.metric_run(n_envs=args.envs)
    return W.config2(n_envs=args.envs)


def workload_config(args, wl):
    return {
        "workload": (f"{args.workload}: {wl.n_envs} envs x {wl.max_links} links, "
                     f"{wl.n_active // wl.n_envs} active taxels/env, 64 objects as 96^3 FP16 SDF grids "
                     "(exact-mesh bake), full noise model (dead 2%, hysteresis 0.1, 3x3 crosstalk 0.05, drift 1e-3)"),
        "envs_per_gpu": wl.n_envs,
        "active_taxels_per_gpu": wl.n_active,
        "grid": "96^3 fp16",
        "objects": len(wl.objects),
        "l2": "no flush: every step streams ~4.8 GB of taxel state/outputs, far above the 129 MB L2",
        "placement": "per env a target share f ~ U(0.1, 0.3) of active taxels penetrating at the time-0 poses, "
                     "all links pressed by one depth of at most 2 mm (no probe deeper than 3 mm); the timed "
                     "replays run steps 0..K-1 of a fresh episode (warm-up replays first, then reset and rewind)",
    }


# ---------------------------------------------------------------------------
# the CPU oracle legs (cpu_baseline and --impl reference)
# ---------------------------------------------------------------------------
class OracleSample:
    """Bounded sample of the workload for the CPU oracle: the envs that use the
    `oracle_objects` objects with the fewest faces (at most `oracle_envs` envs),
    whose 96^3 grids the oracle bakes itself from the exact meshes (untimed)."""

    def __init__(self, args, wl):
        sys.path.insert(0, os.path.join(ROOT, "tests"))
        from _scenes import bake_objects_oracle, oracle_scene

        counts = np.bincount(wl.obj_id, minlength=len(wl.objects))
        cand = sorted((k for k in range(len(wl.objects)) if counts[k] > 0), key=lambda i: len(wl.objects[i].faces))
        ks = cand[: args.oracle_objects]
        envs = np.flatnonzero(np.isin(wl.obj_id, ks))[: args.oracle_envs]
        sub = wl.subset(envs)
        t0 = time.time()
        baked = bake_objects_oracle([wl.objects[k] for k in ks])
        self.bake_s = time.time() - t0
        objs = list(wl.objects)  # the subset references objects ks only
        for k, b in zip(ks, baked):
            objs[k] = b
        for k in range(len(objs)):
            if k not in ks:
                objs[k] = baked[0]
        sub.objects = objs
        self.sub, self.ks, self.n_envs = sub, ks, len(envs)
        self.faces = [len(wl.objects[k].faces) for k in ks]
        self.sc = oracle_scene(sub)
        self.st = self.sc.new_state()
        self.sc.reset(self.st, 0)
        self.threads = os.cpu_count() or 1
        self.t = 0

    def step_seconds(self):
        t0 = time.time()
        self.sc.step(self.st, self.sub.inputs(self.t), threads=self.threads)
        self.t += 1
        return time.time() - t0

    def describe(self, steps, secs):
        q = self.sub.n_active * steps
        return (f"{self.n_envs} envs x {self.sub.n_active // max(self.n_envs, 1)} taxels x {steps} steps of the same "
                f"workload (the envs of objects {self.ks}, {self.faces} faces; their 96^3 grids baked exactly by the "
                f"oracle in {self.bake_s:.1f} s, untimed); {q} queries in {secs:.2f} s")


def oracle_baseline(args, wl):
    o = OracleSample(args, wl)
    secs = sum(o.step_seconds() for _ in range(args.oracle_steps))
    q = o.sub.n_active * args.oracle_steps
    return {"value": q / secs, "unit": UNIT, "cores": o.threads, "per_core": q / secs / o.threads,
            "kind": "oracle", "sample": o.describe(args.oracle_steps, secs)}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    wl = make_workload(args)
    o = OracleSample(args, wl)
    for _ in range(args.warmup):
        o.step_seconds()
    secs = sum(o.step_seconds() for _ in range(args.steps))
    value = o.sub.n_active * args.steps / secs
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": secs / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(args, wl), "impl": "reference",
        "cpu_baseline": {"kind": "oracle", "cores": o.threads, "sample": o.describe(args.steps, secs),
                         "value": value, "unit": UNIT},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out))


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
class ClockSampler:
    def __init__(self, path):
        self.path = path
        self.p = None

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.p = subprocess.Popen(
                ["nvidia-smi", "-i", os.environ.get("CUDA_VISIBLE_DEVICES", "0").split(",")[0],
                 "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.p = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.p is not None:
            self.p.terminate()
            self.p.wait()
            self.f.close()

    def summary(self):
        if self.p is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        for line in open(self.path):
            parts = [t.strip() for t in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), float(parts[3]) if parts[3] not in ("[N/A]", "N/A") else 0.0,
                             parts[5], parts[6], parts[7], parts[8]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        pmax = max(r[2] for r in rows)
        load = [r for r in rows if r[2] >= 0.5 * pmax] or rows
        reasons = set()
        for r in load:
            for name, v in zip(("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"), r[3:]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": float(np.median([r[0] for r in load])), "sm_max_mhz": float(max(r[1] for r in rows)),
                "reasons": sorted(reasons), "samples": len(rows), "power_w_max": pmax}


def warm_then_rewind(sc, args, dt, stream=None):
    """W untimed graph replays (steps 0..W-1), then every env reset to episode
    0 and the graph rewound to step 0: the timed replays run steps 0..K-1
    from the time-0 placement, as a fresh episode does."""
    sc.graph_launch(args.warmup)
    sc.reset(0)
    sc.graph_seek(0, 0.0, dt)


def accuracy_vs_mesh(args, wl, envs, nobjs, objs):
    """One step of the envs `envs` with the learned SDFs, the plain grids and
    the exact meshes: contact-flag agreement, depth and force errors of each
    pair (None without envs)."""
    import paper_2606_22332_gb300.tg as tg
    from paper_2606_22332_gb300 import workload as W

    if not len(envs):
        return None
    sub = wl.subset(envs)
    inp = sub.inputs(args.warmup)
    outs = {}
    for name, ol in (("neural", nobjs), ("grid", objs),
                     ("mesh", [W.ObjectSpec(kind="mesh", verts=o.verts, faces=o.faces) for o in wl.objects])):
        s2 = tg.Scene(sub.geom(), dict(sub.params, nsdf_max_err_mm=args.neural_max_err_mm), taxel_gid0=0, env_gid0=0)
        s2.upload_objects(ol)
        s2.step(inp)
        outs[name] = {"flags": s2.read(tg.CH_STATE_FLAGS) & 1, "depth": s2.read(tg.CH_DEPTH).astype(np.float64),
                      "f": s2.read(tg.CH_FORCE_TORQUE)[:3].astype(np.float64)}
        s2.sync()
        s2.close()
    act = sub.R > 0

    def cmp(a, b):
        pen = act & ((outs[a]["depth"] > 0) | (outs[b]["depth"] > 0))
        dd = np.abs(outs[a]["depth"] - outs[b]["depth"])[pen] * 1e3
        df = np.linalg.norm(outs[a]["f"] - outs[b]["f"], axis=0)[pen]
        fb = np.linalg.norm(outs[b]["f"], axis=0)[pen]
        return {"contact_flag_agreement": float(np.mean(outs[a]["flags"][act] == outs[b]["flags"][act])),
                "depth_err_mm": {"mean": float(dd.mean()), "p99": float(np.quantile(dd, 0.99)),
                                 "max": float(dd.max())},
                "force_err_N": {"mean": float(df.mean()), "p99": float(np.quantile(df, 0.99))},
                "force_rel_err_median": float(np.median(df / np.maximum(fb, 1e-9)))}

    return {"envs": int(len(envs)), "neural_vs_exact_mesh": cmp("neural", "mesh"),
            "grid_vs_exact_mesh": cmp("grid", "mesh"), "neural_vs_grid": cmp("neural", "grid")}


def train_networks(args, objects, dev, n_points, n_steps, n_streams, seed0):
    """One learned SDF per object, trained on the GPU (labels: the exact-mesh
    query on n_points sampled points, half within 5 mm of the surface), up
    to n_streams networks at once on their own streams; each probed on 8,192
    fresh points.  Returns the networks and (max, mean, p99) probe errors in mm."""
    import torch
    import paper_2606_22332_gb300.tg as tg
    from paper_2606_22332_gb300 import workload as W

    from concurrent.futures import ThreadPoolExecutor

    nets, stats = [None] * len(objects), [None] * len(objects)
    streams = [torch.cuda.Stream(device=dev) for _ in range(max(1, n_streams))]
    # the training loop is bound by its launches on the host: each network's
    # loop runs in its own host thread (the library call releases the
    # interpreter lock) on its own stream
    pool = ThreadPoolExecutor(max_workers=len(streams))
    for g0 in range(0, len(objects), len(streams)):
        group = list(range(g0, min(g0 + len(streams), len(objects))))
        jobs = []
        for k, st in zip(group, streams):
            o = objects[k]
            rng = np.random.default_rng(seed0 + k)
            with torch.cuda.stream(st):
                P = torch.from_numpy(W.sdf_sample_points(rng, o.verts, o.faces, o.lo, o.hi, n_points)).to(dev)
                lab, _ = tg.mesh_sdf(o.verts, o.faces, P, with_grad=False, stream=st.cuda_stream)
                lab_mm = lab * 1e3
            nets[k] = tg.Nsdf(o.lo, o.hi, seed=k)
            jobs.append((pool.submit(nets[k].train, P, lab_mm, steps=n_steps, batch=1 << 14, lr0=1e-2,
                                     lr_final=3e-4, seed=k, record_losses=False, stream=st.cuda_stream), P, lab_mm))
        for j, _, _ in jobs:
            j.result()
        torch.cuda.synchronize()
        del jobs
        for k in group:
            o = objects[k]
            probe = torch.from_numpy(W.sdf_sample_points(np.random.default_rng(seed0 + 50000 + k), o.verts, o.faces,
                                                         o.lo, o.hi, 8192)).to(dev)
            mx, mean = nets[k].probe(o.verts, o.faces, probe)
            ex, _ = tg.mesh_sdf(o.verts, o.faces, probe, with_grad=False)
            p99 = float(torch.quantile((nets[k].eval(probe) - ex).abs() * 1e3, 0.99).item())
            stats[k] = (mx, mean, p99)
    return nets, stats


def config4_line(args, dev, stream):
    """Configuration 4: 20,480 envs with T_e ~ U{200..1000} taxels over
    L_e ~ U{10..20} links, 256 distinct objects, one learned SDF per object
    (trained here on the GPU) answering the near-field contact query with
    fallback to the object's 96^3 FP16 grid where its error probe exceeds
    0.2 mm, per-step domain randomisation of mu, k and the object scale,
    500 graph-replayed steps; the same workload with the plain grids timed
    alongside, and a subset of envs compared against the exact meshes."""
    import torch
    import paper_2606_22332_gb300.tg as tg
    from paper_2606_22332_gb300 import workload as W

    t_setup = time.time()
    wl = W.config4(n_envs=args.envs, n_objects=args.config4_objects)
    objs = []
    for o in wl.objects:
        vals = tg.bake_grid(o.verts, o.faces, o.dims, o.lo, o.hi, fp16=o.fp16)
        objs.append(W.ObjectSpec(kind="grid", dims=o.dims, lo=o.lo, hi=o.hi, fp16=o.fp16, values=vals, name=o.name))
    d_in = {k: torch.as_tensor(getattr(wl, k)).to(dev) for k in ("link_pose", "link_vel", "obj_pose", "obj_vel", "obj_id")}
    dt = wl.params["dt"]
    steps = args.config4_steps

    def timed(objects, params, sched=None):
        sc = tg.Scene(wl.geom(), params)
        sc.upload_objects(objects)
        tune = None
        if sched is None:
            sc.step(dict(d_in, pose_dt=0.0, step=0))
            tune = sc.autotune(dict(d_in, pose_dt=0.0, step=0), steps=3)
            sched = {"schedule": tune["chosen"]["schedule"], "sorted": bool(tune["chosen"]["sorted"])}
        sc.set_schedule(**sched)
        sc.profile(True)
        sc.graph_capture(dict(d_in, pose_dt=0.0, step=0), pose_dt_per_step=dt)
        warm_then_rewind(sc, args, dt)
        torch.cuda.synchronize()
        sc.profile_read()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sc.graph_launch(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        _, step_ms, n = sc.profile_read()
        used = [k for k in range(len(objects)) if sc.object_info(k)[0] == tg.TG_OBJ_NEURAL]
        sc.graph_release()
        sc.close()
        return ms, step_ms / max(n, 1), sched, tune, used

    ms_plain, step_plain, sched, tune, _ = timed(objs, wl.params)
    t0 = time.time()
    nets, stats = train_networks(args, wl.objects, dev, args.config4_points, args.config4_train_steps,
                                 args.config4_streams, seed0=7000)
    train_s = time.time() - t0
    nobjs = [W.ObjectSpec(kind="neural", dims=objs[k].dims, lo=objs[k].lo, hi=objs[k].hi, fp16=objs[k].fp16,
                          values=objs[k].values, net=nets[k], nsdf_err_mm=stats[k][0], name=objs[k].name)
             for k in range(len(objs))]
    ms_net, step_net, _, _, used = timed(nobjs, dict(wl.params, nsdf_max_err_mm=args.neural_max_err_mm), sched)
    envs = np.flatnonzero(np.isin(wl.obj_id, used))[: args.neural_check_envs]
    acc = accuracy_vs_mesh(args, wl, envs, nobjs, objs)
    for net in nets:
        net.close()
    pm = np.array(stats)
    n_q = wl.n_active
    faces = [len(o.faces) for o in wl.objects]
    return {
        "workload": f"configuration 4: {wl.n_envs} envs, uneven 200-1,000 taxels over 10-20 links "
                    f"({n_q} active taxels), {len(wl.objects)} distinct objects of {min(faces)}-{max(faces)} faces, "
                    "per-step domain randomisation (mu U(0.4, 1.2), k U(5e3, 2e4) N/m, scale U(0.8, 1.2)), "
                    f"{steps} graph-replayed steps, schedule {sched}",
        "value": n_q * steps / (ms_net * 1e-3), "unit": UNIT, "ms_per_step": ms_net / steps,
        "step_kernels_ms": round(step_net, 4),
        "plain_grid": {"value": n_q * steps / (ms_plain * 1e-3), "ms_per_step": ms_plain / steps,
                       "step_kernels_ms": round(step_plain, 4)},
        "vs_plain_grid": round(ms_plain / ms_net, 4),
        "objects_using_network": len(used), "fallback_above_mm": args.neural_max_err_mm,
        "envs_using_network": int(np.isin(wl.obj_id, used).sum()),
        "training": {"points_per_object": args.config4_points, "steps": args.config4_train_steps,
                     "batch": 1 << 14, "networks_at_once": args.config4_streams, "seconds_total": round(train_s, 1),
                     "labels": "GPU exact-mesh query"},
        "probe_err_mm": {"max_over_objects": float(pm[:, 0].max()), "median_of_max": float(np.median(pm[:, 0])),
                         "mean": float(pm[:, 1].mean()), "p99_median": float(np.median(pm[:, 2]))},
        "accuracy": acc,
        "autotune": tune["candidates"] if tune else None,
        "gpu_launches": steps * (5 + (1 if sched["schedule"].startswith("pipe") or sched["sorted"] else 0)),
        "setup_s": round(time.time() - t_setup, 1),
    }


def neural_line(args, dev, stream, step_inputs):
    """Configuration 3: learned SDFs for 64 procedural meshes of 5k-20k faces
    (the headline's layout of envs, links and taxels, placed on these
    objects), each trained on the GPU on 2M points labelled by the exact-mesh
    query and probed against it; the workload is timed with the plain 96^3
    FP16 grids and with the networks answering the contact query (fallback to
    the grid above 0.2 mm), and a subset of envs is compared against the grid
    and the exact mesh."""
    import torch
    import paper_2606_22332_gb300.tg as tg
    from paper_2606_22332_gb300 import workload as W

    wl = W.metric_run(seed=20260004, n_envs=args.envs, faces=(5000, 20000))
    objs = []
    for o in wl.objects:
        vals = tg.bake_grid(o.verts, o.faces, o.dims, o.lo, o.hi, fp16=o.fp16)
        objs.append(W.ObjectSpec(kind="grid", dims=o.dims, lo=o.lo, hi=o.hi, fp16=o.fp16, values=vals, name=o.name))
    d_in = {k: torch.as_tensor(getattr(wl, k)).to(dev) for k in ("link_pose", "link_vel", "obj_pose", "obj_vel", "obj_id")}
    dt = wl.params["dt"]
    # the plain grid path on this workload, in the schedule the autotuner picks for it
    sc0 = tg.Scene(wl.geom(), wl.params)
    sc0.upload_objects(objs)
    sc0.step(step_inputs(0, d_in))
    sched = sc0.autotune(step_inputs(0, d_in), steps=3)["chosen"]
    sched = {"schedule": sched["schedule"], "sorted": bool(sched["sorted"])}
    sc0.set_schedule(**sched)
    sc0.graph_capture(step_inputs(0, d_in), pose_dt_per_step=dt)
    warm_then_rewind(sc0, args, dt)
    torch.cuda.synchronize()
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    p0.record(stream)
    sc0.graph_launch(args.steps)
    p1.record(stream)
    torch.cuda.synchronize()
    t_plain_ms = p0.elapsed_time(p1)
    sc0.graph_release()
    sc0.close()
    n_obj = min(args.neural_objects, len(wl.objects))
    t0 = time.time()
    nets, probe_stats = [], []
    for k in range(n_obj):
        o = wl.objects[k]
        rng = np.random.default_rng(1000 + k)
        P = torch.from_numpy(W.sdf_sample_points(rng, o.verts, o.faces, o.lo, o.hi, args.neural_points)).to(dev)
        lab, _ = tg.mesh_sdf(o.verts, o.faces, P, with_grad=False)
        net = tg.Nsdf(o.lo, o.hi, seed=k)
        net.train(P, lab * 1e3, steps=args.neural_steps, batch=1 << 14, lr0=1e-2, lr_final=3e-4, seed=k,
                  record_losses=False)
        probe = torch.from_numpy(W.sdf_sample_points(np.random.default_rng(5000 + k), o.verts, o.faces, o.lo, o.hi,
                                                     8192)).to(dev)
        mx, mean = net.probe(o.verts, o.faces, probe)
        ex, _ = tg.mesh_sdf(o.verts, o.faces, probe, with_grad=False)
        p99 = float(torch.quantile((net.eval(probe) - ex).abs() * 1e3, 0.99).item())
        nets.append(net)
        probe_stats.append((mx, mean, p99))
        del P, lab
    torch.cuda.synchronize()
    train_s = time.time() - t0
    nobjs = [W.ObjectSpec(kind="neural", dims=objs[k].dims, lo=objs[k].lo, hi=objs[k].hi, fp16=objs[k].fp16,
                          values=objs[k].values, net=nets[k], nsdf_err_mm=probe_stats[k][0], name=objs[k].name)
             for k in range(n_obj)] + list(objs[n_obj:])
    sc = tg.Scene(wl.geom(), dict(wl.params, nsdf_max_err_mm=args.neural_max_err_mm))
    sc.upload_objects(nobjs)
    used = [k for k in range(n_obj) if sc.object_info(k)[0] == tg.TG_OBJ_NEURAL]
    sc.set_schedule(**sched)
    sc.profile(True)
    sc.graph_capture(step_inputs(0, d_in), pose_dt_per_step=dt)
    warm_then_rewind(sc, args, dt)
    torch.cuda.synchronize()
    sc.profile_read()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sc.graph_launch(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    pose_ms, step_ms, nsteps = sc.profile_read()
    sc.graph_release()
    sc.close()
    q_used = int(np.isin(wl.obj_id, used).sum()) * (wl.n_active // wl.n_envs)

    # accuracy on envs whose object uses its network: network vs 96^3 grid vs exact mesh, one step
    envs = np.flatnonzero(np.isin(wl.obj_id, used))[: args.neural_check_envs]
    acc = accuracy_vs_mesh(args, wl, envs, nobjs, objs)
    pm = np.array(probe_stats)
    for net in nets:
        net.close()
    return {
        "objects_with_network": n_obj, "objects_using_network": len(used), "envs_using_network": int(np.isin(wl.obj_id, used).sum()),
        "fallback_above_mm": args.neural_max_err_mm,
        "training": {"points_per_object": args.neural_points, "steps": args.neural_steps, "batch": 1 << 14,
                     "seconds_total": round(train_s, 1), "labels": "GPU exact-mesh query"},
        "probe_err_mm": {"max_over_objects": float(pm[:, 0].max()), "median_of_max": float(np.median(pm[:, 0])),
                         "mean": float(pm[:, 1].mean()), "p99_median": float(np.median(pm[:, 2]))},
        "value": wl.n_active * args.steps / (ms / 1e3), "unit": UNIT, "ms_per_step": ms / args.steps,
        "vs_plain_grid": round(t_plain_ms / ms, 4), "plain_grid_ms_per_step": t_plain_ms / args.steps,
        "workload": f"configuration 3: {wl.n_envs} envs x {wl.max_links} links x 50 taxels on 64 meshes of "
                    f"{min(len(o.faces) for o in wl.objects)}-{max(len(o.faces) for o in wl.objects)} faces "
                    "(superquadrics and subdivided hulls), schedule " + f"{sched}",
        "queries_answered_by_network_per_step": q_used,
        "step_kernels_ms": round((step_ms) / max(nsteps, 1), 4),
        "accuracy": acc,
    }


READ_DELAY_RING_BYTES = 64.0  # per query: this step's noisy-chain input written (8 x 4 B), a delayed one read


def read_delay_line(args, wl, objs, dev, stream, sched, peaks_fn):
    """The headline workload with a read delay of 2 steps and a jitter of 1
    (Sensor Noise Model, base noise): the same graph-replayed step with each
    taxel's delayed-readout ring (8 channels x 4 slots) in HBM."""
    import torch

    import paper_2606_22332_gb300.tg as tg

    dt = wl.params["dt"]
    sc = tg.Scene(wl.geom(), dict(wl.params, read_delay=2, read_jitter=1))
    sc.upload_objects(objs)
    d_in = {k: torch.as_tensor(getattr(wl, k)).to(dev) for k in ("link_pose", "link_vel", "obj_pose", "obj_vel", "obj_id")}
    sc.set_schedule(**sched)
    sc.profile(True)
    sc.graph_capture(dict(d_in, pose_dt=0.0, step=0), pose_dt_per_step=dt)
    warm_then_rewind(sc, args, dt)
    torch.cuda.synchronize()
    sc.profile_read()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sc.graph_launch(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    pose_ms, step_ms, n = sc.profile_read()
    sc.graph_release()
    sc.close()
    bpq = BYTES_PER_QUERY + READ_DELAY_RING_BYTES
    step_avg = step_ms / max(n, 1)
    achieved = bpq * wl.n_active / (step_avg * 1e-3) / 1e9
    peak, kind = peaks_fn()
    return {"sensors": "headline step with a read delay of 2 steps and a jitter of 1 step on the noisy readout",
            "value": wl.n_active * args.steps / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms / args.steps,
            "step_kernel_ms": round(step_avg, 4),
            "step_kernel_roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                                     "frac": round(achieved / peak, 4), "peak_kind": kind,
                                     "algorithmic_bytes_per_query": bpq},
            "ring_bytes": 4 * 8 * 4 * wl.n_taxels, "gpu_launches": 4 * args.steps}


def config2_line(args, dev, stream, pg, peaks_fn):
    """Configuration 2 as stated: 20,480 envs with T_e ~ U{200..1000}
    taxels over L_e ~ U{10..20} links, 64 objects as 96^3 FP16 grids baked
    from the exact meshes, proximity (8 rays, 50 mm) and elastomer markers
    (5 pads x 16 x 16) on, the full noise model, 200 graph-replayed steps of
    a fresh episode (schedule picked by the autotuner for this workload)."""
    import torch

    import paper_2606_22332_gb300.tg as tg
    from paper_2606_22332_gb300 import workload as W
    from paper_2606_22332_gb300.dist import max_over_ranks

    wl = W.config2(n_envs=args.envs)
    objs = []
    for o in wl.objects:
        vals = tg.bake_grid(o.verts, o.faces, o.dims, o.lo, o.hi, fp16=o.fp16)
        objs.append(W.ObjectSpec(kind="grid", dims=o.dims, lo=o.lo, hi=o.hi, fp16=o.fp16, values=vals, name=o.name))
    sc = tg.Scene(wl.geom(), wl.params, sensors=tg.TG_SENSOR_PROX | tg.TG_SENSOR_MARKERS, pads=wl.pads)
    sc.upload_objects(objs)
    d_in = {k: torch.as_tensor(getattr(wl, k)).to(dev) for k in ("link_pose", "link_vel", "obj_pose", "obj_vel", "obj_id")}
    dt = wl.params["dt"]
    sc.step(dict(d_in, pose_dt=0.0, step=0))
    tune = sc.autotune(dict(d_in, pose_dt=0.0, step=0), steps=3)
    sc.profile(True)
    sc.graph_capture(dict(d_in, pose_dt=0.0, step=0), pose_dt_per_step=dt)
    warm_then_rewind(sc, args, dt)
    torch.cuda.synchronize()
    sc.profile_read()
    steps = args.config2_steps
    if pg:
        pg.barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sc.graph_launch(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = max_over_ranks(e0.elapsed_time(e1), dev)
    pose_ms, step_ms, n = sc.profile_read()
    pen = float((sc.buffer(tg.CH_DEPTH) > 0).sum().item()) / max(wl.n_active, 1)
    sc.graph_release()
    sc.close()
    n_q = wl.n_active
    step_avg = step_ms / max(n, 1)
    achieved = BYTES_PER_QUERY * n_q / (step_avg * 1e-3) / 1e9
    peak, kind = peaks_fn()
    return {"sensors": "configuration 2: uneven envs (200-1,000 taxels over 10-20 links), 64 objects as 96^3 FP16 "
                       "grids, proximity (8 rays, 50 mm) and markers (5 pads x 16x16), full noise model",
            "envs": wl.n_envs, "active_taxels": n_q, "steps": steps, "value": n_q * steps / (ms * 1e-3),
            "unit": UNIT, "ms_per_step": ms / steps, "step_kernel_ms": round(step_avg, 4),
            "step_kernel_roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                                     "frac": round(achieved / peak, 4), "peak_kind": kind,
                                     "algorithmic_bytes_per_query": BYTES_PER_QUERY},
            "penetrating_share_last_step": round(pen, 4), "placement": wl.meta.get("placement"),
            "schedule": {"chosen": tune["chosen"], "candidates": tune["candidates"],
                         "sensor_kernel_threads": tune["sensor_chosen"],
                         "sensor_candidates": tune["sensor_candidates"]},
            # pose, [order], step, proximity, markers, step-counter advance
            "gpu_launches": steps * (5 + (1 if tune["chosen"]["schedule"].startswith("pipe") or tune["chosen"]["sorted"]
                                          else 0))}


def tune_sensor_shapes(sc, inputs, sched):
    """The autotuner's launch shapes for the scene's sensor kernels, on the
    step schedule `sched` (kept); returns {kernel: threads} and the trials."""
    sc.step(inputs)
    tune = sc.autotune(inputs, steps=2)
    sc.set_schedule(**sched)
    return tune["sensor_chosen"], tune["sensor_candidates"]


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


STEP_KERNEL_SOURCES = ("step.cu", "step_common.cuh", "geom.cuh", "df.cuh", "rng.cuh", "internal.h")


def step_kernel_sha():
    """sha256 (16 hex digits) over the step kernel's source files."""
    h = hashlib.sha256()
    for f in STEP_KERNEL_SOURCES:
        h.update(open(os.path.join(ROOT, "paper_2606_22332_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def traffic_from_profile():
    """dram bytes per launch of the step kernel from the committed ncu summary,
    if it was taken on the current kernel sources (else None)."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    rec = json.load(open(p)).get("step_kernel")
    if not rec or rec.get("source_sha") != step_kernel_sha():
        return None
    return rec.get("dram_bytes_per_launch_full")


def _quat_mat(q):
    """rotation matrices [n][3][3] of unit quaternions [n][4] (w, x, y, z)"""
    w, x, y, z = (q[:, i].astype(np.float64) for i in range(4))
    return np.stack([np.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)], 1),
                     np.stack([2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)], 1),
                     np.stack([2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], 1)], 1)


def raycast_line(args, wl, objs, dev, stream):
    """Raycast depth backend: every active taxel of the headline workload (its
    time-0 pose) queried against its env object's triangle mesh through a
    bounding volume hierarchy, one launch per object."""
    import time

    import torch

    from paper_2606_22332_gb300 import tg

    E, L = wl.n_envs, wl.max_links
    counts = (wl.link_rows * wl.link_cols).astype(np.int64)
    link_of = np.repeat(np.arange(E * L), counts)
    act = wl.R > 0
    lp = wl.link_pose.reshape(E * L, 7)[link_of]
    xw = np.einsum("nij,nj->ni", _quat_mat(lp[:, 3:]),
                   np.stack([wl.x, wl.y, wl.z], 1).astype(np.float64)) + lp[:, :3]
    env_of = link_of // L
    op = wl.obj_pose[env_of]
    q = np.einsum("nji,nj->ni", _quat_mat(op[:, 3:]), xw - op[:, :3])  # R_C^T (x_w - p_C)
    oid = wl.obj_id[env_of]
    groups = []
    for o, ob in enumerate(objs):
        sel = np.flatnonzero(act & (oid == o))
        if ob.verts is None or len(sel) == 0:
            continue
        bvh = tg.MeshBvh(ob.verts, ob.faces)
        groups.append((bvh, torch.as_tensor(q[sel].astype(np.float32), device=dev),
                       torch.as_tensor(wl.R[sel].astype(np.float32), device=dev), sel))
    n = sum(len(g[3]) for g in groups)
    outs = [None] * len(groups)

    def one_pass():
        for k, (bvh, qd, rd, _) in enumerate(groups):
            outs[k] = bvh.depth(qd, rd, stream=stream.cuda_stream)

    for _ in range(max(args.warmup, 1)):
        one_pass()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        one_pass()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    touching = sum(int((o[0] > 0).sum().item()) for o in outs)
    out = {"sensors": f"raycast depth backend over {n} active taxels of the headline workload (time-0 poses), "
                      f"{len(groups)} object meshes of 3k-6k faces, one tree per mesh",
           "value": n / (ms * 1e-3), "unit": "probe-queries/s", "ms_per_pass": ms,
           "probes_in_contact": round(touching / max(n, 1), 4), "gpu_launches": len(groups) * args.steps}
    if not args.no_cpu_baseline:
        import oracle

        rng = np.random.default_rng(20260013)
        k = min(400, n)
        pick = rng.choice(n, k, replace=False)
        allsel = np.concatenate([g[3] for g in groups])
        t0 = time.perf_counter()
        for i in allsel[pick]:
            ob = objs[oid[i]]
            oracle.raycast_depth(ob.verts, ob.faces, 1.0, q[i:i + 1], np.array([[0.0, 0.0, 1.0]]), float(wl.R[i]))
        el = time.perf_counter() - t0
        out["cpu_baseline"] = {"value": k / el, "unit": "probe-queries/s", "cores": 1, "kind": "oracle",
                               "sample": f"{k} random active taxels of the same workload, brute force over the faces"}
    for g in groups:
        g[0].close()
    return out


def raycast_step_line(args, wl, dev, stream, sched, plain_step_ms, launches_per_step):
    """The headline step with the raycast contact-depth backend selected: the
    same envs, poses and noise model, every object answered by its triangle
    mesh (the one behind its baked grid) through a bounding volume hierarchy.
    Per step one pre-pass launch finds each taxel's nearest triangle within
    R, then the step kernel reads that distance and the face normal."""
    import dataclasses

    import torch

    import paper_2606_22332_gb300.tg as tg

    dt = wl.params["dt"]
    objs = [dataclasses.replace(o, kind="mesh", values=None) for o in wl.objects]
    sc = tg.Scene(wl.geom(), dict(wl.params, depth_backend="raycast"))
    sc.upload_objects(objs)
    d_in = {k: torch.as_tensor(getattr(wl, k)).to(dev) for k in ("link_pose", "link_vel", "obj_pose", "obj_vel", "obj_id")}
    sc.set_schedule(**sched)
    sc.profile(True)
    sc.graph_capture(dict(d_in, pose_dt=0.0, step=0), pose_dt_per_step=dt)
    warm_then_rewind(sc, args, dt)
    torch.cuda.synchronize()
    sc.profile_read()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sc.graph_launch(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    _, step_ms, n = sc.profile_read()
    contact = float(np.count_nonzero(sc.read(tg.CH_CONTACT, False))) / wl.n_active
    sc.graph_release()
    sc.close()
    step_avg = step_ms / max(n, 1)
    faces = [len(o.faces) for o in objs]
    return {"sensors": f"headline step with the raycast contact-depth backend: {len(objs)} triangle meshes of "
                       f"{min(faces)}-{max(faces)} faces, one tree per mesh, nearest triangle within R per taxel",
            "value": wl.n_active * args.steps / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms / args.steps,
            "step_kernels_ms": round(step_avg, 4),
            "raycast_prepass_ms": round(step_avg - plain_step_ms, 4),
            "contact_share_last_step": round(contact, 4),
            "gpu_launches": (launches_per_step + 1) * args.steps}


TEMP_BYTES_PER_CELL = 16.0  # T and T_meas, each read and written once per step


def temperature_line(args, dev, stream, pg, peaks_fn):
    """TemperatureGrid: one 8 x 8 x 16 grid per fingertip link (5 per env) at
    200 Hz, 20 % of the grids touching a ball each step; cells/s, the step
    kernel's HBM roofline and the oracle on a sample of grids."""
    import torch

    from paper_2606_22332_gb300 import tg
    from paper_2606_22332_gb300 import workload as W
    from paper_2606_22332_gb300.dist import max_over_ranks

    dims = (8, 8, 16)
    wl = W.temperature_grids(n_envs=args.envs, links_per_env=5, dims=dims)
    G, cells = wl["G"], dims[0] * dims[1] * dims[2]
    rng = np.random.default_rng(20260012)
    contacts = W.temperature_contacts(rng, G, dims, share=0.2)
    cd = {k: torch.as_tensor(v, device=dev) for k, v in contacts.items()}
    grids = tg.TempGrid(dims, wl["voxel"], wl["material"])
    dt, t_amb = 1.0 / 200.0, 22.0
    s_ptr = stream.cuda_stream
    for _ in range(args.warmup):
        grids.step(dt, t_amb, contacts=cd, stream=s_ptr)
    torch.cuda.synchronize()
    if pg:
        pg.barrier()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(args.steps):
        grids.step(dt, t_amb, contacts=cd, stream=s_ptr)
    t1.record(stream)
    torch.cuda.synchronize()
    ms = max_over_ranks(t0.elapsed_time(t1), dev) / args.steps
    tmax = float(grids.buffer().max().item())
    grids.close()
    peak, kind = peaks_fn()
    achieved = TEMP_BYTES_PER_CELL * G * cells / (ms * 1e-3) / 1e9
    out = {"sensors": f"TemperatureGrid: {G} grids (5 fingertip links x {args.envs} envs) of 8x8x16 cells, "
                      "2.5 mm voxels, silicone-like skin, 200 Hz, 20 % of the grids touching a ball (1 in 8 hot, 45 C)",
           "value": G * cells / (ms * 1e-3), "unit": "grid-cells/s", "ms_per_step": ms,
           "contacts_per_step": int(contacts["offsets"][-1]), "max_cell_temp_c": round(tmax, 3),
           "gpu_launches": args.steps,
           "roofline": {"bound": "hbm", "kernel": "temp_step_kernel", "achieved": round(achieved, 1),
                        "peak": peak, "unit": "GB/s", "frac": round(achieved / peak, 4), "peak_kind": kind,
                        "algorithmic_bytes_per_cell": TEMP_BYTES_PER_CELL}}
    if not args.no_cpu_baseline and dist_env()[1] == 0:
        import time

        from oracle import temperature as TO

        n_s = min(G, 256)
        T0 = np.full(dims, 22.0)
        tc = time.perf_counter()
        for g in range(n_s):
            m = wl["material"][g].astype(np.float64)
            mat = dict(k=m[0], rho=m[1], cp=m[2], emissivity=m[3], h=m[4], tau=m[5])
            cs = [(int(contacts["cell"][c]), float(contacts["temp"][c]), float(contacts["k"][c]),
                   float(contacts["area"][c])) for c in range(contacts["offsets"][g], contacts["offsets"][g + 1])]
            TO.step(T0, T0, wl["voxel"][g].astype(np.float64), mat, dt, t_amb, contacts=cs)
        el = time.perf_counter() - tc
        out["cpu_baseline"] = {"value": n_s * cells / el, "unit": "grid-cells/s", "cores": 1, "kind": "oracle",
                               "sample": f"{n_s} grids x 1 step of the same workload (numpy FFT, one core)"}
    return out


def run_tg(args):
    import torch

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)
        pg = dist
    import paper_2606_22332_gb300.tg as tg
    from paper_2606_22332_gb300 import workload as W

    t_setup = time.time()
    wl = make_workload(args, rank)
    E, T = wl.n_envs, wl.n_taxels
    # objects: the exact-mesh bake of every grid on the GPU
    objs = []
    for o in wl.objects:
        vals = tg.bake_grid(o.verts, o.faces, o.dims, o.lo, o.hi, fp16=o.fp16)
        objs.append(W.ObjectSpec(kind="grid", dims=o.dims, lo=o.lo, hi=o.hi, fp16=o.fp16, values=vals, name=o.name))
    torch.cuda.synchronize()
    bake_s = time.time() - t_setup
    from paper_2606_22332_gb300.dist import max_over_ranks, shard_ids

    gid0, egid0 = shard_ids(rank, E, T)
    scene = tg.Scene(wl.geom(), wl.params, taxel_gid0=gid0, env_gid0=egid0)
    scene.upload_objects(objs)
    d_in = {k: torch.as_tensor(getattr(wl, k)).to(dev) for k in ("link_pose", "link_vel", "obj_pose", "obj_vel", "obj_id")}
    stream = torch.cuda.current_stream()
    dt = wl.params["dt"]

    def step_inputs(t, src):
        return dict(src, pose_dt=t * dt, step=t)

    # schedule picked by the autotuner on the live scene (state restored after)
    scene.step(step_inputs(0, d_in))
    if args.schedule == "auto":
        tune = scene.autotune(step_inputs(0, d_in), steps=3)
    else:
        scene.set_schedule(args.schedule.split("-")[0], sorted=args.schedule.endswith("sorted"))
        tune = {"candidates": "fixed by --schedule"}
    sched = scene.schedule()
    # pose, [order / order records], step, advance
    launches_per_step = 3 + (1 if sched["schedule"].startswith("pipe") or (sched["sorted"] and len(wl.objects) > 1)
                             else 0)

    # the step as a CUDA graph: replay r runs step r with pose_dt = r dt
    scene.profile(True)
    scene.reset(0)
    scene.graph_capture(step_inputs(0, d_in), pose_dt_per_step=dt)
    scene.graph_launch(1)                       # step 0 from a fresh episode: the shares at the placement
    torch.cuda.synchronize()
    act_n = max(wl.n_active, 1)
    pen_share0 = float((scene.buffer(tg.CH_DEPTH) > 0).sum().item()) / act_n
    contact_share0 = float((scene.read(tg.CH_STATE_FLAGS) & 1).sum()) / act_n
    scene.graph_launch(max(args.warmup - 1, 0))
    scene.reset(0)
    scene.graph_seek(0, 0.0, dt)
    torch.cuda.synchronize()
    scene.sync()
    scene.profile_read()

    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clk = ClockSampler(args.clocks_csv.replace("{rank}", str(rank)) if args.clocks_csv
                       else f"/tmp/tg_clocks_{os.getpid()}_rank{rank}.csv")
    with clk:
        ev0.record(stream)
        scene.graph_launch(args.steps)
        ev1.record(stream)
        torch.cuda.synchronize()
    if pg:
        pg.barrier()
    ms = ev0.elapsed_time(ev1)
    pose_ms, step_ms, nsteps = scene.profile_read()
    scene.sync()
    pen_share_last = float((scene.buffer(tg.CH_DEPTH) > 0).sum().item()) / act_n
    contact_share_last = float((scene.read(tg.CH_STATE_FLAGS) & 1).sum()) / act_n
    scene.graph_release()
    scene.profile(False)
    t_max = max_over_ranks(ms, dev)
    n_q = wl.n_active * ws
    value = n_q * args.steps / (t_max / 1e3)

    # e2e: host inputs through the C-ABI (H2D inside), per-link results read back to host
    e2e = e2e_taxel = None
    if not args.no_e2e:
        pinned = {k: torch.as_tensor(getattr(wl, k)).pin_memory() for k in d_in}
        out_w = torch.empty((E * wl.max_links, tg.LINK_REC), dtype=torch.float32).pin_memory()
        out_c = torch.empty((E * wl.max_links, 2), dtype=torch.int32).pin_memory()
        h2d = sum(v.numel() * v.element_size() for v in pinned.values())
        d2h = out_w.numel() * 4 + out_c.numel() * 4
        k2 = args.steps
        for t in range(args.warmup):
            scene.step(step_inputs(t, pinned))
            scene.read(tg.CH_LINK_WRENCH, out=out_w)
        scene.reset(0)
        torch.cuda.synchronize()
        if pg:
            pg.barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for t in range(k2):  # the same step indices (same poses) as the device-timed region
            scene.step(step_inputs(t, pinned))
            scene.read(tg.CH_LINK_WRENCH, out=out_w)
            scene.read(tg.CH_LINK_COUNT, out=out_c)
        e1.record(stream)
        torch.cuda.synchronize()
        ems = max_over_ranks(e0.elapsed_time(e1), dev)
        e2e = {"value": n_q * k2 / (ems / 1e3), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h),
               "note": "time-0 poses/velocities copied from pinned host memory every step (the C-ABI stages them); "
                       "per-link wrench sums and contact counts (agg_force / agg_bool observations) read back to "
                       "pinned host memory every step; same step indices as the device-timed region"}
        # the same, reading every taxel's noisy readout back instead (contact bit, depth, force/torque)
        T_all = wl.n_taxels
        o_c = torch.empty(T_all, dtype=torch.uint8).pin_memory()
        o_d = torch.empty(T_all, dtype=torch.float32).pin_memory()
        o_f = torch.empty((6, T_all), dtype=torch.float32).pin_memory()
        d2h_t = o_c.numel() + o_d.numel() * 4 + o_f.numel() * 4
        scene.reset(0)
        torch.cuda.synchronize()
        if pg:
            pg.barrier()
        e0.record(stream)
        for t in range(k2):
            scene.step(step_inputs(t, pinned))
            scene.read(tg.CH_CONTACT, noisy=True, out=o_c)
            scene.read(tg.CH_DEPTH, noisy=True, out=o_d)
            scene.read(tg.CH_FORCE_TORQUE, noisy=True, out=o_f)
        e1.record(stream)
        torch.cuda.synchronize()
        ems2 = max_over_ranks(e0.elapsed_time(e1), dev)
        e2e_taxel = {"value": n_q * k2 / (ems2 / 1e3), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                     "d2h_bytes_per_step": int(d2h_t),
                     "note": "as e2e, but every taxel's noisy contact bit, depth and force/torque (29 B per "
                             "taxel) read back to pinned host memory every step instead of the per-link sums"}

    # second line: the same workload with proximity rays and marker pads on
    full = None
    if not args.no_full_sensors:
        wlf = W.add_pads(wl)
        pf = dict(wl.params, prox_rays=8)
        sc2 = tg.Scene(wlf.geom(), pf, sensors=tg.TG_SENSOR_PROX | tg.TG_SENSOR_MARKERS, taxel_gid0=gid0,
                       env_gid0=egid0, pads=wlf.pads)
        sc2.upload_objects(objs)
        shapes2, _ = tune_sensor_shapes(sc2, step_inputs(0, d_in), sched)
        sc2.graph_capture(step_inputs(0, d_in), pose_dt_per_step=dt)
        warm_then_rewind(sc2, args, dt)
        torch.cuda.synchronize()
        if pg:
            pg.barrier()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        sc2.graph_launch(args.steps)
        f1.record(stream)
        torch.cuda.synchronize()
        fms = max_over_ranks(f0.elapsed_time(f1), dev)
        prox_share = float((sc2.buffer(tg.CH_PROX) > 0).sum().item()) / max(wl.n_active, 1)
        sc2.graph_release()
        sc2.close()
        full = {"sensors": "headline step + proximity (8 rays, 50 mm range, sphere tracing) + marker dilation "
                           "(5 pads x 16x16 markers per env, 5x5 Gaussian kernel, sigma 1.5 mm)",
                "value": n_q * args.steps / (fms / 1e3), "unit": UNIT, "ms_per_step": fms / args.steps,
                "prox_markers_ms_per_step": (fms - t_max) / args.steps,
                "taxels_with_proximity_reading": round(prox_share, 4),
                "sensor_kernel_threads": shapes2,
                "gpu_launches": (launches_per_step + 2) * args.steps}
    # third line: the point-cloud ProximityTaxel (the paper's experiment settings) on the same workload
    pcl = None
    if not args.no_pc_prox:
        import dataclasses
        rngc = np.random.default_rng(20260099)
        objs_c = [dataclasses.replace(objs[k], cloud=W.object_cloud(rngc, wl.objects[k], args.pc_points))
                  for k in range(len(objs))]
        pcp = dict(wl.params, pc_radius=0.01, pc_k=300.0, pc_ks=10.0, pc_density=100.0)
        sc3 = tg.Scene(wl.geom(), pcp, sensors=tg.TG_SENSOR_PCPROX, taxel_gid0=gid0, env_gid0=egid0)
        sc3.upload_objects(objs_c)
        shapes3, _ = tune_sensor_shapes(sc3, step_inputs(0, d_in), sched)
        sc3.graph_capture(step_inputs(0, d_in), pose_dt_per_step=dt)
        warm_then_rewind(sc3, args, dt)
        torch.cuda.synchronize()
        if pg:
            pg.barrier()
        c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        c0.record(stream)
        sc3.graph_launch(args.steps)
        c1.record(stream)
        torch.cuda.synchronize()
        cms = max_over_ranks(c0.elapsed_time(c1), dev)
        pcf = sc3.buffer(tg.CH_PC_FT).reshape(6, -1)
        pc_share = float((pcf[:3].abs().sum(0) > 0).sum().item()) / max(wl.n_active, 1)
        sc3.graph_release()
        sc3.close()
        pcl = {"sensors": f"headline step + point-cloud ProximityTaxel ({args.pc_points} tracked surface points per "
                          "object in a uniform cell grid, sensing radius 10 mm, k 300, ks 10, density 100)",
               "value": n_q * args.steps / (cms / 1e3), "unit": UNIT, "ms_per_step": cms / args.steps,
               "pc_prox_ms_per_step": (cms - t_max) / args.steps,
               "taxels_with_reading": round(pc_share, 4),
               "sensor_kernel_threads": shapes3,
               "gpu_launches": (launches_per_step + 1) * args.steps}
    # fourth line: elastomer markers with shear anchors (the paper's experiment settings)
    shear = None
    if not args.no_shear:
        import dataclasses
        rngs = np.random.default_rng(20260098)
        objs_s = [dataclasses.replace(objs[k], cloud=W.object_cloud(rngs, wl.objects[k], args.shear_points))
                  for k in range(len(objs))]
        pads_s = dict(W.add_pads(wl).pads, shear_points=args.shear_points, s_s=100.0, lambda_s=2000.0,
                      eta_enter=1e-5, eta_exit=1e-4, thickness=2e-3)
        sc4 = tg.Scene(wl.geom(), wl.params, sensors=tg.TG_SENSOR_MARKERS, taxel_gid0=gid0, env_gid0=egid0,
                       pads=pads_s)
        sc4.upload_objects(objs_s)
        shapes4, _ = tune_sensor_shapes(sc4, step_inputs(0, d_in), sched)
        sc4.graph_capture(step_inputs(0, d_in), pose_dt_per_step=dt)
        warm_then_rewind(sc4, args, dt)
        torch.cuda.synchronize()
        if pg:
            pg.barrier()
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        sc4.graph_launch(args.steps)
        s1.record(stream)
        torch.cuda.synchronize()
        sms = max_over_ranks(s0.elapsed_time(s1), dev)
        n_anch = int(sc4.buffer(tg.CH_SHEAR_ANCHORS).sum().item())
        n_pads = wl.n_envs * pads_s["pads_per_env"]
        sc4.graph_release()
        sc4.close()
        shear = {"sensors": f"headline step + elastomer markers (5 pads x 16x16 per env, dilation 5x5) with shear "
                            f"anchors ({args.shear_points} tracked surface points per object, s_s 100, lambda_s 2000, "
                            "eta_enter 1e-5 m, eta_exit 1e-4 m, 2 mm elastomer)",
                 "value": n_q * args.steps / (sms / 1e3), "unit": UNIT, "ms_per_step": sms / args.steps,
                 "markers_shear_ms_per_step": (sms - t_max) / args.steps,
                 "anchored_points_per_pad": round(n_anch / max(n_pads, 1), 2),
                 "sensor_kernel_threads": shapes4,
                 "anchor_state_bytes": n_pads * args.shear_points * 8,
                 "gpu_launches": (launches_per_step + 1) * args.steps}
    delay = None
    if not args.no_read_delay:
        delay = read_delay_line(args, wl, objs, dev, stream, sched, peaks)
    cfg2 = None
    if not args.no_config2:
        cfg2 = config2_line(args, dev, stream, pg, peaks)
    ray = ray_step = None
    if not args.no_raycast and ws == 1:
        ray = raycast_line(args, wl, wl.objects, dev, stream)  # the meshes behind the baked grids
        ray_step = raycast_step_line(args, wl, dev, stream, sched, step_ms / max(nsteps, 1), launches_per_step)
    temp = None
    if not args.no_temperature:
        temp = temperature_line(args, dev, stream, pg, peaks)
    neural = None
    if args.neural_objects > 0 and ws == 1:
        neural = neural_line(args, dev, stream, step_inputs)
    cfg4 = None
    if not args.no_config4 and ws == 1:
        cfg4 = config4_line(args, dev, stream)
    del objs

    peak, peak_kind = peaks()
    bpq = BYTES_PER_QUERY
    step_avg_ms = step_ms / max(nsteps, 1)
    achieved = bpq * wl.n_active / (step_avg_ms / 1e3) / 1e9
    traffic = traffic_from_profile()
    roofline = {
        "bound": "hbm", "kernel": "step_kernel", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
        "frac": round(achieved / peak, 4), "peak_kind": peak_kind, "traffic": traffic,
        "algorithmic_bytes_per_query": bpq,
        "step_kernel_ms": round(step_avg_ms, 4), "prologue_kernels_ms": round(pose_ms / max(nsteps, 1), 4),
        "step_kernel_share": round(step_ms / max(step_ms + pose_ms, 1e-9), 4),
    }
    clocks = clk.summary()

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = oracle_baseline(args, wl)

    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": t_max / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic", "config": workload_config(args, wl), "clocks": clocks,
            "e2e": e2e, "e2e_per_taxel": e2e_taxel, "gpu_launches": launches_per_step * args.steps,
            "roofline": roofline, "cpu_baseline": cpu,
            "penetrating_share": {"step_0": round(pen_share0, 4), f"step_{args.steps - 1}": round(pen_share_last, 4),
                                  "placement": wl.meta.get("placement")},
            "contact_share": {"step_0": round(contact_share0, 4),
                              f"step_{args.steps - 1}": round(contact_share_last, 4)},
            "schedule": {"chosen": sched, "autotune": tune["candidates"], "replay": "CUDA graph per step"},
            "full_sensor_set": full,
            "config2": cfg2,
            "read_delay": delay,
            "point_cloud_proximity": pcl,
            "elastomer_shear": shear,
            "temperature_grid": temp,
            "raycast_depth": ray,
            "raycast_step": ray_step,
            "neural_sdf": neural,
            "config4": cfg4,
            "setup_s": {"bake": round(bake_s, 2), "total": round(time.time() - t_setup, 1)},
        }
        print(json.dumps(out))
    scene.close()
    if pg:
        pg.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_tg(args)


if __name__ == "__main__":
    main()
