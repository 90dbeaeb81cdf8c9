#!/usr/bin/env python3
"""Benchmark: million site updates per second (MSUPS) of the fused sparse
LBGK collide-and-stream on one GB300, with its HBM roofline fraction.

Workload (default): the seeded six-generation bifurcating vessel tree with
every length x1.86 (root radius 89.28, Murray's law, 2048^3 box, 69,461,776
fluid sites; the at-scale tree of ~80M sites), D3Q19 LBGK, tau = 0.6, one
inlet at rho 1.001 and 32 outlets at rho 1.0, synthetic data.  ``--workload
vessel_tree`` runs the same tree at its stated root radius 48 in 1024^3
(10,787,566 sites).  One benchmark step = 100 lattice-Boltzmann time steps
(fused collide-and-stream kernels, AA-pattern streaming in place by default,
sites kept in (z, y, x) row order, ``--site-order``) + density/velocity/wall-
shear-stress fields + the float64 mass reduction.  value = fluid sites x LB
time steps / device time, fp32 storage; the fp16-deviation storage form and
the pull streaming form are reported beside it.  The inputs (~13 GB touched
per LB step) are far larger than the 126 MB L2, so no flush is needed.

``--impl reference`` times the FP64 CPU oracle on this machine's host cores
on the same workload and metric (a few LB steps per benchmark step).
"""
from __future__ import annotations

import argparse
import hashlib
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

from paper_1906_11925_gb300 import geometry as G  # noqa: E402
from paper_1906_11925_gb300 import metrics  # noqa: E402
from paper_1906_11925_gb300 import replicas  # noqa: E402

LB_STEPS_PER_BENCH_STEP = 100
# committed ncu summaries of the step kernels, per (workload, streaming form):
# the DRAM traffic per launch that the roofline object reports
PROFILE_SUMMARY = {
    ("vessel_tree_large", "aa"): os.path.join(ROOT, "profiles", "k_step_aa_q19_vessel_tree_large.md"),
    ("vessel_tree_large", "pull"): os.path.join(ROOT, "profiles", "k_step_pull_q19_vessel_tree_large.md"),
}
# the step kernels' sources: the summaries' hash is over these files' bytes in this order
KERNEL_SOURCES = [os.path.join(ROOT, "paper_1906_11925_gb300", "csrc", f)
                  for f in ("lbm_step.cu", "staging.cuh")]


def kernel_source_sha256() -> str:
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(f, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()
# the metric both arms report
METRIC = "MSUPS (million fluid-site updates per second), fused LBGK collide-and-stream"
FALLBACK_HBM_GBS = 6800.0
NOMINAL_HBM_GBS = 7900.0  # HBM3e data-sheet figure, for context beside the measured peak

WORKLOADS = {
    "vessel_tree": dict(q=19, tau=0.6, desc="seeded 6-generation bifurcating vessel tree, "
                        "root r=48, Murray exponent 3, asymmetry U(0.7,1), angles U(25,45) deg, "
                        "branch length 5.5 r, 1024^3 box, 1 inlet rho=1.001 + 32 outlets rho=1.0"),
    "vessel_tree_large": dict(q=19, tau=0.6, desc="the same seeded vessel tree with every length "
                              "x1.86 (root r=89.28, branch length 5.5 r), 2048^3 box, ~69.5M fluid "
                              "sites, 1 inlet rho=1.001 + 32 outlets rho=1.0"),
    "aneurysm": dict(q=15, tau=0.55, desc="quarter-arc tube r=20 on R=150 with fused sphere "
                     "r=40, 256^3 box, pulsatile inlet 1+0.001 sin(2 pi t/4000), outlet 1.0"),
    "tube": dict(q=15, tau=0.8, desc="straight tube r=8, 17x17x64, rho 1.001 -> 0.999"),
}


# --site-order: the binding's constant and a description
SITE_ORDERS = {"rows": ("ORDER_ROWS", "(z, y, x) row order"),
               "runs": ("ORDER_MORTON_RUNS", "Morton curve of 32-site runs along x"),
               "morton": ("ORDER_MORTON", "Morton (Z-order) curve of (x, y, z)")}

RENDER_SPINUP = 2000
I16_SCALE_LOG2 = 24  # int16 leg: step 2^-24, range |d| < 1.95e-3


def render_view(V, tf_scale: float):
    """The benchmark's view of a volume: 1920 x 1080, orbiting eye at 1.6x the
    largest extent, texture filter, default transfer function."""
    from paper_1906_11925_gb300 import lbm

    dims = np.array(V.shape[::-1], np.float64)
    return lbm.View.orbit((dims - 1) / 2.0, 1.6 * dims.max(), 0.6, 0.25, 1920, 1080, fov_y=0.75,
                          dt=0.5, tf_scale=tf_scale, lut=lbm.default_lut(0.3), a_stop=0.99)


def make_geometry(name: str):
    cache = os.path.join(tempfile.gettempdir(), "hemelb_gb300_geom_%s.npz" % name)
    if os.path.exists(cache):
        z = np.load(cache)
        meta = json.loads(str(z["meta"])) if "meta" in z.files else {}
        return G.Geometry(name=str(z["name"]), xyz=z["xyz"], io_xyz=z["io_xyz"], io_id=z["io_id"],
                          periodic=z["periodic"], rho_mean=z["rho_mean"], amp=z["amp"],
                          period=z["period"], phase=z["phase"], meta=meta)
    g = {"vessel_tree": G.vessel_tree, "aneurysm": G.aneurysm, "tube": G.tube,
         "vessel_tree_large": lambda: G.vessel_tree(root_r=48.0 * 1.86, box=2048)}[name]()
    try:
        np.savez(cache + ".tmp.npz", name=g.name, xyz=g.xyz, io_xyz=g.io_xyz, io_id=g.io_id,
                 periodic=g.periodic, rho_mean=g.rho_mean, amp=g.amp, period=g.period,
                 phase=g.phase, meta=json.dumps({"shape": g.meta.get("shape")}))
        os.replace(cache + ".tmp.npz", cache)
    except OSError:
        pass
    return g


def wall_fractions_cached(g, q: int, link):
    """Wall fractions of the geometry's analytic shape (G.wall_fractions),
    cached beside the geometry (only the wall links are stored)."""
    from paper_1906_11925_gb300 import lbm

    cache = os.path.join(tempfile.gettempdir(), "hemelb_gb300_wallq_%s_q%d.npz" % (g.name, q))
    if os.path.exists(cache):
        z = np.load(cache)
        wq = np.full((q, g.n), 0.5)
        wq.reshape(-1)[z["idx"]] = z["val"]
        return wq
    wq = G.wall_fractions(g, lbm.lattice_vectors(q), link)
    idx = np.flatnonzero((np.asarray(link) == 1).reshape(-1))
    try:
        np.savez(cache + ".tmp.npz", idx=idx, val=wq.reshape(-1)[idx])
        os.replace(cache + ".tmp.npz", cache)
    except OSError:
        pass
    return wq


dist_env = replicas.rank_env


def read_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def recorded_traffic(summary):
    """DRAM bytes per launch of the step kernel from a committed ncu summary,
    or None when it is missing or was taken on a different kernel source."""
    try:
        src = kernel_source_sha256()
        fields = {}
        for line in open(summary):
            if ":" in line and line.startswith("- "):
                k, v = line[2:].split(":", 1)
                fields[k.strip()] = v.strip().strip("`")
        if fields.get("kernel_source_sha256") != src:
            return None
        return {k: float(fields[k]) for k in ("traffic_bytes_per_launch_fp32",
                                               "traffic_bytes_per_launch_fp16") if k in fields}
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi clock and throttle-reason samples during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.out = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.out, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.out.close()
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = max(mx, float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def run_ours(args):
    import torch
    import torch.distributed as dist
    from paper_1906_11925_gb300 import lbm

    rank, local_rank, world = dist_env()
    torch.cuda.set_device(local_rank)
    if world > 1:
        dist.init_process_group("nccl")
    W = WORKLOADS[args.workload]
    q, tau = W["q"], W["tau"]
    g = make_geometry(args.workload)
    nbr, link = lbm.links_build(q, g.xyz, g.io_xyz, g.io_id, g.periodic)
    stream = torch.cuda.Stream()
    inner = args.inner
    legs = set(args.legs.split(","))

    def barrier():
        replicas.barrier(world)
        torch.cuda.synchronize()

    def max_over_ranks(v):
        return replicas.max_over_ranks(v, world, device="cuda")

    main_form = args.streaming
    alt_form = "pull" if main_form == "aa" else "aa"
    # the order the device keeps the sites in (every order gives the same
    # results to the bit; on the 69.5M-site tree the (z, y, x) row order makes
    # the odd AA step's scattered accesses faster than the Morton curve of
    # 32-site runs: 1,903 / 1,318 us per fp32 / fp16 step against 1,948 / 1,438)
    main_order = getattr(lbm, SITE_ORDERS[args.site_order][0])
    stream_id = {"pull": lbm.STREAM_PULL, "aa": lbm.STREAM_AA}

    def device_leg(storage, sampler=None, streaming=lbm.STREAM_PULL, wall_q=None,
                   site_order=None, scale_log2=None):
        site_order = main_order if site_order is None else site_order
        L = lbm.Lattice(q, g.xyz, nbr, link, tau, storage=storage, rho_mean=g.rho_mean,
                        amp=g.amp, period=g.period, phase=g.phase, stream=stream,
                        streaming=streaming, wall_q=wall_q, site_order=site_order,
                        fp16_scale_log2=scale_log2)
        rho = torch.empty(g.n, dtype=torch.float32, device="cuda")
        u = torch.empty(g.n, 3, dtype=torch.float32, device="cuda")
        wss = torch.empty(g.n, dtype=torch.float32, device="cuda")
        mass_dev = []

        def bench_step(ev=None):
            if ev is not None:
                ev[0].record(stream)
            L.step(inner)
            if ev is not None:
                ev[1].record(stream)
            L.macros(rho, u, wss)
            mass_dev.append(L.mass())

        for _ in range(args.warmup):
            bench_step()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        if sampler:
            sampler.start()
        t0.record(stream)
        for k in range(args.steps):
            bench_step(evs[k])
        t1.record(stream)
        torch.cuda.synchronize()
        barrier()
        clocks = sampler.stop() if sampler else None
        total_ms = max_over_ranks(t0.elapsed_time(t1))
        step_kernel_ms = sum(a.elapsed_time(b) for a, b in evs)
        finite = all(math.isfinite(m) for m in mass_dev)
        chunks = L.slab_chunks()
        L.close()
        return dict(total_ms=total_ms, step_kernel_ms=step_kernel_ms, clocks=clocks, finite=finite,
                    mass_last=mass_dev[-1] if mass_dev else None, chunks=chunks)

    def e2e_leg():
        # the user's call path with host buffers: per benchmark step, the inlet
        # and outlet densities of its LB steps go host -> device from pinned
        # memory, and the resulting total mass comes back device -> host.
        L = lbm.Lattice(q, g.xyz, nbr, link, tau, storage=lbm.STORE_FP32, rho_mean=g.rho_mean,
                        amp=g.amp, period=g.period, phase=g.phase, stream=stream,
                        streaming=stream_id[main_form], site_order=main_order)
        K = g.n_iolets
        rows = []
        for s in range(args.warmup + args.steps):
            t = np.arange(s * inner, (s + 1) * inner, dtype=np.float64)[:, None]
            r = g.rho_mean[None, :] + np.where(g.period > 0, g.amp, 0.0)[None, :] * np.sin(
                2 * np.pi * t / np.where(g.period > 0, g.period, 1.0)[None, :] + g.phase[None, :])
            rows.append(torch.from_numpy(np.ascontiguousarray(r)).pin_memory())
        for s in range(args.warmup):
            L.step_driven(rows[s], mass=False)
            L.mass()
        barrier()
        t0 = time.perf_counter()
        for s in range(args.warmup, args.warmup + args.steps):
            L.step_driven(rows[s], mass=False)
            L.mass()
        barrier()
        dt = max_over_ranks(time.perf_counter() - t0)
        L.close()
        return dict(seconds=dt, h2d=inner * K * 8, d2h=8)

    def adjoint_leg():
        # gradient of the inlet-to-outlet pressure drop, averaged over every
        # state of the run, with respect to tau and the mean density of all 33
        # iolets: fp16-deviation forward, float32 adjoint, float64 accumulation,
        # binomial checkpointing with as many snapshots as fit in 150 GB
        L = lbm.Lattice(q, g.xyz, nbr, link, tau, storage=lbm.STORE_FP16, rho_mean=g.rho_mean,
                        amp=g.amp, period=g.period, phase=g.phase, stream=stream,
                        streaming=stream_id[main_form], site_order=main_order)
        nsteps = args.adjoint_steps
        inlet = (link == 2).any(axis=0)
        outlet = (link >= 3).any(axis=0)
        weight = np.where(inlet, 1.0 / (3.0 * max(inlet.sum(), 1)), 0.0) - np.where(
            outlet, 1.0 / (3.0 * max(outlet.sum(), 1)), 0.0)
        state_bytes = L.state_bytes()
        n_snap = int(max(2, min(nsteps + 1, (150 << 30) // state_bytes - 1)))
        if args.adjoint_snapshots:
            n_snap = args.adjoint_snapshots
        t0 = L.time
        L.objective_grad(lbm.OBJ_DENSITY, weight, 20, t0, t0 + 21, n_snap=min(n_snap, 21))  # warm-up
        t0 = L.time
        torch.cuda.synchronize()
        w0 = time.perf_counter()
        r = L.objective_grad(lbm.OBJ_DENSITY, weight, nsteps, t0, t0 + nsteps + 1,
                             scale=1.0 / (nsteps + 1), n_snap=n_snap)
        wall = time.perf_counter() - w0
        fw, ad = L.adjoint_counts()
        sweep = L.adjoint_sweep_ms()
        # forward step time of this context, for the adjoint/forward ratio
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        L.step(100)
        b.record(stream)
        torch.cuda.synchronize()
        fwd_ms = a.elapsed_time(b) / 100
        L.close()
        adj_ms = (sweep - fw * fwd_ms) / ad
        return {"objective": "pressure drop, inlet-adjacent minus outlet-adjacent mean c_s^2 rho, "
                             "averaged over all states",
                "storage": "fp16 forward, fp32 adjoint, fp64 accumulation", "streaming": main_form,
                "steps": nsteps,
                "snapshots": n_snap, "snapshot_gb": round(n_snap * state_bytes / 2 ** 30, 1),
                "forward_steps": fw, "adjoint_steps": ad, "sweep_ms": round(sweep, 2),
                "wall_s": round(wall, 3), "fwd_step_ms": round(fwd_ms, 4),
                "adjoint_step_ms": round(adj_ms, 4),
                "adjoint_step_vs_fwd": round(adj_ms / fwd_ms, 3),
                "gradient_vs_forward_run": round(sweep / (nsteps * fwd_ms), 3),
                "J": r["J"], "dJ_dtau": r["dtau"], "n_gradients": 1 + len(r["dmean"]),
                "finite": bool(np.isfinite(r["dtau"]) and np.all(np.isfinite(r["dmean"])))}

    def render_leg():
        # visualisation (Section 3.3.2): after RENDER_SPINUP LB steps, every
        # frame writes the speed |u| of all sites into the 3D texture and
        # ray-marches a 1920 x 1080 image of it
        L = lbm.Lattice(q, g.xyz, nbr, link, tau, storage=lbm.STORE_FP32, rho_mean=g.rho_mean,
                        amp=g.amp, period=g.period, phase=g.phase, stream=stream)
        L.step(args.render_spinup)
        _, u, _ = L.macros(want=("u",))
        umax = float(torch.linalg.vector_norm(u, dim=1).max())
        V = lbm.Volume.for_lattice(L)
        view = render_view(V, 1.0 / umax)  # noqa: F821 (module level)
        img = torch.empty(view.height, view.width, 4, dtype=torch.float32, device="cuda")
        for _ in range(args.warmup):
            V.from_lattice(L, lbm.QTY_SPEED)
            V.render(view, img, stream)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        fill_ms = render_ms = 0.0
        for _ in range(args.steps):
            ev[0].record(stream)
            V.from_lattice(L, lbm.QTY_SPEED)
            ev[1].record(stream)
            V.render(view, img, stream)
            ev[2].record(stream)
            torch.cuda.synchronize()
            fill_ms += ev[0].elapsed_time(ev[1])
            render_ms += ev[1].elapsed_time(ev[2])
        alpha = img[..., 3]
        # one more frame with the kernel's sample counters (not timed)
        cnt = torch.zeros(2, dtype=torch.int64, device="cuda")
        view.counters = cnt
        V.render(view, img, stream)
        torch.cuda.synchronize()
        samples, jumps = [int(x) for x in cnt.cpu()]
        out = {"quantity": "speed |u|", "spinup_lb_steps": args.render_spinup,
               "volume_voxels": list(V.shape[::-1]), "image": [view.width, view.height],
               "filter": "texture trilinear", "dt": view.dt, "a_stop": view.a_stop,
               "empty_skipping": "8^3 bricks",
               "fill_ms": round(fill_ms / args.steps, 4), "render_ms": round(render_ms / args.steps, 4),
               "frames_per_s": round(1e3 * args.steps / (fill_ms + render_ms), 1),
               "mrays_per_s": round(view.width * view.height * args.steps / render_ms / 1e3, 1),
               "samples_per_frame": samples, "brick_jumps_per_frame": jumps,
               "gsamples_per_s": round(samples * args.steps / render_ms / 1e6, 2),
               "covered_pixels": round(float((alpha > 0.01).float().mean()), 4),
               "fill_gbs": round(metrics.volume_fill_bytes(q, g.n) * args.steps / fill_ms / 1e6, 1)}
        V.close()
        L.close()
        return out

    sampler = ClockSampler(local_rank) if rank == 0 else None
    r32 = device_leg(lbm.STORE_FP32, sampler, streaming=stream_id[main_form])
    r16 = device_leg(lbm.STORE_FP16, streaming=stream_id[main_form]) if "fp16" in legs else None
    # int16 fixed point at the scale 2^-24 (deviations of these flows stay below 1e-3)
    ri16 = device_leg(lbm.STORE_I16, streaming=stream_id[main_form], scale_log2=I16_SCALE_LOG2) \
        if "i16" in legs else None
    # the other streaming form, for comparison
    alt = alt_form in legs
    raa32 = device_leg(lbm.STORE_FP32, streaming=stream_id[alt_form]) if alt else None
    raa16 = device_leg(lbm.STORE_FP16, streaming=stream_id[alt_form]) if alt else None
    # AA step pairs fused over slab chunks of whole z planes (the odd step
    # reads the even step's output back from L2), beside the unfused AA step
    slabs = "slabs" in legs and main_form == "aa"
    rsl32 = device_leg(lbm.STORE_FP32, streaming=lbm.STREAM_AA, site_order=lbm.ORDER_SLABS) if slabs else None
    rsl16 = device_leg(lbm.STORE_FP16, streaming=lbm.STREAM_AA, site_order=lbm.ORDER_SLABS) if slabs else None
    e2e = e2e_leg() if "e2e" in legs else None
    adj = adjoint_leg() if "adjoint" in legs else None
    rnd = render_leg() if "render" in legs else None
    if "bfl" in legs:
        # interpolated walls at the analytic wall positions of the tree
        wq = wall_fractions_cached(g, q, link)
        # (pull streaming; the plain Morton order measured faster with these walls)
        rbfl32 = device_leg(lbm.STORE_FP32, wall_q=wq, site_order=lbm.ORDER_MORTON)
        rbfl16 = device_leg(lbm.STORE_FP16, wall_q=wq, site_order=lbm.ORDER_MORTON)
        n_bfl_sites = int(((np.asarray(link) == 1) & (wq != 0.5)).any(axis=0).sum())
    else:
        rbfl32 = rbfl16 = None

    n_lb = args.steps * inner
    value = world * metrics.msups(g.n, n_lb, r32["total_ms"] / 1e3)
    peak, peak_kind = read_peaks()

    def roofline(res, storage, streaming="pull"):
        bps = metrics.bytes_per_site_update(q, storage, streaming)
        per_launch_s = res["step_kernel_ms"] / 1e3 / n_lb
        achieved = bps * g.n / per_launch_s / 1e9
        return dict(bound="hbm", achieved=round(achieved, 1), peak=peak, unit="GB/s",
                    frac=round(achieved / peak, 4), peak_source=peak_kind,
                    frac_of_nominal=round(achieved / NOMINAL_HBM_GBS, 4),
                    nominal_peak=NOMINAL_HBM_GBS,
                    bytes_per_site_update=bps, launch_us=round(per_launch_s * 1e6, 2))

    summary = PROFILE_SUMMARY.get((args.workload, main_form))
    traffic = recorded_traffic(summary) if summary else None
    rf32 = roofline(r32, "fp32", main_form)
    rf32["traffic"] = traffic.get("traffic_bytes_per_launch_fp32") if traffic else None
    if r16:
        rf16 = roofline(r16, "fp16", main_form)
        rf16["traffic"] = traffic.get("traffic_bytes_per_launch_fp16") if traffic else None
    forms = {"pull": "pull: gather through the neighbour table from one buffer into another",
             "aa": "AA pattern: one buffer updated in place, even steps on a site's own slots, "
                   "odd steps through the neighbour table"}

    # resident fp32 state of the main form (populations and table) against the L2 size
    resident = g.n * (q * 4 * (1 if main_form == "aa" else 2) + 4 * (q - 1))
    l2_bytes = torch.cuda.get_device_properties(local_rank).L2_cache_size
    l2_note = ("inputs larger than L2 (no flush)" if resident > l2_bytes else
               "working set (%.0f MB) fits in the %.0f MB L2: an L2-resident parity-size workload, "
               "not an HBM roofline case" % (resident / 1e6, l2_bytes / 1e6))
    out = {
        "metric": METRIC,
        "value": round(value, 2),
        "unit": "MSUPS",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(r32["total_ms"] / args.steps, 4),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic (seeded vessel geometry, fluid initialised at rest)",
        "config": {"workload": args.workload, "description": W["desc"], "lattice": "D3Q%d" % q,
                   "tau": tau, "fluid_sites": g.n, "iolets": g.n_iolets, "storage": "fp32",
                   "streaming": forms[main_form],
                   "site_order": SITE_ORDERS[args.site_order][1],
                   "lb_steps_per_bench_step": inner,
                   "bench_step": "%d fused collide-stream steps + rho/u/WSS fields + fp64 mass"
                                 % inner,
                   "l2": l2_note,
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "roofline": rf32,
        "paper_context": {"value": 15.17, "unit": "MSUPS",
                          "hardware": "Exxact TWS: Intel i7-5960X + 4x GeForce GTX 1080 Ti",
                          "workload": "patient aneurysm, 296,814 sites, D3Q19 (Table III)",
                          "note": "another machine and workload: context, not the target"},
        "fp16": None if not r16 else {
            "value": round(world * metrics.msups(g.n, n_lb, r16["total_ms"] / 1e3), 2),
            "unit": "MSUPS", "ms_per_step": round(r16["total_ms"] / args.steps, 4),
            "roofline": rf16, "speedup_vs_fp32": round(r32["total_ms"] / r16["total_ms"], 3)},
        "i16": None if not ri16 else {
            "storage": "int16 fixed-point deviations round(d 2^%d)" % I16_SCALE_LOG2,
            "value": round(world * metrics.msups(g.n, n_lb, ri16["total_ms"] / 1e3), 2),
            "unit": "MSUPS", "ms_per_step": round(ri16["total_ms"] / args.steps, 4),
            "roofline": roofline(ri16, "fp16", main_form),
            "speedup_vs_fp32": round(r32["total_ms"] / ri16["total_ms"], 3)},
        "e2e": None if not e2e else {
            "value": round(world * metrics.msups(g.n, n_lb, e2e["seconds"]), 2),
            "unit": "MSUPS", "h2d_bytes_per_step": e2e["h2d"], "d2h_bytes_per_step": e2e["d2h"],
            "path": "lbm_step_driven (host iolet densities, pinned) + lbm_mass (host)"},
        alt_form: None if not raa32 else {
            "streaming": forms[alt_form],
            "fp32": {"value": round(world * metrics.msups(g.n, n_lb, raa32["total_ms"] / 1e3), 2),
                     "unit": "MSUPS", "ms_per_step": round(raa32["total_ms"] / args.steps, 4),
                     "roofline": roofline(raa32, "fp32", alt_form)},
            "fp16": {"value": round(world * metrics.msups(g.n, n_lb, raa16["total_ms"] / 1e3), 2),
                     "unit": "MSUPS", "ms_per_step": round(raa16["total_ms"] / args.steps, 4),
                     "roofline": roofline(raa16, "fp16", alt_form)}},
        "slabs": None if not rsl32 else {
            "streaming": "AA step pairs fused over slab chunks of whole z planes (row order): one "
                         "persistent launch per even+odd pair, the odd step of a chunk reading the "
                         "even step's output back from L2",
            "chunks": {"fp32": rsl32["chunks"], "fp16": rsl16["chunks"]},
            "fp32": {"value": round(world * metrics.msups(g.n, n_lb, rsl32["total_ms"] / 1e3), 2),
                     "unit": "MSUPS", "ms_per_step": round(rsl32["total_ms"] / args.steps, 4),
                     "launch_us": round(rsl32["step_kernel_ms"] * 1e3 / n_lb, 2),
                     "speedup_vs_unfused": round(r32["total_ms"] / rsl32["total_ms"], 3)},
            "fp16": {"value": round(world * metrics.msups(g.n, n_lb, rsl16["total_ms"] / 1e3), 2),
                     "unit": "MSUPS", "ms_per_step": round(rsl16["total_ms"] / args.steps, 4),
                     "launch_us": round(rsl16["step_kernel_ms"] * 1e3 / n_lb, 2),
                     "speedup_vs_unfused": None if not r16 else round(r16["total_ms"] / rsl16["total_ms"], 3)}},
        "adjoint": adj,
        "render": rnd,
        "bfl": None if not rbfl32 else {
            "walls": "Bouzidi-Firdaouss-Lallemand interpolation at the analytic wall positions",
            "sites_with_interpolated_links": n_bfl_sites,
            "fp32": {"value": round(world * metrics.msups(g.n, n_lb, rbfl32["total_ms"] / 1e3), 2),
                     "unit": "MSUPS", "ms_per_step": round(rbfl32["total_ms"] / args.steps, 4),
                     "roofline": roofline(rbfl32, "fp32")},
            "fp16": {"value": round(world * metrics.msups(g.n, n_lb, rbfl16["total_ms"] / 1e3), 2),
                     "unit": "MSUPS", "ms_per_step": round(rbfl16["total_ms"] / args.steps, 4),
                     "roofline": roofline(rbfl16, "fp16")}},
        # per benchmark step: inner x (bulk-site launch + iolet-site launch),
        # the fields, and the two mass kernels
        "gpu_launches": args.steps * (inner * (2 if g.n_iolets else 1) + 1 + 2),
        "clocks": r32["clocks"],
        "finite": all(r is None or r["finite"] for r in (r32, r16, ri16, raa32, raa16, rbfl32, rbfl16, rsl32,
                                                          rsl16)),
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(args.workload, g, nbr, link, q, tau,
                                           budget_s=args.cpu_budget)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()


def cpu_baseline(workload, g, nbr, link, q, tau, budget_s=15.0, lb_steps=None):
    """The FP64 oracle as it stands, on this machine's host cores, on the same
    geometry; about budget_s seconds of CPU work."""
    import oracle
    f = oracle.rest_state(q, g.n)
    t0 = time.perf_counter()
    f = oracle.step(q, nbr, link, tau, f, t=0, geom=g)
    one = time.perf_counter() - t0
    n = lb_steps or max(1, int(budget_s / max(one, 1e-6)))
    t0 = time.perf_counter()
    oracle.run(q, nbr, link, tau, f, n, t0=1, geom=g)
    dt = time.perf_counter() - t0
    out = {"value": round(metrics.msups(g.n, n, dt), 3), "unit": "MSUPS",
           "cores": oracle.num_threads(), "kind": "oracle",
           "sample": "%d LB steps of the full %s workload (%d sites), float64, push form"
                     % (n, workload, g.n)}
    if lb_steps is None:
        # the same on one core, about 2 s of LB steps (at least one)
        nt = oracle.num_threads()
        n1 = max(1, int(2.0 / max(one * nt, 1e-6)))
        oracle.set_threads(1)
        try:
            t0 = time.perf_counter()
            oracle.run(q, nbr, link, tau, f, n1, t0=1, geom=g)
            d1 = time.perf_counter() - t0
        finally:
            oracle.set_threads(nt)
        out["one_core"] = {"value": round(metrics.msups(g.n, n1, d1), 3), "unit": "MSUPS",
                           "sample": "%d LB step(s) of the same workload on 1 core" % n1}
    return out


def run_reference(args):
    rank, _, world = dist_env()
    if rank != 0:
        return
    import oracle
    W = WORKLOADS[args.workload]
    q, tau = W["q"], W["tau"]
    g = make_geometry(args.workload)
    nbr, link = oracle.links_build(q, g.xyz, g.io_xyz, g.io_id, g.periodic)
    o = oracle.default()
    # one state stepped in place (no per-call copy of the populations), as
    # cpu_baseline's single oracle.run call does
    f = o.rest_state(q, g.n)
    work = np.empty_like(f)
    per_step = 2  # LB steps per benchmark step on the CPU (a bounded sample)
    t = 0
    for _ in range(args.warmup):
        o.run_inplace(q, nbr, link, tau, f, work, per_step, t0=t, geom=g)
        t += per_step
    t0 = time.perf_counter()
    for _ in range(args.steps):
        o.run_inplace(q, nbr, link, tau, f, work, per_step, t0=t, geom=g)
        t += per_step
    dt = time.perf_counter() - t0
    v = metrics.msups(g.n, args.steps * per_step, dt)
    sample = "%d LB step(s) of the full %s workload (%d sites) per benchmark step, float64 oracle" % (
        per_step, args.workload, g.n)
    print(json.dumps({
        "impl": "reference",
        "metric": METRIC,
        "value": round(v, 3), "unit": "MSUPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(dt * 1e3 / args.steps, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded vessel geometry, fluid initialised at rest)",
        "config": {"workload": args.workload, "description": W["desc"], "lattice": "D3Q%d" % q,
                   "tau": tau, "fluid_sites": g.n, "iolets": g.n_iolets},
        "cpu_baseline": {"value": round(v, 3), "unit": "MSUPS", "cores": oracle.num_threads(),
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": round(v, 3), "unit": "MSUPS", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="vessel_tree_large")
    ap.add_argument("--inner", type=int, default=LB_STEPS_PER_BENCH_STEP,
                    help="LB time steps per benchmark step")
    ap.add_argument("--streaming", choices=("aa", "pull"), default="aa",
                    help="streaming form of the main legs (the other one is the comparison leg)")
    ap.add_argument("--legs", default="fp32,fp16,i16,pull,aa,slabs,e2e,adjoint,render,bfl",
                    help="comma list of fp32 (always run), fp16, i16, pull, aa (the comparison "
                         "leg of the form not chosen by --streaming), e2e, adjoint, render, bfl")
    ap.add_argument("--adjoint-steps", type=int, default=3000)
    ap.add_argument("--adjoint-snapshots", type=int, default=0,
                    help="snapshot count (default: as many as fit in 150 GB)")
    ap.add_argument("--render-spinup", type=int, default=RENDER_SPINUP,
                    help="LB steps before the render leg's frames")
    ap.add_argument("--site-order", choices=sorted(SITE_ORDERS), default="rows",
                    help="order the device keeps the sites in, for every leg but the interpolated-wall "
                         "and slab-chunk legs")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
