"""Benchmark: rays/s of GB300 inverse ray-shooting on the paper-shaped mid-size
workload (kappa_* = 0.45, kappa_s = 0, gamma = 0.45, 1e5 Salpeter lenses in
0.1-1 rescaled to kappa_*, 2000^2 map over 20 x 20 theta_E, 100 rays per
unlensed pixel: 1.12e10 rays per map).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--method interp|brute]
                  [--impl ours|reference]

One step = one magnification map through irs_make_map (INTERP: mass sum, cell
lists, far field, ray pass, binning, magnification).  The plain brute-force map of the
same workload costs ~1e15 pair terms (minutes), so it is timed on a band of
lattice rows through irs_make_map_rows and reported per ray, with the same
band made by the interpolated method as the accuracy check (per-pixel
magnification relative RMS over pixels with >= 100 rays).

Multi-GPU: maps are independent problems, so each rank makes its own map
(weak scaling, no collective on the data path); value = all ranks' rays / the
slowest rank's time.

--impl reference times the FP64 CPU oracle (the plain definition the GPU path
is checked against) on a bounded sample of the same workload on the host
cores.
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = dict(name="paper-mid: kappa*=0.45 kappa_s=0 gamma=0.45, 1e5 Salpeter lenses, "
                     "2000^2 px over 20x20 thetaE, 100 rays/px",
                kappa_star=0.45, kappa_s=0.0, gamma=0.45, S=20.0, npix=2000, nav=100.0,
                n_star=100000, shape="salpeter", seed=2)
# high resolution: 1e6 lenses, 1e8-pixel map (count map larger than L2)
WORKLOAD_HIGHRES = dict(name="high-res: kappa*=0.35 kappa_s=0.15 gamma=0.4, 1e6 uniform lenses 0.1-1, "
                             "10000^2 px over 25x25 thetaE, 40 rays/px",
                        kappa_star=0.35, kappa_s=0.15, gamma=0.4, S=25.0, npix=10000, nav=40.0,
                        n_star=1000000, shape="uniform", seed=3)
# the learned far field's workload
WORKLOAD_LEARNED = dict(name="learned: kappa*=0.4 kappa_s=0.1 gamma=0.35, 2e5 equal-mass lenses, "
                             "4000^2 px over 20x20 thetaE, 64 rays/px",
                        kappa_star=0.4, kappa_s=0.1, gamma=0.35, S=20.0, npix=4000, nav=64.0,
                        n_star=200000, shape="equal", seed=5)
BRUTE_ROWS = 256            # band of lattice rows for the brute-force timing
L2_FLUSH_BYTES = 512 << 20  # > 129 MB L2


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                                         text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        mhz, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                mhz.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        if not mhz:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": float(np.median(mhz)), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(mhz)}


def slowest_rank_ms(my_ms, dist, device):
    """Max over ranks of this rank's timed milliseconds (the job ends with the slowest)."""
    import torch
    t = torch.tensor([float(my_ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rays_per_s(rays_per_step_per_rank, world, ms_per_step):
    """Weak scaling: every rank makes its own map, so the job shoots world x the rays."""
    return rays_per_step_per_rank * world / (ms_per_step * 1e-3)


def dist_init():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def workload_params(irs, method, w=WORKLOAD):
    S = w["S"]
    m = {"interp": irs.IRS_INTERP, "brute": irs.IRS_BRUTE, "mlp": irs.IRS_MLP}[method]
    return irs.make_params(w["kappa_star"], w["kappa_s"], w["gamma"], (-S / 2, S / 2, -S / 2, S / 2),
                           w["npix"], w["nav"], n_star=w["n_star"], method=m)


def lens_field(lensgen, box, seed, w=WORKLOAD):
    area = (box[1] - box[0]) * (box[3] - box[2])
    return lensgen.lens_field(w["n_star"], box, shape=w["shape"], seed=seed,
                              total_mass=w["kappa_star"] * area / np.pi)


# ------------------------------------------------------------------ ours
# Per-ray work of the interpolated ray pass, in flops: 10 per near pair (the
# same pair arithmetic as the brute force), 8 per complex multiply-add of the
# level-2 Horner (K2 - 1 of them for K2 series terms), and 20 for the smooth
# terms, sub-cell index and pixel.
IP_VARIANT_K2 = [8, 6, 6, 6, 6, 6, 6, 6, 6, 8]  # series terms K2 of ray-pass variants 0..9
IP_FLOPS_OTHER = 20


def ip_flops_fixed(variant):
    return 8 * (IP_VARIANT_K2[variant] - 1) + IP_FLOPS_OTHER


# DRAM bytes per launch of the ray pass (ncu dram__bytes_read.sum +
# dram__bytes_write.sum), valid only for the kernel build, workload and cell
# size they were captured on: (workload, cell multiplier, variant) -> bytes.
# Source: profiles/k_ip_ray_paper-mid-full.md.
IP_TRAFFIC = {("paper-mid", 1.0, 7): 46.848768e6 + 11.264e3}


def mean_near_lenses(info, xy):
    """Mean over rays of the lenses in a ray's 3x3 block of level-1 cells."""
    h = info.cell_x
    ncx, ncy = info.ncell_x, info.ncell_y
    gx0 = info.lens_x0 - 0.0  # rectangular plane: grid origin = plane corner
    gy0 = info.lens_y0
    cx = np.clip(np.floor((xy[:, 0] - gx0) / h).astype(np.int64), 0, ncx - 1)
    cy = np.clip(np.floor((xy[:, 1] - gy0) / h).astype(np.int64), 0, ncy - 1)
    cnt = np.zeros((ncy + 2, ncx + 2))
    np.add.at(cnt, (cy + 1, cx + 1), 1.0)
    blk = sum(cnt[1 + dy:1 + dy + ncy, 1 + dx:1 + dx + ncx] for dy in (-1, 0, 1) for dx in (-1, 0, 1))
    k = info.rays_per_cell_x
    wx = np.full(ncx, k, dtype=np.float64)
    wx[-1] = info.n_rays_x - k * (ncx - 1)
    wy = np.full(ncy, k, dtype=np.float64)
    wy[-1] = info.n_rays_y - k * (ncy - 1)
    w = wy[:, None] * wx[None, :]
    return float((blk * w).sum() / w.sum())


def run_ours(args):
    import torch
    import torch.distributed as dist

    world, rank, local = dist_init()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_2204_10871_gb300 import build as libbuild
    libbuild.build()
    from paper_2204_10871_gb300 import irs, lensgen

    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    props = torch.cuda.get_device_properties(local)
    n_sms = props.multi_processor_count
    named = {"paper-mid": WORKLOAD, "high-res": WORKLOAD_HIGHRES, "learned": WORKLOAD_LEARNED}
    w = dict(named[args.workload] if args.workload else
             (WORKLOAD_LEARNED if args.method == "mlp" else WORKLOAD))
    if args.n_star:
        w["n_star"] = args.n_star
    if args.npix:
        w["npix"] = args.npix
    if args.nav:
        w["nav"] = args.nav
    full = args.method != "brute"

    params = workload_params(irs, args.method, w)
    probe = irs.Plan(params)  # the lens plane does not depend on the tuning
    box = (probe.info.lens_x0, probe.info.lens_x1, probe.info.lens_y0, probe.info.lens_y1)
    probe.close()
    xy, m = lens_field(lensgen, box, w["seed"] + 1000 * rank, w)
    dxy = torch.from_numpy(xy).to(dev)
    dm = torch.from_numpy(m).to(dev)
    tune = None
    if args.variant >= 0:
        params.kernel_variant = args.variant
    elif args.method == "interp" and not args.no_tune:  # untimed: pick cell size and ray-pass variant
        t0 = time.perf_counter()
        params, res = irs.irs_autotune(params, dxy, dm)
        tune = {"cell_mult": res.cell_mult, "kernel_variant": res.kernel_variant,
                "candidates": res.candidates, "est_ms_tuned": res.ms_per_map,
                "est_ms_default": res.ms_default, "from_cache": bool(res.from_cache),
                "tuning_s": time.perf_counter() - t0}
    plan = irs.Plan(params)
    info = plan.info
    learned = None
    if args.method == "mlp":  # untimed: train the network on this lens field
        rep = irs.irs_mlp_train(plan.handle, dxy, dm, seed=11)
        learned = {"samples": rep.samples, "steps": rep.steps, "loss_first": rep.loss_first,
                   "loss_final": rep.loss_final, "heldout_rel_rms": rep.valid_rel_rms,
                   "target_rms_thetaE": rep.target_rms, "ms_samples": rep.ms_samples,
                   "ms_train": rep.ms_train}
    shape = (w["npix"], w["npix"])
    counts = torch.zeros(shape, dtype=torch.uint32, device=dev)
    mag = torch.zeros(shape, dtype=torch.float32, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    irs.irs_plan_set_timing(plan.handle, True)
    band_rows = args.band_rows or BRUTE_ROWS
    r0 = (info.n_rays_y // 2 // 64) * 64  # whole brute tiles (64 rows)
    band = (r0, min(info.n_rays_y, r0 + band_rows))

    def step():
        if full:
            irs.irs_make_map(plan.handle, dxy, dm, counts, mag)
        else:
            counts.zero_()
            irs.irs_make_map_rows(plan.handle, dxy, dm, band[0], band[1], counts)

    rays_per_step = info.n_rays if full else (band[1] - band[0]) * info.n_rays_x
    for _ in range(args.warmup):
        step()
    plan.sync()

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    ray_ms, tot_ms, launches = [], [], 0
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        t_wall = time.perf_counter()
        for k in range(args.steps):
            flush.fill_(float(k))  # evict L2 between timed steps
            ev[k][0].record(stream)
            step()
            ev[k][1].record(stream)
            t = irs.irs_plan_timings(plan.handle)  # events of this map (syncs on them)
            ray_ms.append(t.ms_raypass)
            tot_ms.append(t.ms_total)
            launches += t.launches
        torch.cuda.synchronize()
        wall = time.perf_counter() - t_wall
    plan.sync()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    my_ms = float(np.sum(step_ms))
    if world > 1:
        my_ms = slowest_rank_ms(my_ms, dist, dev)
        dist.barrier()
    ms_per_step = my_ms / args.steps
    value = whole_job_rays_per_s(rays_per_step, world, ms_per_step)

    # ---- end to end through the public API with host buffers
    h_xy = torch.from_numpy(xy).pin_memory()
    h_m = torch.from_numpy(m).pin_memory()
    h_counts = torch.empty(shape, dtype=torch.uint32).pin_memory()
    e2e_steps = max(1, min(args.steps, 3))
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(e2e_steps):
        dxy.copy_(h_xy, non_blocking=True)
        dm.copy_(h_m, non_blocking=True)
        step()
        h_counts.copy_(counts, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1) / e2e_steps
    h2d = xy.nbytes + m.nbytes
    d2h = h_counts.numel() * 4
    clocks = clk.summary()

    # ---- roofline of the dominant kernel (the ray pass): FP32 ALU bound
    pk = peaks() or {}
    sm_max = float(pk.get("sm_max_mhz", 2070.0))
    peak_tflops = n_sms * 128 * 2 * sm_max * 1e6 / 1e12
    ray_ms_mean = float(np.mean(ray_ms))
    traffic = None
    if full:
        n_near = mean_near_lenses(info, xy)
        variant = int(params.kernel_variant)
        flops_per_ray = 10.0 * n_near + ip_flops_fixed(variant)
        kname = f"k_ip_ray variant {variant} (near pair sum + level-2 Horner, FP32 pipe + MUFU)"
        key = (w["name"].split(":")[0], round(float(params.cell_mult or 1.0), 2), variant)
        if key in IP_TRAFFIC:
            traffic = IP_TRAFFIC[key]
    else:
        n_near = None
        flops_per_ray = 10.0 * w["n_star"]
        kname = "k_brute (pair sum, FP32 pipe + MUFU)"
    achieved = flops_per_ray * rays_per_step / (ray_ms_mean * 1e-3) / 1e12
    roofline = {"bound": "alu", "kernel": kname, "achieved": achieved, "peak": peak_tflops,
                "unit": "TFLOP/s", "frac": achieved / peak_tflops, "traffic": traffic,
                "peak_basis": f"{n_sms} SMs x 128 FP32 lanes x 2 flop x {sm_max:.0f} MHz "
                              "(max SM clock of MEASURED_PEAKS.json)",
                "flops_per_ray": flops_per_ray}
    if n_near is not None:
        roofline["mean_near_lenses"] = n_near
    if clocks.get("sm_mhz"):
        roofline["frac_at_measured_clock"] = achieved / (n_sms * 256 * clocks["sm_mhz"] * 1e6 / 1e12)

    # ---- brute force on a band of the same lattice: rays/s and the accuracy judge
    brute = None
    if full and not args.no_brute and rank == 0:
        brute = brute_band(irs, torch, w, xy, m, dxy, dm, band, plan, n_sms, peak_tflops, value)
    if learned is not None and rank == 0:
        # the series form on the same workload, and its error on the same band
        pi = irs.Plan(workload_params(irs, "interp", w))
        irs.irs_plan_set_timing(pi.handle, True)
        ms = []
        for k in range(3):
            irs.irs_make_map(pi.handle, dxy, dm, counts, mag)
            t = irs.irs_plan_timings(pi.handle)
            if k:
                ms.append(t.ms_total)
        learned["interp_rays_per_s"] = info.n_rays / (float(np.mean(ms)) * 1e-3)
        if brute is not None:
            learned["interp_map_rel_rms_vs_brute"] = band_rel_rms(irs, torch, pi, dxy, dm, band, shape)
        pi.close()

    if rank == 0:
        cpu = cpu_baseline(xy, m, w) if (world == 1 and not args.no_cpu) else None
        line = {
            "metric": "rays/s per GB300 (" + args.method + ")",
            "value": value, "unit": "rays/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32 (pairs), f64 (far field, setup)",
            "data": "synthetic (seeded lens fields; the paper's lens catalogues are not public)",
            "config": {"workload": w["name"] if not (args.n_star or args.npix or args.nav)
                       else "reduced case for profiling", "method": args.method,
                       "rays_per_step": rays_per_step, "n_star": w["n_star"], "npix": w["npix"],
                       "rays_per_pixel": w["nav"],
                       "band_rows": None if full else [int(band[0]), int(band[1])],
                       "l2": "flushed between steps (512 MB write)",
                       "parallelism": f"replicas x{world}"},
            "e2e": {"value": rays_per_step / (e2e_ms * 1e-3), "unit": "rays/s",
                    "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
            "gpu_launches": int(launches),
            "autotune": tune,
            "learned": learned,
            "roofline": roofline,
            "clocks": clocks,
            "stage_ms": {"raypass_mean": ray_ms_mean, "map_total_mean": float(np.mean(tot_ms)),
                         "wall_s": wall},
            "brute": brute,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line))
    plan.close()
    if world > 1:
        dist.destroy_process_group()


BRUTE_BAND_MAP = {}


def band_rel_rms(irs, torch, plan, dxy, dm, band, shape):
    """Per-pixel magnification rel RMS of `plan` against the last brute band map."""
    a = BRUTE_BAND_MAP["counts"]
    c = torch.zeros(shape, dtype=torch.uint32, device=dxy.device)
    irs.irs_make_map_rows(plan.handle, dxy, dm, band[0], band[1], c)
    plan.sync()
    b = c.cpu().numpy().astype(np.float64)
    sel = a >= 100
    r = (b[sel] - a[sel]) / a[sel]
    return float(np.sqrt(np.mean(r * r))) if sel.any() else None


def brute_band(irs, torch, w, xy, m, dxy, dm, band, plan_fast, n_sms, peak_tflops, fast_value):
    """Brute force over `band` rows: rays/s, its kernel's FP32 fraction, and the
    per-pixel magnification relative RMS of the fast method on the same rays
    (pixels with >= 100 rays)."""
    dev = dxy.device
    shape = (w["npix"], w["npix"])
    pb = irs.Plan(workload_params(irs, "brute", w))
    irs.irs_plan_set_timing(pb.handle, True)
    cb = torch.zeros(shape, dtype=torch.uint32, device=dev)
    ms = []
    for k in range(3):
        cb.zero_()
        irs.irs_make_map_rows(pb.handle, dxy, dm, band[0], band[1], cb)
        t = irs.irs_plan_timings(pb.handle)
        if k:
            ms.append((t.ms_total, t.ms_raypass))
    pb.sync()
    rays = (band[1] - band[0]) * pb.info.n_rays_x
    tot = float(np.mean([a for a, _ in ms]))
    ray = float(np.mean([b for _, b in ms]))
    ach = 10.0 * len(m) * rays / (ray * 1e-3) / 1e12
    cf = torch.zeros(shape, dtype=torch.uint32, device=dev)
    irs.irs_make_map_rows(plan_fast.handle, dxy, dm, band[0], band[1], cf)
    plan_fast.sync()
    a = cb.cpu().numpy().astype(np.float64)
    b = cf.cpu().numpy().astype(np.float64)
    sel = a >= 100
    rel = (b[sel] - a[sel]) / a[sel]
    pb.close()
    value = rays / (tot * 1e-3)
    BRUTE_BAND_MAP["counts"] = a
    return {"value": value, "unit": "rays/s", "band_rows": [int(band[0]), int(band[1])],
            "rays": int(rays), "ms_per_band": tot,
            "roofline": {"bound": "alu", "kernel": "k_brute", "achieved": ach, "peak": peak_tflops,
                         "unit": "TFLOP/s", "frac": ach / peak_tflops},
            "speedup_of_fast_method": fast_value / value,
            "map_rel_rms_vs_brute": float(np.sqrt(np.mean(rel * rel))) if sel.any() else None,
            "pixels_compared": int(sel.sum()), "min_rays_per_pixel": 100}


def cpu_baseline(xy, m, w, target_s=15.0):
    """The FP64 oracle timed on this host's cores on a bounded band of the same
    lattice (all lenses, a few thousand rays)."""
    import oracle
    S = w["S"]
    po = oracle.make_params(w["kappa_star"], w["kappa_s"], w["gamma"], (-S / 2, S / 2, -S / 2, S / 2),
                            w["npix"], w["nav"])
    qo = oracle.size(po)
    cores = os.cpu_count() or 1
    r0 = qo.nry // 2
    rows = cores
    t0 = time.perf_counter()
    probe = 64
    oracle.make_map(po, qo, xy, m, rows=(r0, r0 + rows), cols=(0, probe), threads=cores)
    dt = time.perf_counter() - t0
    cols = int(max(probe, min(qo.nrx, probe * target_s / max(dt, 1e-3))))
    t0 = time.perf_counter()
    oracle.make_map(po, qo, xy, m, rows=(r0, r0 + rows), cols=(0, cols), threads=cores)
    dt = time.perf_counter() - t0
    rays = rows * cols
    return {"value": rays / dt, "unit": "rays/s", "cores": cores, "kind": "oracle",
            "sample": f"{rows} lattice rows x {cols} rays ({rays} rays, all {len(m)} lenses, "
                      f"FP64 brute force) in {dt:.1f} s"}


# ------------------------------------------------------------------ reference arm
def run_reference(args):
    world, rank, local = dist_init()
    if rank != 0:
        return
    import oracle
    from paper_2204_10871_gb300 import lensgen
    w = WORKLOAD
    S = w["S"]
    po = oracle.make_params(w["kappa_star"], w["kappa_s"], w["gamma"], (-S / 2, S / 2, -S / 2, S / 2),
                            w["npix"], w["nav"])
    qo = oracle.size(po)
    xy, m = lens_field(lensgen, (qo.a1, qo.a2, qo.b1, qo.b2), w["seed"])
    cores = os.cpu_count() or 1
    budget = max(20.0, 60.0 / max(1, args.steps + args.warmup))
    r0 = qo.nry // 2
    t0 = time.perf_counter()
    oracle.make_map(po, qo, xy, m, rows=(r0, r0 + cores), cols=(0, 32), threads=cores)
    per_ray = (time.perf_counter() - t0) / (cores * 32)
    cols = int(max(32, min(qo.nrx, budget / max(args.steps + args.warmup, 1) / per_ray)))
    times = []
    for k in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        oracle.make_map(po, qo, xy, m, rows=(r0, r0 + cores), cols=(0, cols), threads=cores)
        dt = time.perf_counter() - t0
        if k >= args.warmup:
            times.append(dt)
    rays = cores * cols
    ms = 1e3 * float(np.mean(times))
    value = rays / (ms * 1e-3)
    print(json.dumps({
        "impl": "reference", "metric": "rays/s per GB300 (" + args.method + ")", "value": value,
        "unit": "rays/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": w["name"], "method": "oracle brute force (FP64, CPU)"},
        "cpu_baseline": {"value": value, "unit": "rays/s", "cores": cores, "kind": "oracle",
                         "sample": f"{cores} lattice rows x {cols} rays per step, all lenses"},
        "e2e": {"value": value, "unit": "rays/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--method", default="interp", choices=["interp", "brute", "mlp"])
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-brute", action="store_true", help="skip the brute-force band")
    ap.add_argument("--no-tune", action="store_true", help="paper-rule cells, default ray pass")
    ap.add_argument("--variant", type=int, default=-1, help="fixed kernel variant (skips tuning)")
    ap.add_argument("--workload", default="", choices=["", "paper-mid", "high-res", "learned"],
                    help="default: paper-mid (learned for --method mlp)")
    ap.add_argument("--band-rows", type=int, default=0, help="brute band height (rows)")
    ap.add_argument("--n-star", type=int, default=0, help="override the lens count (profiling)")
    ap.add_argument("--npix", type=int, default=0, help="override the map side (profiling)")
    ap.add_argument("--nav", type=float, default=0.0, help="override rays per pixel (profiling)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
